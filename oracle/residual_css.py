"""Online column subset selection by residual-based sampling (the paper's Algorithm 1, reviewed in
Sec. 2.2.1 from Bhaskara et al.): the comparison selector of the accuracy tables.

Test infrastructure (see ``oracle/__init__``): a plain FP64 restatement, one column at a time.

For each arriving column a (global index j):

* p_a = k ||Pi_perp a||^2 / xi, where Pi_perp projects onto the orthogonal complement of the span
  of the previously selected columns C_pre (the residual is formed explicitly here,
  a - Q (Q^T a) with Q an orthonormal basis of that span);
* a joins C_cur with probability min(p_a, 1): u_j < min(p_a, 1) with u_j the 53-bit uniform of
  Philox((j mod 2^32, j >> 32, TAG_RCSS, 0)) (words 0 and 1, as every uniform of this project);
* if p_a < 1, the residual mass sigma grows by p_a;
* if p_a >= 1 or sigma >= 1, C_pre takes C_cur's columns, sigma = 0 and C_cur is emptied.

The selection is C_pre followed by C_cur, in order of arrival.  With ``limit`` set, the selection
stops growing at ``limit`` columns, the treatment of the experiments (Sec. 4.1: the subset is
expanded only until k columns are selected); reading: a column whose keep decision comes after
that is not added, and p, sigma and the steps go on as before.  Reading (the paper is silent):
the basis Q of span(C_pre) grows by each column of C_cur in order, orthogonalized against the
basis so far; a column whose residual norm is at most RANK_TOL times its norm adds no direction
(it lies in the span numerically) but stays in the selection.

Parity: pinned by tests/test_oracle_pins.py (greedy limit for tiny xi against a brute-force rank
count, no selection for huge xi, selection frequency of the first column over seeds, exact
recovery of a rank-r stream, the bookkeeping of sigma on a hand-checked sequence).
"""
import numpy as np

from . import philox

TAG_RCSS = 0x52435331        # 'RCS1'
RANK_TOL = 1e-12


def uniform(seed, j):
    """u_j: the uniform behind the keep decision of column j."""
    k0, k1 = philox.seed_key(seed)
    w = philox.philox4x32(np.uint64(j & 0xFFFFFFFF), np.uint64(j >> 32), TAG_RCSS, 0, k0, k1)
    return float(philox.uniform53(w[0], w[1]))


def probability(a, Q, k, xi):
    """p_a = k ||Pi_perp a||^2 / xi with Pi_perp = I - Q Q^T (Q orthonormal columns), the residual
    a - Q (Q^T a) formed explicitly."""
    res = a - Q @ (Q.T @ a)
    return k * float(res @ res) / xi


def replay(p, seed, limit=None):
    """The decisions of Algorithm 1 for a given sequence of p (the bookkeeping alone: keep draws,
    sigma, steps, the limit): (selection, sigma, steps)."""
    o = ResidualCSS(1, 1, 1.0, seed, limit)
    for pj in p:
        o._decide(float(pj), None)
    return o.selection(), o.sigma, o.steps


class ResidualCSS:
    """Algorithm 1 over a stream of m-vectors."""

    def __init__(self, m, k, xi, seed=0, limit=None):
        if not xi > 0:
            raise ValueError("xi must be positive")
        self.m, self.k, self.xi, self.seed, self.limit = m, k, float(xi), seed, limit
        self.Q = np.zeros((m, 0))
        self.pre = []               # indices of C_pre
        self.cur = []               # indices of C_cur
        self.cur_cols = []
        self.sigma = 0.0
        self.n_obs = 0
        self.p = []                 # p_a of every column, in order (for tests)
        self.steps = []             # columns after which C_pre was updated

    def ingest(self, A):
        A = np.asarray(A, dtype=np.float64)
        for q in range(A.shape[1]):
            self._column(A[:, q])

    def _column(self, a):
        self._decide(probability(a, self.Q, self.k, self.xi), a)

    def _decide(self, p, a):
        """Steps 5-11 of the loop for column j = n_obs with probability p (a = None: bookkeeping
        only, the basis is not grown)."""
        j = self.n_obs
        self.p.append(p)
        full = self.limit is not None and len(self.pre) + len(self.cur) >= self.limit
        if uniform(self.seed, j) < min(p, 1.0) and not full:
            self.cur.append(j)
            self.cur_cols.append(None if a is None else a.copy())
        if p < 1.0:
            self.sigma += p
        if p >= 1.0 or self.sigma >= 1.0:
            for c in self.cur_cols:
                if c is not None:
                    self._extend(c)
            self.pre += self.cur
            self.cur, self.cur_cols = [], []
            self.sigma = 0.0
            self.steps.append(j)
        self.n_obs += 1

    def _extend(self, c):
        r = c - self.Q @ (self.Q.T @ c)
        r = r - self.Q @ (self.Q.T @ r)            # a second projection (twice is enough)
        nr = np.linalg.norm(r)
        if nr > RANK_TOL * np.linalg.norm(c):
            self.Q = np.hstack([self.Q, (r / nr)[:, None]])

    def selection(self):
        return np.array(self.pre + self.cur, dtype=np.int64)
