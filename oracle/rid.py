"""FP64 restatement of the single-pass randomized ID (Algorithm 3 with Algorithms 4-8).

Test infrastructure (see ``oracle/__init__``).  Plain numpy, no blocking, no
fusion; each step follows the paper's order and notation.  Library primitives
used as single steps: ``solve``, ``lstsq``, ``pinv``, ``qr``, ``eigvalsh``.

Readings where the paper is silent, ambiguous or at odds with itself:

R1  Omega scale.  Omega has unit-variance entries (``randn`` in Algorithm 3);
    every quantity that meets unsketched data uses the scaled sketch
    S~ = Omega A / sqrt(s), so that ||S~_k||_F^2 is comparable with
    ||A_obs||_F^2 in Eq. 23 and Y of Algorithm 5 approximates A_J^T A_obs.
R2  lambda = (||A_obs||^2 - ||S~_k||^2)/k is floored at 1e-12 ||A_obs||^2/k;
    a fixed lambda may be given instead (for example ||A - A_k||^2/k).
R3  Eq. 23 uses (S~S~^T + lambda I)^{-1} when lambda > 0, the pseudo-inverse
    otherwise.
R4  The left sketch has s rows; the Hutch++ probes are h further independent
    rows of the same generator, split contiguously into floor(c1 h),
    floor(c2 h) and the rest (Omega_1, Omega_2, Omega_3 of Sec. 3.3).  h = 0
    selects the paper-literal shared mode: the split is taken from the s left
    rows themselves.
R6  Every column is appended to D and to ||A_obs||^2 first; the batch step runs
    when count reaches t (the literal if/else skips every (t+1)-th column).
R7  Refill: candidates r = 1..count are scanned in order; the first success
    whose column is not already in C fills the slot; probabilities are
    clipped to [0, 1]; a slot dropped in iteration i is refilled in the same
    iteration.  u < p means success.
R7p (alternative, ``refill="proportional"``): the same scan decides whether
    slot i is refilled; the column it takes is then drawn among the buffered
    columns not already in C with probability tau^D_r / sum tau^D (Sec. 2.3
    reads the normalized ridge score as the selection probability): one more
    uniform u(batch, i, count + 1) is compared with the running sums of the
    scores, added in column order.  With the refill probabilities of R8 every
    p is clipped to 1 on the benchmark streams, so R7 takes the first columns
    of each batch while R7p spreads the choice by score.
R8  c = 1 and natural logarithms in the refill probability.
R9  After the last column, a batch step runs over the count < t buffered
    columns (finalize).
R10 Algorithms 6 and 7 need P_prev for columns observed since the last batch
    step; those columns take the preliminary estimate P_4 (Sec. 3.2.1 computes
    Algorithm 4 every batch for exactly this use).  For Algorithm 7 the new
    columns are copied after the transform.
R10b Algorithm 6 solves the residual least-squares problem for the rows of the
    new basis elements only, as the prose of Sec. 3.2.3 describes it (old rows
    keep their coefficients, new rows are fitted to the residual).  Solving over all of A_J, as the
    listing reads, gives P_prev + (Omega A_J)^+(Omega A - Omega A_J P_prev)
    = (Omega A_J)^+ Omega A, i.e. Algorithm 4 again whenever Omega A_J has full
    column rank, whereas the paper's tables report different errors for the two.
R11 Empty slots (index -1) are left out of Algorithms 4-8; their rows of P are 0.
R12 G^{-1} in Algorithm 5 is the pseudo-inverse (Eq. 25 writes A_J^+).
R13 The pseudo-inverse in Eq. 37 uses rcond = max(c1 h, c2 h) * eps64.
R14 The estimate of ||A - A_J P||_F^2 is reported signed; the error is
    sqrt(max(e2, 0)).  q* = argmin over the signed estimates.
R15 Ties in the argmin go to the lowest q.
R16 Gradient mode (Sec. 3.4): the ridge scores use the sketch of [a; G a],
    computed as Omega a + Omega_g (G a) with an independent Omega_g, and the
    squared norm ||a||^2 + ||G a||^2; coefficients and the error estimate use
    the plain sketch Omega a.
R19 Indices are 0-based; -1 marks an empty slot.

The optional right sketch Y = sum_j a_j omega_j^T (m x l, unit-variance omega_j of l entries
keyed by the snapshot index j) is not part of the paper's method; it is kept beside the
stream when ``right_l`` > 0 (``right_sketch`` gives it for a whole matrix).
"""
from dataclasses import dataclass, field
import math

import numpy as np

from . import gcv as gcv_mod
from . import philox

EPS64 = np.finfo(np.float64).eps


@dataclass
class RIDConfig:
    m: int
    k: int                      # target rank; the basis size t equals k (Sec. 2.2.2)
    s: int                      # left-sketch rows (ell of Algorithm 3)
    h: int = 0                  # independent Hutch++ probe rows (R4)
    c1: float = 1.0 / 6.0
    c2: float = 1.0 / 3.0
    eps: float = 0.5
    delta: float = 0.05
    c_const: float = 1.0
    lambda_mode: str = "streaming"     # or "fixed"
    lambda_fixed: float = 0.0
    omega_kind: str = "rademacher"     # or "gaussian"
    seed: int = 0
    grad_op: object = None             # sparse (d*m) x m simplex-gradient operator, Eq. 42
    right_l: int = 0                   # columns of the optional right sketch Y (0: off)
    grad_coeff: bool = False           # keep Omega G^p a for the gradient-augmented coefficients
    refill: str = "first"              # R7 ("first") or R7p ("proportional")
    selector: str = "ridge"            # "ridge" (Algorithm 3) or "residual" (Algorithm 1, below)
    rcss_xi: float = 1.0               # xi of Algorithm 1 when selector == "residual"
    rcss_seed: int = 0                 # seed of Algorithm 1's uniforms

    @property
    def t(self):
        return self.k

    def probe_split(self):
        """Row ranges (start, stop) of Omega_1, Omega_2, Omega_3 inside the sketch (R4)."""
        if self.h > 0:
            base, n = self.s, self.h
        else:
            base, n = 0, self.s
        n1 = int(math.floor(self.c1 * n))
        n2 = int(math.floor(self.c2 * n))
        return ((base, base + n1), (base + n1, base + n1 + n2), (base + n1 + n2, base + n))


def refill_scale(cfg):
    """c (k log k + k log(1/delta)/eps) / t, the factor of tau^D in Algorithm 3's refill."""
    k = cfg.k
    return cfg.c_const * (k * math.log(k) + k * math.log(1.0 / cfg.delta) / cfg.eps) / cfg.t


def right_sketch(A, l, kind, seed):
    """Y = A W, W[j, r] = omega_j[r]: the right sketch of the m x n matrix A (all columns)."""
    n = A.shape[1]
    W = philox.omega_block(kind, seed, np.arange(l), 0, n, right=True).T     # n x l
    return A @ W


def streaming_lambda(SSt_scaled, fro2, k):
    """(||A_obs||^2 - ||S~_k||^2)/k of Eq. 23, floored as in R2."""
    mu = np.linalg.eigvalsh(SSt_scaled)[::-1]
    lam = (fro2 - mu[:k].sum()) / k
    return max(lam, 1e-12 * fro2 / k)


def sketched_ridge_scores(SSt_scaled, lam, V):
    """Eq. 23: tau_i = v_i^T (S~S~^T + lambda I)^+ v_i for the scaled sketch columns V."""
    M = SSt_scaled + lam * np.eye(SSt_scaled.shape[0])
    if lam > 0:
        X = np.linalg.solve(M, V)
    else:
        X = np.linalg.pinv(M) @ V
    return np.einsum("ij,ij->j", V, X)


def css_update(cfg, batch, JC, tau_old, tau_C, JD, tau_D, margins=None, target=None, flips=None):
    """Prune and refill the basis slots (Algorithm 3, following Cohen et al.; R7, R8).

    JC, tau_old are updated copies; tau_C are min(tau_old, scores of C) for the
    occupied slots; JD, tau_D the buffered columns and their scores.  If
    ``margins`` is a list, the relative distance of every decision's score
    from the score at which that decision would flip is appended to it.

    Re-synchronisation (test use only): with ``target`` (the slot contents another
    implementation chose at this step) each slot whose outcome differs from target's
    takes target's outcome before the next slot is decided, and (slot, kind, margin)
    of the decision that differed is appended to ``flips`` -- kind "prune" for the
    keep-or-prune draw, "refill" for the first buffered column whose acceptance draw
    went the other way, "draw" for R7p's proportional pick.  The decisions of the
    later slots are then taken on the same state as target's.
    """
    JC = JC.copy()
    tau_old = tau_old.copy()
    scale = refill_scale(cfg)
    for i in range(cfg.t):
        old = int(JC[i])
        prune_margin = None
        if JC[i] >= 0:
            u = float(philox.uniform(cfg.seed, batch, i, 0))
            if tau_C[i] > 0:
                prune_margin = abs(u - (1.0 - tau_C[i] / tau_old[i])) * tau_old[i] / tau_C[i]
                if margins is not None:
                    margins.append(prune_margin)
            if u < 1.0 - tau_C[i] / tau_old[i]:
                JC[i] = -1
                tau_old[i] = 1.0
            else:
                tau_old[i] = tau_C[i]
        kept = JC[i] >= 0
        tgt_kept = target is not None and old >= 0 and int(target[i]) == old
        if target is not None and old >= 0 and kept != tgt_kept:
            # the keep-or-prune draw of slot i went the other way in target
            flips.append((i, "prune", prune_margin if prune_margin is not None else 0.0))
            if tgt_kept:
                JC[i] = old
                tau_old[i] = tau_C[i]
            else:
                JC[i] = -1
                tau_old[i] = 1.0
                kept = False
        if not kept:
            hit = None
            rmargins = []
            for r in range(len(JD)):
                p = min(max(tau_D[r] * scale, 0.0), 1.0)
                u = float(philox.uniform(cfg.seed, batch, i, 1 + r))
                rm = abs(u - p) / p if (p < 1.0 and tau_D[r] > 0) else float("inf")
                if margins is not None and p < 1.0 and tau_D[r] > 0:
                    margins.append(rm)
                rmargins.append(rm)
                if u < p and JD[r] not in JC:
                    hit = r
                    break
            first = hit
            dmargins = [] if flips is not None else margins
            cand = [r for r in range(len(JD)) if JD[r] not in JC]      # R7p's candidates, in order
            if hit is not None and cfg.refill == "proportional":
                hit = proportional_draw(cfg, batch, i, JC, JD, tau_D, hit, dmargins)
                if margins is not None and dmargins is not margins:
                    margins.extend(dmargins)
            if hit is not None:
                JC[i] = JD[hit]
                tau_old[i] = tau_D[hit]
            if target is not None and int(JC[i]) != int(target[i]):
                want = int(target[i])
                if want >= 0 and want not in JD:
                    raise ValueError(f"target slot {i} holds column {want}, neither kept nor buffered at step {batch}")
                rt = JD.index(want) if want in JD else None
                if cfg.refill == "proportional" and first is not None and rt is not None:
                    # both accepted a refill; the pick went the other way at the boundary of the
                    # cumulative scores between the two picks
                    kb = min(cand.index(hit), cand.index(rt)) if (hit in cand and rt in cand) else 0
                    flips.append((i, "draw", dmargins[kb] if kb < len(dmargins) else 0.0))
                else:
                    # the first buffered column whose acceptance draw differs from target's
                    cut = min(x for x in (first, rt) if x is not None) if (first is not None or rt is not None) else 0
                    flips.append((i, "refill", rmargins[cut] if cut < len(rmargins) else 0.0))
                JC[i] = want
                tau_old[i] = tau_D[rt] if rt is not None else 1.0
    return JC, tau_old


def proportional_draw(cfg, batch, i, JC, JD, tau_D, fallback, margins=None):
    """R7p: the buffered column r (not already in C) with probability tau^D_r / sum tau^D,
    by inverse CDF on u(batch, i, count + 1) over the scores summed in column order."""
    cand = [r for r in range(len(JD)) if JD[r] not in JC]
    total = 0.0
    for r in cand:
        total += max(float(tau_D[r]), 0.0)
    if not total > 0.0:
        return fallback
    x = float(philox.uniform(cfg.seed, batch, i, 1 + len(JD))) * total
    run = 0.0
    pick = None
    for r in cand:
        run += max(float(tau_D[r]), 0.0)
        if margins is not None:
            margins.append(abs(x - run) / total)
        if pick is None and x < run:
            pick = r
    return pick if pick is not None else cand[-1]


def coeff_alg4(SJ, SA):
    """Algorithm 4, Eq. 24: P = (Omega A_J)^+ (Omega A_obs)."""
    return np.linalg.lstsq(SJ, SA, rcond=None)[0]


def coeff_alg5(G, SJ, SA):
    """Algorithm 5: G = A_J^T A_J, Y = (Omega A_J)^T (Omega A_obs) (scaled sketch, R1), P = G^{-1} Y.

    G^{-1} is taken as the pseudo-inverse G^+ (R12): Eq. 25 writes the same
    estimate as A_J^+ Omega^T Omega A = (A_J^T A_J)^+ A_J^T Omega^T Omega A,
    which stays defined when A_J is rank deficient.
    """
    return np.linalg.pinv(G, hermitian=True) @ (SJ.T @ SA)


def coeff_alg6(SJ, SA, P_prev_ext, kept):
    """Algorithm 6, Eqs. 27-30 with the new-basis-rows reading R10b."""
    Pp = P_prev_ext * kept[:, None]              # Eq. 27: zero the rows of replaced columns
    rA = SA - SJ @ Pp                            # Eq. 28: residual of the unchanged basis
    dP = np.zeros_like(Pp)
    new = ~kept
    if new.any():
        dP[new] = np.linalg.lstsq(SJ[:, new], rA, rcond=None)[0]   # Eq. 29 on the new rows
    return Pp + dP                               # Eq. 30


def coeff_alg7(AJ, AJprev, P_prev):
    """Algorithm 7, Eqs. 31-32: A_J = QR, T = R^+ Q^T A_Jprev, P = T P_prev."""
    Q, R = np.linalg.qr(AJ)
    T = np.linalg.pinv(R) @ (Q.T @ AJprev)
    return T @ P_prev


def na_hutchpp_sq_error(H, HJ, P, G, fro2, split, rcond=None):
    """Algorithm 8: estimate ||A_obs - A_J P||_F^2 from sketches only (Eqs. 36-37).

    H  : probe sketch Omega A_obs of all observed columns (unit-variance rows)
    HJ : the same rows restricted to the basis columns, Omega A_J
    P  : coefficients over the active basis columns
    G  : A_J^T A_J
    split : row ranges of Omega_1, Omega_2, Omega_3 inside H (relative to H)
    """
    (a1, b1), (a2, b2), (a3, b3) = split
    O1A, O2A, O3A = H[a1:b1], H[a2:b2], H[a3:b3]
    O2AJP = HJ[a2:b2] @ P
    O3AJP = HJ[a3:b3] @ P
    n1, n2, n3 = b1 - a1, b2 - a2, b3 - a3
    if n1 > 0 and n2 > 0:
        X = O1A @ O2AJP.T                           # Omega_1 A (Omega_2 A_J P)^T
        if rcond is None:
            rcond = max(n1, n2) * EPS64
        Xp = np.linalg.pinv(X, rcond=rcond)
        term1 = np.trace(Xp @ (O1A @ P.T) @ G @ (O2A @ P.T).T)
        corr = np.trace(O3AJP @ O2A.T @ Xp @ O1A @ O3AJP.T)
    else:                                           # plain Hutchinson, Eq. 33
        term1, corr = 0.0, 0.0
    direct = np.trace(O3A @ O3AJP.T)
    cross = term1 + (direct - corr) / n3            # Eq. 37
    return fro2 - 2.0 * cross + np.trace(G @ P @ P.T)   # Eq. 36


@dataclass
class BatchRecord:
    batch: int
    n_obs: int
    lam: float
    JC: np.ndarray
    est_sq: np.ndarray          # signed estimates for q = 4..7
    q_star: int
    kept: np.ndarray = field(default=None)


class OnlineRID:
    """Streaming state of Algorithm 3.  Feed columns with ``ingest``; call ``finalize`` at the end."""

    def __init__(self, cfg: RIDConfig):
        self.cfg = cfg
        t, s, h = cfg.t, cfg.s, cfg.h
        self.rows = s + h
        self.n_obs = 0
        self.fro2 = 0.0                 # ||A_obs||_F^2
        self.fro2_lev = 0.0             # ||[A_obs; G A_obs]||_F^2 in gradient mode (R16)
        self.S = np.zeros((self.rows, 0))           # Omega A_obs, unit-variance rows
        self.S_lev = np.zeros((s, 0))               # sketch used by the ridge scores
        self.SSt = np.zeros((s, s))                 # S_lev S_lev^T (unscaled)
        self.cols = {}                              # global index -> column, for C and D
        self.JC = -np.ones(t, dtype=np.int64)
        self.JC_prev = -np.ones(t, dtype=np.int64)
        self.tau_old = np.ones(t)
        self.JD = []
        self.P = np.zeros((t, 0))
        self.batch = 0
        self.history = []
        self._omega = None
        self._omega_g = None
        self.margins = []
        self.resync = None          # test use: {batch: slot contents to re-synchronise to}
        self.flips = []             # (batch, slot, kind, margin) of the decisions re-synchronised
        self.Y = np.zeros((cfg.m, cfg.right_l)) if cfg.right_l > 0 else None
        self.SG = None                              # d x s x n_obs: Omega G^p A_obs (unit variance)
        # The online rows of the paper's tables with Algorithm 1 as the selector (Sec. 4.1):
        # Algorithm 1 decides each column as it arrives, its subset capped at t columns; each batch
        # step puts the columns it kept from the batch into the empty slots in order (it never
        # drops one) and computes Algorithms 4-8 for that basis as for Algorithm 3's.
        self.rcss = None
        if cfg.selector == "residual":
            from .residual_css import ResidualCSS
            self.rcss = ResidualCSS(cfg.m, cfg.k, cfg.rcss_xi, cfg.rcss_seed, limit=t)

    # Omega is materialized once: this is the slow, obviously correct form.
    def omega(self):
        if self._omega is None:
            c = self.cfg
            self._omega = philox.omega_block(c.omega_kind, c.seed, np.arange(self.rows), 0, c.m)
        return self._omega

    def omega_g(self):
        if self._omega_g is None:
            c = self.cfg
            dm = c.grad_op.shape[0]
            self._omega_g = philox.omega_block(c.omega_kind, c.seed, np.arange(c.s), 0, dm, grad=True)
        return self._omega_g

    def ingest(self, A):
        """Read columns one at a time (Algorithm 3); A is m x b (or a single m-vector)."""
        A = np.asarray(A, dtype=np.float64)
        if A.ndim == 1:
            A = A[:, None]
        for j in range(A.shape[1]):
            self._ingest_one(A[:, j].copy())

    def _ingest_one(self, a):
        c = self.cfg
        j = self.n_obs
        if self.rcss is not None:
            self.rcss.ingest(a[:, None])
        s_j = self.omega() @ a                               # s_j = Omega a_j
        self.S = np.concatenate([self.S, s_j[:, None]], axis=1)
        lev = s_j[: c.s].copy()
        fro_lev = a @ a
        if c.grad_op is not None:                            # R16: sketch of [a; G a]
            ga = c.grad_op @ a
            lev = lev + self.omega_g() @ ga
            fro_lev += ga @ ga
        self.S_lev = np.concatenate([self.S_lev, lev[:, None]], axis=1)
        self.SSt += np.outer(lev, lev)                       # SS^T <- SS^T + s_j s_j^T
        if c.grad_coeff:                                     # Omega G^p a_j for Sec. 3.4's coefficients
            Gs = gcv_mod.split_gradient(c.grad_op, c.m)
            col = np.stack([self.omega()[: c.s] @ (Gp @ a) for Gp in Gs])[:, :, None]
            self.SG = col if self.SG is None else np.concatenate([self.SG, col], axis=2)
        if c.right_l > 0:                                    # Y <- Y + a_j omega_j^T
            w = philox.omega_block(c.omega_kind, c.seed, np.arange(c.right_l), j, j + 1, right=True)[:, 0]
            self.Y += np.outer(a, w)
        self.cols[j] = a                                     # d_count = a_j (R6)
        self.JD.append(j)
        self.fro2 += a @ a
        self.fro2_lev += fro_lev
        self.n_obs += 1
        if len(self.JD) == c.t:
            self.batch_step()

    def finalize(self):
        """Run the tail batch step (R9) and return (J, P)."""
        if self.JD:
            self.batch_step()
        return self.JC.copy(), self.P.copy()

    def gradient_coefficients(self, lo=-3.0, hi=3.0, tol=1e-3):
        """Sec. 3.4's gradient-augmented coefficients for the final basis, lambda by the
        sketched GCV (``oracle.gcv``): returns (lambda*, P (t x n, rows of empty slots 0),
        GCV(lambda*))."""
        c = self.cfg
        s = c.s
        act = np.nonzero(self.JC >= 0)[0]
        Jact = self.JC[act]
        S = self.S[:s] / math.sqrt(s)
        G = [self.SG[p] / math.sqrt(s) for p in range(self.SG.shape[0])]
        Om = self.omega()[:s]
        K = [Om @ (Gp @ Om.T) / s for Gp in gcv_mod.split_gradient(c.grad_op, c.m)]
        lam, Pa, g = gcv_mod.gradient_coefficients(S[:, Jact], S, [x[:, Jact] for x in G], G, K, lo, hi, tol)
        P = np.zeros((c.t, self.n_obs))
        P[act] = Pa
        return lam, P, g

    def batch_step(self):
        c = self.cfg
        t, s = c.t, c.s
        n = self.n_obs
        SSt_scaled = self.SSt / s
        lam_fro = self.fro2_lev if c.grad_op is not None else self.fro2
        if c.lambda_mode == "fixed":
            lam = c.lambda_fixed
        else:
            lam = streaming_lambda(SSt_scaled, lam_fro, c.k)

        # ApproximateRidgeScores_Sketch for C and D (Eq. 23 on the scaled sketch, R1)
        Vlev = self.S_lev / math.sqrt(s)
        occ = self.JC >= 0
        tau_C = np.ones(t)
        if occ.any():
            sc = sketched_ridge_scores(SSt_scaled, lam, Vlev[:, self.JC[occ]])
            tau_C[occ] = np.minimum(self.tau_old[occ], sc)
        JD = list(self.JD)
        tau_D = sketched_ridge_scores(SSt_scaled, lam, Vlev[:, JD])
        JC_prev = self.JC.copy()
        target = self.resync.get(self.batch) if self.resync else None
        flips = [] if target is not None else None
        if self.rcss is not None:
            JC, tau_old = self.JC.copy(), self.tau_old.copy()
            new = [int(j) for j in self.rcss.selection() if JD and JD[0] <= j <= JD[-1]]
            free = [i for i in range(t) if JC[i] < 0]
            for i, j in zip(free, new):
                JC[i] = j
        else:
            JC, tau_old = css_update(c, self.batch, self.JC, self.tau_old, tau_C, JD, tau_D, self.margins, target,
                                     flips)
        if flips:
            self.flips.extend((self.batch,) + f for f in flips)

        # Coefficient candidates over the active slots (R11)
        act = np.nonzero(JC >= 0)[0]
        Jact = JC[act]
        SA = self.S[:s] / math.sqrt(s)
        SJ = SA[:, Jact]
        AJ = np.stack([self.cols[j] for j in Jact], axis=1) if len(act) else np.zeros((c.m, 0))
        G = AJ.T @ AJ
        n_prev = self.P.shape[1]
        cand = []
        P4a = coeff_alg4(SJ, SA)
        cand.append(P4a)
        cand.append(coeff_alg5(G, SJ, SA))
        kept = JC[act] == JC_prev[act]
        P_prev_ext = np.zeros((len(act), n))
        P_prev_ext[:, :n_prev] = self.P[act, :]
        P_prev_ext[:, n_prev:] = P4a[:, n_prev:]               # R10
        cand.append(coeff_alg6(SJ, SA, P_prev_ext, kept))
        pact = np.nonzero(JC_prev >= 0)[0]
        P7a = np.zeros((len(act), n))
        if len(pact):
            AJprev = np.stack([self.cols[j] for j in JC_prev[pact]], axis=1)
            P7a[:, :n_prev] = coeff_alg7(AJ, AJprev, self.P[pact, :])
        P7a[:, n_prev:] = P4a[:, n_prev:]                       # R10
        cand.append(P7a)

        # Algorithm 8 for each candidate, then q* = argmin (R14, R15)
        split = c.probe_split()
        base = split[0][0]
        H = self.S[base: split[2][1]]
        rel = tuple((a - base, b - base) for a, b in split)
        HJ = H[:, Jact]
        est = np.array([na_hutchpp_sq_error(H, HJ, Pq, G, self.fro2, rel) for Pq in cand])
        qi = int(np.argmin(est))

        P = np.zeros((t, n))
        P[act] = cand[qi]
        self.P = P
        self.JC_prev = JC.copy()
        self.JC = JC
        self.tau_old = tau_old
        self.history.append(BatchRecord(self.batch, n, lam, JC.copy(), est, 4 + qi, kept))
        self.batch += 1
        self.JD = []
        keep = set(int(j) for j in JC if j >= 0)
        self.cols = {j: v for j, v in self.cols.items() if j in keep}
        self._last_candidates = cand
        self._last_active = act

    def error_estimates(self):
        """(signed estimates of ||A - A_J P||^2 for q = 4..7, q*) of the last batch step."""
        r = self.history[-1]
        return r.est_sq.copy(), r.q_star
