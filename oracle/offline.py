"""Offline reference quantities (multi-pass), used to pin and to score the streaming method.

Test infrastructure (see ``oracle/__init__``).

* ``cpqr_id``: Sec. 2.1, Eqs. 5-11 -- A Z = Q R, J = first k pivots,
  P = [I_k, R11^{-1} R12] Z^T.  Ties between pivots follow the library's
  column-pivoted QR (LAPACK geqp3).
* ``ridge_leverage_scores``: Eq. 16, tau_j = a_j^T (A A^T + lambda I)^+ a_j.
* ``truncated_svd_error`` and ``tail_energy``: ||A - A_k||_F from the SVD
  (Eckart-Young, Eq. 1).
* ``hutchinson_trace`` (Eq. 33) and ``na_hutchpp_trace`` (Eqs. 34-35) on an
  explicit square matrix B, for pinning the sketch-only form of Eq. 37.
"""
import numpy as np
import scipy.linalg


def cpqr_id(A, k):
    """Column ID from column-pivoted QR (Eqs. 5-11); returns (J, P) with A ~ A[:, J] P."""
    Q, R, piv = scipy.linalg.qr(A, mode="economic", pivoting=True)
    n = A.shape[1]
    T = scipy.linalg.solve_triangular(R[:k, :k], R[:k, k:], lower=False)
    P = np.zeros((k, n))
    P[:, piv[:k]] = np.eye(k)
    P[:, piv[k:]] = T
    return piv[:k].copy(), P


def tail_energy(A, k):
    """||A - A_k||_F^2 (Eckart-Young)."""
    sv = np.linalg.svd(A, compute_uv=False)
    return float(np.sum(sv[k:] ** 2))


def truncated_svd_error(A, k):
    """Relative Frobenius error of the best rank-k approximation."""
    return float(np.sqrt(tail_energy(A, k)) / np.linalg.norm(A))


def ridge_leverage_scores(A, lam):
    """Eq. 16 for every column of A."""
    m = A.shape[0]
    M = A @ A.T + lam * np.eye(m)
    X = np.linalg.pinv(M) @ A
    return np.einsum("ij,ij->j", A, X)


def id_error(A, J, P):
    """Exact ||A - A_J P||_F (empty slots, index < 0, contribute nothing)."""
    J = np.asarray(J)
    act = J >= 0
    R = A - A[:, J[act]] @ P[act]
    return float(np.linalg.norm(R))


def hutchinson_trace(B, Om):
    """Eq. 33: tr(B) ~ tr(Omega B Omega^T) / ell."""
    return float(np.trace(Om @ B @ Om.T) / Om.shape[0])


def na_hutchpp_trace(B, Om1, Om2, Om3, rcond=None):
    """Eqs. 34-35 on an explicit B: B~ = (Om2 B)^T (Om1 B Om2^T)^+ (Om1 B), debiased by Om3."""
    X = Om1 @ B @ Om2.T
    if rcond is None:
        rcond = max(X.shape) * np.finfo(np.float64).eps
    Xp = np.linalg.pinv(X, rcond=rcond)
    Bt = (Om2 @ B).T @ Xp @ (Om1 @ B)
    return float(np.trace(Bt) + (np.trace(Om3 @ B @ Om3.T) - np.trace(Om3 @ Bt @ Om3.T)) / Om3.shape[0])
