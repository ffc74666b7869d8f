"""Gradient-augmented coefficients with a sketched GCV choice of lambda (Sec. 3.4).

Test infrastructure (see ``oracle/__init__``).  Plain numpy, following the paper's order:

* Eq. (augmented least squares, full sketching): for the final basis J,
      P(lam) = argmin_X ||S~_J X - S~||_F^2 + lam sum_p ||G~_J^p X - G~^p||_F^2,
  S~ = Omega A / sqrt(s), G~^p = Omega G^p A / sqrt(s) (the left-sketch rows of Omega, unit
  variance; the 1/sqrt(s) scale of reading R1), _J = the basis columns.
* The sketched GCV function
      GCV(lam) = ||(I - C(lam)) S~||_F^2 / tr(I - C(lam))^2,
      C(lam) = S~_J (S~_J^T S~_J + lam sum_p G~_J^p^T G~_J^p)^{-1}
               (S~_J + lam sum_p (K^p)^T G~_J^p)^T,   K^p = Omega G^p Omega^T / s,
  evaluated from its definition (the s x s matrix C is formed).
* lam* = the golden-section minimiser of GCV over [1e-3, 1e3] at the end of the stream.

Readings: the search runs on log10(lam) in [-3, 3] (the range spans six
decades) with golden ratio steps until the bracket is narrower than 1e-3 in log10(lam), and
returns the midpoint of the last bracket; GCV of a candidate is compared with plain "<" (ties
keep the left probe); the gradient operators G^p are those of ``oracle.gradient`` (one-sided at
the boundary); Omega is the left sketch of the stream (its first s rows).
"""
import math

import numpy as np

INV_PHI = (math.sqrt(5.0) - 1.0) / 2.0     # 1 / golden ratio


def split_gradient(grad_op, m):
    """The d blocks G^1 .. G^d (each m x m) of the stacked (d m) x m operator."""
    d = grad_op.shape[0] // m
    return [grad_op[p * m:(p + 1) * m] for p in range(d)]


def p_of_lambda(SJ, S, GJ, G, lam):
    """The full-sketch augmented least-squares solution, by its normal equations."""
    M = SJ.T @ SJ + lam * sum(g.T @ g for g in GJ)
    R = SJ.T @ S + lam * sum(gj.T @ ga for gj, ga in zip(GJ, G))
    return np.linalg.solve(M, R)


def c_matrix(SJ, GJ, K, lam):
    """C(lam) of the sketched GCV function (s x s)."""
    M = SJ.T @ SJ + lam * sum(g.T @ g for g in GJ)
    W = SJ + lam * sum(k.T @ g for k, g in zip(K, GJ))
    return SJ @ np.linalg.solve(M, W.T)


def gcv(SJ, S, GJ, K, lam):
    s = SJ.shape[0]
    C = c_matrix(SJ, GJ, K, lam)
    R = S - C @ S
    return float(np.sum(R * R) / (s - np.trace(C)) ** 2)


def golden_section(f, lo=-3.0, hi=3.0, tol=1e-3):
    """Minimiser of a unimodal f on [lo, hi] by golden-section search (returns the midpoint of
    the final bracket, narrower than tol); f is evaluated once per probe point."""
    a, b = lo, hi
    x1 = b - INV_PHI * (b - a)
    x2 = a + INV_PHI * (b - a)
    f1, f2 = f(x1), f(x2)
    while b - a > tol:
        if f1 < f2:
            b, x2, f2 = x2, x1, f1
            x1 = b - INV_PHI * (b - a)
            f1 = f(x1)
        else:
            a, x1, f1 = x1, x2, f2
            x2 = a + INV_PHI * (b - a)
            f2 = f(x2)
    return 0.5 * (a + b)


def gradient_coefficients(SJ, S, GJ, G, K, lo=-3.0, hi=3.0, tol=1e-3):
    """(lam*, P(lam*), GCV(lam*)) for scaled sketches (see the module docstring)."""
    x = golden_section(lambda t: gcv(SJ, S, GJ, K, 10.0 ** t), lo, hi, tol)
    lam = 10.0 ** x
    return lam, p_of_lambda(SJ, S, GJ, G, lam), gcv(SJ, S, GJ, K, lam)
