"""FP8 (E4M3) block-scaled operands for the reduced-precision sketch forms.

Test infrastructure (see ``oracle/__init__``).  The paper computes in FP64; the FP8 form of the
sketch contraction is a precision variant of this implementation, so this module writes out the
arithmetic it is defined by, for the parity tests of such a form:

* E4M3FN values as the FP8 formats define them (Micikevicius et al., "FP8 formats for deep
  learning", 2022; the OCP 8-bit floating point specification): sign, 4 exponent bits with bias
  7, 3 mantissa bits, subnormals below 2^-6, no infinities, the largest finite value 448.
  Conversion rounds to nearest with ties to an even mantissa and saturates at +-448.
* Block scaling along the contraction (the coordinate axis): each block of ``block`` consecutive
  coordinates of a column shares one power-of-two scale, as the microscaling (MX) formats store
  it (an 8-bit exponent); the scale is the smallest power of two that keeps the block's largest
  magnitude within 448, so no element saturates (reading: the MX formats also allow a scale that
  lets the largest element clip; this one never clips).
* The two-term split a ~ hi + lo: hi is the block-scaled E4M3 image of a, lo that of the
  residual a - hi with its own block scales; the sketch of the split is Omega (hi + lo) in FP64.

Parity status: every function is pinned in ``tests/test_oracle_pins.py`` (the E4M3 grid from
the bit definition, rounding against brute-force nearest-grid search, saturation and
subnormals, the scale rule, the split's error bound).
"""
import numpy as np

E4M3_MAX = 448.0
E4M3_MIN_NORMAL = 2.0 ** -6
E4M3_MIN_SUBNORMAL = 2.0 ** -9


def e4m3_grid():
    """All finite non-negative E4M3FN values, from the bit fields (exponent 15 with mantissa 7 is
    NaN; exponent 0 encodes the subnormals m/8 * 2^-6)."""
    vals = set()
    for e in range(16):
        for m in range(8):
            if e == 15 and m == 7:
                continue
            vals.add((m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(sorted(vals))


def e4m3_round(x):
    """Nearest E4M3FN value of each element (ties to an even mantissa), saturating at +-448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, ex = np.frexp(np.maximum(a, E4M3_MIN_NORMAL))     # a = f 2^ex, f in [0.5, 1)
    e = np.minimum(ex - 1, 8)                            # binade exponent, normals; 2^-6 floor
    step = np.ldexp(1.0, e - 3)                          # mantissa spacing: 3 fraction bits
    q = np.round(a / step) * step                        # numpy rounds halves to even
    q = np.minimum(q, E4M3_MAX)
    return np.copysign(q, x)


def block_scales(a, block):
    """Per-block power-of-two scales along axis 0 of ``a`` (m x n): for each block of ``block``
    rows and each column, the smallest 2^X with max |a| / 2^X <= 448 (1 for an all-zero block).
    Returns an array of the shape of ``a`` holding each element's scale."""
    a = np.asarray(a, dtype=np.float64)
    m = a.shape[0]
    out = np.empty_like(a)
    for b0 in range(0, m, block):
        amax = np.max(np.abs(a[b0:b0 + block]), axis=0)
        x = np.ceil(np.log2(np.where(amax > 0, amax, 1.0) / E4M3_MAX))
        s = np.ldexp(1.0, x.astype(np.int64))
        # the ceiling of a rounded logarithm can miss by one: enforce the defining inequality
        s = np.where(amax / s > E4M3_MAX, s * 2.0, s)
        s = np.where((amax > 0) & (amax / (s / 2.0) <= E4M3_MAX), s / 2.0, s)
        out[b0:b0 + block] = np.where(amax > 0, s, 1.0)[None, :]
    return out


def quantize_blocked(a, block):
    """The block-scaled E4M3 image of ``a`` (m x n, scaled back): scale * e4m3(a / scale)."""
    s = block_scales(a, block)
    return s * e4m3_round(np.asarray(a, dtype=np.float64) / s)


def split_x2(a, block):
    """(hi, lo): hi = the block-scaled E4M3 image of a, lo = that of the residual a - hi."""
    a = np.asarray(a, dtype=np.float64)
    hi = quantize_blocked(a, block)
    lo = quantize_blocked(a - hi, block)
    return hi, lo


def sketch_fp8x2(omega, a, block):
    """Omega (hi + lo) in FP64 for the two-term block-scaled E4M3 split of the columns of a."""
    hi, lo = split_x2(a, block)
    return omega @ (hi + lo)
