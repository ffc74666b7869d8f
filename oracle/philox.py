"""Philox4x32-10 counter-based generator and the random streams the method draws.

Test infrastructure (see ``oracle/__init__``).

Philox4x32-R is defined in Salmon, Moraes, Dror & Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11): a 128-bit counter and a 64-bit key,
R rounds of two 32x32->64 multiplies (multipliers 0xD2511F53, 0xCD9E8D57)
whose high/low halves are xored with the other counter words and the round
key; the key is bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) before
every round after the first.  Pinned by the published known-answer vectors
(tests/golden/philox4x32_10_kat.txt).

The method draws three kinds of random numbers (Algorithm 3): the entries of
the test matrix Omega (Gaussian in the paper, Rademacher as the sub-Gaussian
alternative allowed by the NA-Hutch++ analysis of Sec. 3.3), and the uniforms
behind every random keep / drop decision of the column subset selection.
Their counter layout is fixed here and restated independently by the CUDA
library:

* Rademacher Omega[r, i]:   one bit of Philox((i // 128, r, TAG_RADEMACHER, 0)); with
  j = i mod 128, word w = j // 32 and e = j mod 32, coordinate pair p = e // 2 takes
  bit 15 - p of word w for even e and bit 31 - p for odd e; a set bit means -1.
* Gaussian Omega[r, i]:     Box-Muller pair from Philox((i // 2, r, TAG_GAUSS, 0));
  even i takes the cosine branch, odd i the sine branch.
* Uniform u(batch, i, r):   53-bit uniform in [0, 1) from words 0, 1 of
  Philox((i, r, TAG_UNIFORM, batch)).
* Gradient-sketch Omega_g[r, q]: as Rademacher/Gaussian with TAG_GRAD_* and
  q = p*m + i the index into the stacked gradient vector (Sec. 3.4).
* Right-sketch omega_j[r] (the optional m x l right sketch Y = sum_j a_j omega_j^T; not part
  of the paper's method): as Rademacher/Gaussian with TAG_RIGHT_*, row r in 0..l-1 and
  i = j the global index of the snapshot.

Keys are (seed & 0xffffffff, seed >> 32).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)

TAG_RADEMACHER = 0x52414431   # 'RAD1'
TAG_GAUSS = 0x47415531        # 'GAU1'
TAG_UNIFORM = 0x554E4931      # 'UNI1'
TAG_GRAD_RADEMACHER = 0x47524431  # 'GRD1'
TAG_GRAD_GAUSS = 0x47524731       # 'GRG1'
TAG_RIGHT_RADEMACHER = 0x52534B31  # 'RSK1'
TAG_RIGHT_GAUSS = 0x52534731       # 'RSG1'

TWO_M53 = 1.0 / 9007199254740992.0   # 2**-53


def philox4x32(c0, c1, c2, c3, k0, k1, rounds=10):
    """Philox4x32-R on broadcastable arrays of uint32 counters; returns 4 uint32 arrays."""
    x0 = np.asarray(c0, dtype=np.uint64) & MASK32
    x1 = np.asarray(c1, dtype=np.uint64) & MASK32
    x2 = np.asarray(c2, dtype=np.uint64) & MASK32
    x3 = np.asarray(c3, dtype=np.uint64) & MASK32
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    x0, x1, x2, x3 = x0.copy(), x1.copy(), x2.copy(), x3.copy()
    key0 = int(k0) & 0xFFFFFFFF
    key1 = int(k1) & 0xFFFFFFFF
    for rnd in range(rounds):
        if rnd > 0:
            key0 = (key0 + W0) & 0xFFFFFFFF
            key1 = (key1 + W1) & 0xFFFFFFFF
        p0 = M0 * x0            # exact: both factors < 2**32
        p1 = M1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(key0), lo1,
                          hi0 ^ x3 ^ np.uint64(key1), lo0)
    return (x0.astype(np.uint32), x1.astype(np.uint32),
            x2.astype(np.uint32), x3.astype(np.uint32))


def seed_key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def uniform53(w0, w1):
    """(w0 >> 5) * 2**26 + (w1 >> 6), scaled by 2**-53: exact doubles in [0, 1)."""
    a = (np.asarray(w0, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    b = (np.asarray(w1, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b) * TWO_M53


def uniform(seed, batch, i, r):
    """The uniform behind one sampling decision of batch step ``batch``."""
    k0, k1 = seed_key(seed)
    w = philox4x32(i, r, TAG_UNIFORM, batch, k0, k1)
    return uniform53(w[0], w[1])


def rademacher_block(seed, rows, i0, i1, tag=TAG_RADEMACHER):
    """Dense +-1 block Omega[rows, i0:i1] (float64)."""
    rows = np.asarray(rows, dtype=np.int64)
    i = np.arange(i0, i1, dtype=np.int64)
    k0, k1 = seed_key(seed)
    blk = i // 128
    w = philox4x32(blk[None, :], rows[:, None], tag, 0, k0, k1)
    pos = (i % 128)[None, :]
    word = pos // 32
    e = pos % 32
    bit = np.where(e % 2 == 0, 15 - e // 2, 31 - e // 2).astype(np.uint64)
    words = np.stack([x.astype(np.uint64) for x in w], axis=0)  # (4, R, N)
    sel = np.take_along_axis(words, np.broadcast_to(word, w[0].shape)[None], axis=0)[0]
    b = (sel >> bit) & np.uint64(1)
    return 1.0 - 2.0 * b.astype(np.float64)


def gauss_block(seed, rows, i0, i1, tag=TAG_GAUSS):
    """Dense N(0,1) block Omega[rows, i0:i1] (float64) by Box-Muller."""
    rows = np.asarray(rows, dtype=np.int64)
    i = np.arange(i0, i1, dtype=np.int64)
    k0, k1 = seed_key(seed)
    w = philox4x32((i // 2)[None, :], rows[:, None], tag, 0, k0, k1)
    u1 = uniform53(w[0], w[1]) + 0.5 * TWO_M53          # (0, 1)
    u2 = uniform53(w[2], w[3])
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    even = (i % 2 == 0)[None, :]
    return np.where(even, rad * np.cos(ang), rad * np.sin(ang))


def omega_block(kind, seed, rows, i0, i1, grad=False, right=False):
    """Omega[rows, i0:i1] for ``kind`` in {'gaussian', 'rademacher'} (``grad``: Omega_g of the
    gradient sketch; ``right``: the right-sketch vectors, row r, column i = snapshot index)."""
    if kind == "rademacher":
        tag = TAG_RIGHT_RADEMACHER if right else (TAG_GRAD_RADEMACHER if grad else TAG_RADEMACHER)
        return rademacher_block(seed, rows, i0, i1, tag)
    if kind == "gaussian":
        tag = TAG_RIGHT_GAUSS if right else (TAG_GRAD_GAUSS if grad else TAG_GAUSS)
        return gauss_block(seed, rows, i0, i1, tag)
    raise ValueError(kind)
