"""Simplex-gradient operator G of Sec. 3.4 (Eqs. 38-43) on a structured grid.

Test infrastructure (see ``oracle/__init__``).

For every vertex v_q the 1-ring neighbourhood N_q is taken from the edges of
the grid graph (the 2*d axis neighbours that exist; boundary vertices have
fewer).  K_q stacks x(v_r) - x(v_q); the least-squares gradient is
K_q^+ f_q (Eqs. 40-41) and G^p(q, r) = K_q^+(p, r), G^p(q, q) = -sum_r
K_q^+(p, r) (Eq. 43).  Several fields stacked in one snapshot are treated
independently (no cross-field entries).  The stacked operator
G = [G^1; ...; G^d] maps an m-vector to d*m gradient values (Eq. 42).
"""
import numpy as np
import scipy.sparse as sp


def grid_gradient_operator(shape, spacing=1.0, nfields=1):
    """Sparse (d * m) x m operator for fields stored with the first axis fastest.

    ``shape`` = (n_1, ..., n_d) with axis 1 varying fastest in memory; the
    snapshot holds ``nfields`` such fields one after another.
    """
    shape = tuple(int(x) for x in shape)
    d = len(shape)
    npts = int(np.prod(shape))
    strides = [int(np.prod(shape[:p])) for p in range(d)]
    rows, cols, vals = [], [], []
    for q in range(npts):
        coord = [(q // strides[p]) % shape[p] for p in range(d)]
        nbrs, offs = [], []
        for p in range(d):
            for sgn in (-1, 1):
                c = coord[p] + sgn
                if 0 <= c < shape[p]:
                    nbrs.append(q + sgn * strides[p])
                    off = np.zeros(d)
                    off[p] = sgn * spacing
                    offs.append(off)
        K = np.array(offs)                   # Eq. 39: rows x(v_r) - x(v_q)
        Kp = np.linalg.pinv(K)               # Eq. 41
        for p in range(d):
            for r, nb in enumerate(nbrs):
                if Kp[p, r] != 0.0:
                    rows.append(p * npts + q)
                    cols.append(nb)
                    vals.append(Kp[p, r])
            rows.append(p * npts + q)
            cols.append(q)
            vals.append(-Kp[p].sum())
    G1 = sp.csr_matrix((vals, (rows, cols)), shape=(d * npts, npts))
    if nfields == 1:
        return G1
    # per field: rows (p, field, q), columns (field, q); fields independent
    blocks = []
    for p in range(d):
        Gp = G1[p * npts:(p + 1) * npts]
        blocks.append(sp.block_diag([Gp] * nfields, format="csr"))
    return sp.vstack(blocks, format="csr")
