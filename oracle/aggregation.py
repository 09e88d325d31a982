"""Oracle: Gamma5-compatible aggregation, prolongation P and restriction R = P^dagger (Sec. 2.3).

TEST INFRASTRUCTURE ONLY.  Each aggregate is a lattice block V_j; it is split
by chirality into A_{j,+} (Gamma5 = +1 dofs) and A_{j,-} (Gamma5 = -1 dofs)
("standard aggregation", Sec. 2.3).  The test vectors restricted to each
aggregate half are orthonormalised (Sec. 2.3) by modified Gram-Schmidt in
index order, applied twice (our reading: the paper does not name the variant).

P is stored as W with shape (2, Nv) + lat + dof: W[s, i] is a field on the
level being aggregated whose restriction to aggregate j is column (j, s, i) of
P.  Coarse dof (j, s, i) has index s*Nv + i inside coarse site j, so
Gamma5_c = tau3 x I_Nv (Sec. 2.3).
"""

import numpy as np

from . import blocks


def build_P(op, v, bdims):
    """P from the test vectors v (shape (Nv,) + lat + dof) on operator op's level."""
    lat = op.lat
    nd = len(op.dof)
    nv = v.shape[0]
    W = np.zeros((2,) + v.shape, dtype=complex)
    for s in range(2):
        W[s] = v * op.chirality_mask(s)
    for s in range(2):
        for _sweep in range(2):
            for i in range(nv):
                for j in range(i):
                    proj = blocks.block_sum(np.conj(W[s, j]) * W[s, i], lat, bdims)
                    W[s, i] = W[s, i] - blocks.broadcast(proj, lat, bdims, nd) * W[s, j]
                nrm = np.sqrt(blocks.block_sum(np.abs(W[s, i]) ** 2, lat, bdims).real)
                W[s, i] = W[s, i] / blocks.broadcast(nrm, lat, bdims, nd)
    return W


def restrict(W, psi, lat, bdims):
    """R psi = P^dagger psi: coarse field of shape coarse_lat + (2 Nv,)."""
    nv = W.shape[1]
    c = blocks.block_sum_keep(np.conj(W) * psi, lat, bdims, 2)  # (2, Nv) + coarse_lat
    c = c.reshape((2 * nv,) + c.shape[2:])
    return np.moveaxis(c, 0, -1)


def prolong(W, c, lat, bdims):
    """P c: fine field from a coarse field c of shape coarse_lat + (2 Nv,)."""
    nv = W.shape[1]
    nd = W.ndim - 2 - 4
    out = np.zeros(W.shape[2:], dtype=complex)
    for s in range(2):
        for i in range(nv):
            out += blocks.broadcast(c[..., s * nv + i], lat, bdims, nd) * W[s, i]
    return out
