"""Oracle: the Galerkin coarse operator D_c = P^dagger D P + i mu Gamma5_c (Sec. 2.3).

TEST INFRASTRUCTURE ONLY.  Only neighbouring aggregates couple (Sec. 2.3), so
D_c is stored as 9 dense (2 Nv x 2 Nv) blocks per coarse site:

* self  : P_j^dagger (site term + hops that stay inside aggregate j) P_j,
* +d    : P_j^dagger (hops of direction +d that leave aggregate j) P_{j+d},
* -d    : the same for -d,

with the twist left out (``CoarseOperator`` adds i mu Gamma5_c on the fly, so
one build serves +mu and -mu, and the coarsest level can use delta*mu).  The
twist is added as i mu Gamma5_c as printed in Sec. 2.3, which equals
P^dagger (i mu Gamma5) P because Gamma5 P = P Gamma5_c and P^dagger P = I.

Every field column is built for all aggregates at once: W[s', j] holds column
(s', j) of every aggregate, so the hops of W[s', j] that cross from aggregate
A into A + d pick up exactly column (s', j) of A + d.
"""

import numpy as np

from . import blocks
from .operators import CoarseOperator


def galerkin(op, W, bdims):
    """Coarse blocks (9,) + coarse_lat + (2Nv, 2Nv) of P^dagger D_W P for operator op."""
    lat = op.lat
    nv = W.shape[1]
    n = 2 * nv
    clat = blocks.coarse_lat(lat, bdims)
    nd = len(op.dof)
    out = np.zeros((9,) + clat + (n, n), dtype=complex)
    Wc = np.conj(W)
    masks = {}
    for d in range(4):
        for sg in (+1, -1):
            masks[(d, sg)] = blocks.crossing_mask(lat, bdims, d, sg).reshape(lat + (1,) * nd)
    for sp in range(2):
        for j in range(nv):
            col = sp * nv + j
            phi = W[sp, j]
            parts = [op.site(phi, 0.0)] + [None] * 8
            for d in range(4):
                for k, sg in enumerate((+1, -1)):
                    h = op.hop_dir(phi, d, sg)
                    m = masks[(d, sg)]
                    parts[0] = parts[0] + h * (~m)
                    parts[1 + 2 * d + k] = h * m
            for idx in range(9):
                rows = blocks.block_sum_keep(Wc * parts[idx], lat, bdims, 2)  # (2, Nv) + clat
                out[idx][..., :, col] = np.moveaxis(rows.reshape((n,) + clat), 0, -1)
    return out


def projected_pweight(op, W, bdims):
    """Q_A = P_A^dagger S P_A per aggregate: the parity weight S of op's level (+1 on even,
    -1 on odd fine sites; already projected on coarse levels) in the coarse basis, so that the
    Galerkin product of a different twist on even and odd sites, i Gamma5 (mbar + d S), is
    i mbar Gamma5_c + i d Q Gamma5_c."""
    lat = op.lat
    nv = W.shape[1]
    n = 2 * nv
    clat = blocks.coarse_lat(lat, bdims)
    out = np.zeros(clat + (n, n), dtype=complex)
    Wc = np.conj(W)
    for sp in range(2):
        for j in range(nv):
            rows = blocks.block_sum_keep(Wc * op.pweight(W[sp, j]), lat, bdims, 2)
            out[..., :, sp * nv + j] = np.moveaxis(rows.reshape((n,) + clat), 0, -1)
    return out


def build_coarse_operator(op, W, bdims):
    """CoarseOperator for the next level: D_c(mu) = P^dagger D_W P + i mu Gamma5_c; the projected
    parity weight (different twists on even and odd sites) is computed when first used."""
    return CoarseOperator(galerkin(op, W, bdims), W.shape[1], Q_fn=lambda: projected_pweight(op, W, bdims))
