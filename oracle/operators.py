"""Oracle: operator objects shared by SAP, aggregation, Galerkin and Krylov code.

TEST INFRASTRUCTURE ONLY.  An operator acts on fields of shape ``lat + dof``
(``lat`` = (T, Z, Y, X) of its level).  It splits, as every level of the
hierarchy does (Sec. 2.3: the coarse operator keeps the nearest-neighbour
structure of the fine one), into

* a site-local part ``site(psi, mu)`` (for the fine level: the clover site term
  plus i mu Gamma5; for a coarse level: the self coupling plus i mu Gamma5_c),
* nearest-neighbour hops ``hop_dir(psi, d, sign)`` whose sum is ``hop``.

``apply(psi, mu) = site(psi, mu) + hop(psi)``.
"""

import numpy as np

from . import dirac


class FineOperator:
    """D(mu) = D_W + i mu Gamma5 on the fine lattice (Sec. 2.1)."""

    def __init__(self, U, kappa, c_sw, bc_t=0, theta=None):
        self.U = U
        self.theta = theta  # twisted boundary angles per direction mu (None: none)
        self.S = dirac.site_term(U, kappa, c_sw)
        self.lat = U.shape[:4]
        self.dof = (4, 3)
        self.bc_t = bc_t
        self._g, self._g5 = dirac.gamma_matrices()
        self._g5_12 = np.kron(np.diag(self._g5).real, np.ones(3))  # gamma5 x I_3 diagonal

    def apply(self, psi, mu):
        return dirac.apply_D(self.U, self.S, psi, mu, self.bc_t, self.theta)

    def site(self, psi, mu):
        out = dirac.apply_site(self.S, psi)
        if mu != 0.0:
            out = out + dirac.apply_twist(psi, mu)
        return out

    def site_matrix(self, mu):
        """(S(x) + i mu gamma5 x I_3) as a 12x12 matrix per site."""
        return self.S + 1j * mu * np.diag(self._g5_12)

    def site_inv(self, psi, mu):
        """Per-site inverse of the site-local part, applied as (S + i mu gamma5)^-1 psi.
        The per-site inverses (library LU inversion) are kept for the last mu."""
        if getattr(self, "_inv_mu", None) != mu:
            self._inv = np.linalg.inv(self.site_matrix(mu))
            self._inv_mu = mu
        lat = psi.shape[:4]
        return np.matmul(self._inv, psi.reshape(lat + (12, 1))).reshape(psi.shape)

    def hop(self, psi):
        return dirac.apply_hopping(self.U, psi, self.bc_t, theta=self.theta)

    def hop_dir(self, psi, d, sign):
        """One hopping direction of Sec. 2.1: sign=+1 gives -1/2 (I-g_d) U_d(x) psi(x+d),
        sign=-1 gives -1/2 (I+g_d) U_d(x-d)^dagger psi(x-d)."""
        U = self.U[..., d, :, :]
        i4 = np.eye(4)
        if sign > 0:
            nb = dirac.shift_fermion(psi, d, +1, self.bc_t, self.theta)
            return -0.5 * np.matmul(i4 - self._g[d], dirac.colour_mul(U, nb))
        nb = dirac.shift_fermion(psi, d, -1, self.bc_t, self.theta)
        Ub = dirac.dagger(dirac.shift(U, d, -1))
        return -0.5 * np.matmul(i4 + self._g[d], dirac.colour_mul(Ub, nb))

    def gamma5(self, psi):
        return dirac.apply_Gamma5(psi)

    def chirality_mask(self, s):
        """Spins {0,1} (Gamma5 = +1) for s = 0, spins {2,3} (Gamma5 = -1) for s = 1 (Sec. 2.3)."""
        m = np.zeros(self.dof, dtype=bool)
        m[2 * s:2 * s + 2, :] = True
        return m


class CoarseOperator:
    """D_c(mu) = P^dagger D P + i mu Gamma5_c stored as 9 blocks per coarse site (Sec. 2.3).

    ``blocks[0]`` is the self coupling without twist, ``blocks[1 + 2*d]`` couples
    x to x + d_hat and ``blocks[2 + 2*d]`` couples x to x - d_hat.  Each entry has
    shape ``lat + (2 Nv, 2 Nv)``; coarse dof index s*Nv + i.
    """

    def __init__(self, blocks, nv):
        self.blocks = blocks
        self.lat = blocks.shape[1:5]
        self.nv = nv
        self.dof = (2 * nv,)
        self.g5c = np.concatenate([np.ones(nv), -np.ones(nv)])  # Gamma5_c = tau3 x I_Nv

    def _mv(self, A, v):
        return np.matmul(A, v[..., None])[..., 0]

    def site(self, v, mu):
        out = self._mv(self.blocks[0], v)
        if mu != 0.0:
            out = out + 1j * mu * self.g5c * v
        return out

    def site_matrix(self, mu):
        return self.blocks[0] + 1j * mu * np.diag(self.g5c)

    def site_inv(self, v, mu):
        if getattr(self, "_inv_mu", None) != mu:
            self._inv = np.linalg.inv(self.site_matrix(mu))
            self._inv_mu = mu
        return self._mv(self._inv, v)

    def hop_dir(self, v, d, sign):
        idx = 1 + 2 * d if sign > 0 else 2 + 2 * d
        return self._mv(self.blocks[idx], dirac.shift(v, d, sign))

    def hop(self, v):
        out = np.zeros_like(v)
        for d in range(4):
            out += self.hop_dir(v, d, +1) + self.hop_dir(v, d, -1)
        return out

    def apply(self, v, mu):
        return self.site(v, mu) + self.hop(v)

    def gamma5(self, v):
        return self.g5c * v

    def chirality_mask(self, s):
        m = np.zeros(self.dof, dtype=bool)
        m[s * self.nv:(s + 1) * self.nv] = True
        return m
