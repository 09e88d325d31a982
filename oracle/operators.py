"""Oracle: operator objects shared by SAP, aggregation, Galerkin and Krylov code.

TEST INFRASTRUCTURE ONLY.  An operator acts on fields of shape ``lat + dof``
(``lat`` = (T, Z, Y, X) of its level).  It splits, as every level of the
hierarchy does (Sec. 2.3: the coarse operator keeps the nearest-neighbour
structure of the fine one), into

* a site-local part ``site(psi, mu)`` (for the fine level: the clover site term
  plus i mu Gamma5; for a coarse level: the self coupling plus i mu Gamma5_c),
* nearest-neighbour hops ``hop_dir(psi, d, sign)`` whose sum is ``hop``.

``apply(psi, mu) = site(psi, mu) + hop(psi)``.

The twist ``mu`` is a number, or a pair ``(mu_e, mu_o)`` for a different twist
on even and odd sites (a library feature of the paper's appendix, used by the
even-odd preconditioned HMC): i Gamma5 (mu_e P_e + mu_o P_o) with P_e, P_o the
projectors on even and odd sites.  Written as i Gamma5 (mbar + d S) with
mbar = (mu_e + mu_o)/2, d = (mu_e - mu_o)/2 and S the site-local parity weight
(+1 on even, -1 on odd sites), it keeps its form on every coarse level: the
Galerkin product of i d Gamma5 S is i d Q Gamma5_c with
Q_A = sum_{x in A} P_A(x)^dagger S(x) P_A(x) (Gamma5 P = P Gamma5_c), a dense
site-local block that commutes with Gamma5_c; ``pweight`` applies S (or Q).
"""

import numpy as np

from . import dirac


def split_twist(mu):
    """(mbar, d) of a twist: a number mu gives (mu, 0), a pair (mu_e, mu_o) gives
    ((mu_e + mu_o)/2, (mu_e - mu_o)/2)."""
    if np.ndim(mu) == 0:
        return float(mu), 0.0
    mu_e, mu_o = mu
    return 0.5 * (mu_e + mu_o), 0.5 * (mu_e - mu_o)


def scale_twist(mu, f):
    """f times a twist (both parities of a pair)."""
    if np.ndim(mu) == 0:
        return f * mu
    return (f * mu[0], f * mu[1])


def negate_twist(mu):
    return scale_twist(mu, -1.0)


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
        self._sgn = np.where(dirac.parity(self.lat) == 0, 1.0, -1.0)  # parity weight S(x)

    def pweight(self, psi):
        """S psi: +psi on even sites, -psi on odd sites."""
        return self._sgn.reshape(self.lat + (1, 1)) * psi

    def apply(self, psi, mu):
        mb, d = split_twist(mu)
        out = dirac.apply_D(self.U, self.S, psi, mb, self.bc_t, self.theta)
        if d != 0.0:
            out = out + dirac.apply_twist(self.pweight(psi), d)
        return out

    def site(self, psi, mu):
        mb, d = split_twist(mu)
        out = dirac.apply_site(self.S, psi)
        if mb != 0.0:
            out = out + dirac.apply_twist(psi, mb)
        if d != 0.0:
            out = out + dirac.apply_twist(self.pweight(psi), d)
        return out

    def site_matrix(self, mu):
        """(S(x) + i (mbar + d S(x)) gamma5 x I_3) as a 12x12 matrix per site."""
        mb, d = split_twist(mu)
        tw = (mb + d * self._sgn)[..., None, None]
        return self.S + 1j * tw * np.diag(self._g5_12)

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

    def __init__(self, blocks, nv, Q=None, Q_fn=None):
        self.blocks = blocks
        self.lat = blocks.shape[1:5]
        self.nv = nv
        self.dof = (2 * nv,)
        self.g5c = np.concatenate([np.ones(nv), -np.ones(nv)])  # Gamma5_c = tau3 x I_Nv
        self._Q = Q         # projected parity weight, lat + (2Nv, 2Nv), or
        self._Q_fn = Q_fn   # a function computing it when first needed (None, None: not available)

    @property
    def Q(self):
        if self._Q is None and self._Q_fn is not None:
            self._Q = self._Q_fn()
        return self._Q

    def _mv(self, A, v):
        return np.matmul(A, v[..., None])[..., 0]

    def pweight(self, v):
        """Q v, the parity weight projected to this level."""
        if self.Q is None:
            raise ValueError("coarse operator built without the projected parity weight")
        return self._mv(self.Q, v)

    def site(self, v, mu):
        mb, d = split_twist(mu)
        out = self._mv(self.blocks[0], v)
        if mb != 0.0:
            out = out + 1j * mb * self.g5c * v
        if d != 0.0:
            out = out + 1j * d * self.pweight(self.g5c * v)
        return out

    def site_matrix(self, mu):
        mb, d = split_twist(mu)
        M = self.blocks[0] + 1j * mb * np.diag(self.g5c)
        if d != 0.0:
            M = M + 1j * d * np.matmul(self.Q, np.diag(self.g5c))
        return M

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
