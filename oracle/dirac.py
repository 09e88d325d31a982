"""Oracle: the twisted-mass clover Wilson-Dirac operator D(mu) = D_W + i mu Gamma5.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain FP64 numpy,
written from Sec. 2.1 of arXiv:1610.02370:

* D_W: the clover-improved Wilson operator (Sec. 2.1, the display defining
  D_W psi): site term (m+4) I_12 - c_sw/32 sum_{mu,nu} (gamma_mu gamma_nu) x
  (Q_mu_nu - Q_nu_mu), and the hopping term -1/2 sum_mu [(I-gamma_mu) x U_mu(x)]
  psi(x+mu) + [(I+gamma_mu) x U_mu(x-mu)^dagger] psi(x-mu).
* Q_mu_nu: the sum of the four oriented plaquette leaves around x (Sec. 2.1,
  the display defining Q_mu_nu).
* gamma5 = gamma0 gamma1 gamma2 gamma3 = diag(1, 1, -1, -1) (Sec. 2.1).  The
  paper prints no gamma_mu; the Hermitian chiral basis below is our reading and
  reproduces that gamma5.
* D(mu) = D_W + i mu Gamma5 (Sec. 2.1, flavour-twist display); the mass is
  m = 1/(2 kappa) - 4 and mu enters as printed, without a 2-kappa factor.
* Boundary conditions (unstated in the paper): periodic, optionally
  antiperiodic in t for the fermion hops (never for the gauge links), and
  optionally twisted (a library feature the paper lists in its appendix):
  psi(x + L_mu mu_hat) = exp(i theta_mu) psi(x), i.e. a hop that wraps
  forward in direction mu reads exp(i theta_mu) psi, one that wraps backward
  exp(-i theta_mu) psi.
"""

import numpy as np

# array axis carrying direction mu (mu = 0:t, 1:x, 2:y, 3:z) for (T, Z, Y, X) arrays
AXIS = (0, 3, 2, 1)


def gamma_matrices():
    """Hermitian chiral basis: gamma_0 = [[0, 1], [1, 0]], gamma_k = [[0, i s_k], [-i s_k, 0]].

    Returns (gammas, gamma5) with gammas a list of four 4x4 complex arrays and
    gamma5 = gamma_0 gamma_1 gamma_2 gamma_3, which equals diag(1, 1, -1, -1)
    as Sec. 2.1 requires.
    """
    i2 = np.eye(2, dtype=complex)
    z2 = np.zeros((2, 2), dtype=complex)
    sig = [np.array([[0, 1], [1, 0]], dtype=complex),
           np.array([[0, -1j], [1j, 0]], dtype=complex),
           np.array([[1, 0], [0, -1]], dtype=complex)]
    g = [np.block([[z2, i2], [i2, z2]])]
    for s in sig:
        g.append(np.block([[z2, 1j * s], [-1j * s, z2]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


def mass_from_kappa(kappa):
    """Bare mass m in the (m+4) normalisation of Sec. 2.1: m = 1/(2 kappa) - 4."""
    return 1.0 / (2.0 * kappa) - 4.0


def dagger(a):
    """Conjugate transpose of the trailing two axes."""
    return np.conj(np.swapaxes(a, -1, -2))


def shift(field, mu, sign):
    """Periodic shift: returns F with F(x) = field(x + sign * mu_hat)."""
    return np.roll(field, -sign, axis=AXIS[mu])


def shift_fermion(psi, mu, sign, bc_t=0, theta=None):
    """Fermion field at x + sign*mu_hat; bc_t = 1 puts a -1 on hops that wrap in t; theta
    (four angles, or None) multiplies hops that wrap forward in mu by exp(i theta_mu) and
    hops that wrap backward by exp(-i theta_mu)."""
    out = shift(psi, mu, sign)
    f = 1.0 + 0j
    if mu == 0 and bc_t == 1:
        f = -f
    if theta is not None and theta[mu] != 0.0:
        f = f * np.exp(1j * sign * theta[mu])
    if f != 1.0:
        out = out.copy()
        edge = [slice(None)] * out.ndim
        # forward: x_mu = L-1 reads psi at x_mu = 0; backward: x_mu = 0 reads x_mu = L-1
        edge[AXIS[mu]] = -1 if sign > 0 else 0
        out[tuple(edge)] *= f
    return out


def _link(U, mu):
    return U[..., mu, :, :]


def clover_leaves(U, mu, nu):
    """Q_mu_nu(x): the four plaquette leaves of Sec. 2.1, in the printed order.

    Returns a (T, Z, Y, X, 3, 3) array.
    """
    Um, Un = _link(U, mu), _link(U, nu)

    def at(F, *moves):
        # F evaluated at x + sum of (sign, direction) moves, periodic
        for d, s in moves:
            F = shift(F, d, s)
        return F

    leaf1 = Um @ at(Un, (mu, +1)) @ dagger(at(Um, (nu, +1))) @ dagger(Un)
    leaf2 = (Un @ dagger(at(Um, (mu, -1), (nu, +1))) @ dagger(at(Un, (mu, -1)))
             @ at(Um, (mu, -1)))
    leaf3 = (dagger(at(Um, (mu, -1))) @ dagger(at(Un, (mu, -1), (nu, -1)))
             @ at(Um, (mu, -1), (nu, -1)) @ at(Un, (nu, -1)))
    leaf4 = (dagger(at(Un, (nu, -1))) @ at(Um, (nu, -1)) @ at(Un, (nu, -1), (mu, +1))
             @ dagger(Um))
    return leaf1 + leaf2 + leaf3 + leaf4


def site_term(U, kappa, c_sw):
    """Site-local part of D_W as a 12x12 matrix per site (index spin*3 + colour).

    S(x) = (m+4) I_12 - c_sw/32 sum_{mu,nu=0..3} (gamma_mu gamma_nu) x (Q_mu_nu(x) - Q_nu_mu(x)),
    summed over all 16 ordered pairs as printed (the mu = nu terms vanish).
    Returns a (T, Z, Y, X, 12, 12) complex array.
    """
    g, _ = gamma_matrices()
    m = mass_from_kappa(kappa)
    lat = U.shape[:4]
    S = np.zeros(lat + (12, 12), dtype=complex)
    S += (m + 4.0) * np.eye(12)
    if c_sw != 0.0:
        for mu in range(4):
            for nu in range(4):
                if mu == nu:
                    continue
                F = clover_leaves(U, mu, nu) - clover_leaves(U, nu, mu)
                gg = g[mu] @ g[nu]
                # (gamma x F)[(s,a),(t,b)] = gg[s,t] * F[a,b]
                S -= (c_sw / 32.0) * np.einsum('st,...ab->...satb', gg, F).reshape(lat + (12, 12))
    return S


def apply_site(S, psi):
    """(S psi)(x) for a site-local 12x12 matrix field S and spinor psi (T,Z,Y,X,4,3)."""
    lat = psi.shape[:4]
    return np.matmul(S, psi.reshape(lat + (12, 1))).reshape(psi.shape)


def apply_twist(psi, mu):
    """i mu Gamma5 psi with Gamma5 = I_V x gamma5 x I_C and gamma5 = diag(1,1,-1,-1)."""
    _, g5 = gamma_matrices()
    return 1j * mu * np.matmul(g5, psi)


def colour_mul(U, psi):
    """(U psi)(x): the colour matrix U(x) on every spin component, psi (...,4,3)."""
    return np.matmul(psi, np.swapaxes(U, -1, -2))


def apply_hopping(U, psi, bc_t=0, mask_from=None, theta=None):
    """Hopping part of D_W (Sec. 2.1):

    -1/2 sum_mu [(I - gamma_mu) x U_mu(x)] psi(x+mu) + [(I + gamma_mu) x U_mu(x-mu)^dagger] psi(x-mu).
    """
    g, _ = gamma_matrices()
    i4 = np.eye(4)
    out = np.zeros_like(psi)
    for mu in range(4):
        Um = _link(U, mu)
        fwd = shift_fermion(psi, mu, +1, bc_t, theta)
        # U_mu(x) acts on colour, (I - gamma_mu) on spin
        out -= 0.5 * np.matmul(i4 - g[mu], colour_mul(Um, fwd))
        bwd = shift_fermion(psi, mu, -1, bc_t, theta)
        Ub = dagger(shift(Um, mu, -1))  # U_mu(x - mu)^dagger
        out -= 0.5 * np.matmul(i4 + g[mu], colour_mul(Ub, bwd))
    return out


def apply_D(U, S, psi, mu=0.0, bc_t=0, theta=None):
    """D(mu) psi = S psi + hopping(psi) + i mu Gamma5 psi.

    ``S`` is the site term from :func:`site_term`; ``psi`` is (T,Z,Y,X,4,3) or has
    a leading right-hand-side axis.
    """
    if psi.ndim == 7:
        return np.stack([apply_D(U, S, p, mu, bc_t, theta) for p in psi])
    out = apply_site(S, psi) + apply_hopping(U, psi, bc_t, theta=theta)
    if mu != 0.0:
        out += apply_twist(psi, mu)
    return out


def apply_Gamma5(psi):
    """Gamma5 psi (sign flip on spins 2, 3)."""
    out = psi.copy()
    out[..., 2:, :] *= -1.0
    return out


def parity(lat):
    """Site parity (t + x + y + z) mod 2 on a (T, Z, Y, X) lattice; 0 = even."""
    T, Z, Y, X = lat
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing='ij')
    return (t + z + y + x) % 2


def inner(a, b):
    """<a, b> = sum conj(a) b over every axis."""
    return np.vdot(a.ravel(), b.ravel())


def norm(a):
    return float(np.sqrt(np.real(inner(a, a))))
