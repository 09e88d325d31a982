"""Pins of the oracle's Dirac operator (Sec. 2.1) against closed forms and invariants.

Each test fixes a property that a plausible slip in the oracle would break:
* free-field plane waves (hopping signs, (1 -/+ gamma) placement, mass term,
  twist, boundary conditions including twisted ones, axis-to-direction mapping);
* twisted boundaries = a U(1) phase on the links crossing the boundary;
* constant non-trivial links (U versus U^dagger and U versus U^T in the hops);
* constant abelian field strength (clover leaves, their orientation and the
  c_sw/32 normalisation);
* gauge covariance (link placement in hops and leaves);
* Gamma5-hermiticity and ||D(mu)x||^2 = ||D_W x||^2 + mu^2 ||x||^2 (Sec. 2.1);
* sigma_min(D(mu)) >= |mu| (Sec. 2.1 SVD argument);
* the c_sw = 0 relation between eigenvalues of D and of its even-odd Schur
  complement (Sec. 2.1).
"""

import numpy as np
import pytest

from oracle import dirac
from paper_1610_02370_gb300 import synth

DIMS = (6, 4, 2, 8)  # T, X, Y, Z: all different, so an axis mix-up changes momenta


def lat_of(dims):
    T, X, Y, Z = dims
    return (T, Z, Y, X)


def coords(dims):
    """Coordinate arrays x_mu (mu = t, x, y, z) on the (T, Z, Y, X) array."""
    T, X, Y, Z = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing='ij')
    return (t, x, y, z)


def plane_wave(dims, p, chi, colour_vec):
    xs = coords(dims)
    ph = np.exp(1j * sum(p[m] * xs[m] for m in range(4)))
    return ph[..., None, None] * np.einsum('s,a->sa', chi, colour_vec)


def test_gamma_basis():
    g, g5 = dirac.gamma_matrices()
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)
        for b in range(4):
            ac = g[a] @ g[b] + g[b] @ g[a]
            assert np.allclose(ac, 2.0 * np.eye(4) * (a == b))
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


def free_symbol(p, m, mu):
    g, g5 = dirac.gamma_matrices()
    M = m + sum(1 - np.cos(p[a]) for a in range(4))
    return M * np.eye(4) + 1j * sum(g[a] * np.sin(p[a]) for a in range(4)) + 1j * mu * g5


@pytest.mark.parametrize("bc_t", [0, 1])
def test_free_field_plane_waves(bc_t):
    rng = np.random.default_rng(3)
    kappa, csw, mu = 0.13, 1.7, 0.23
    m = 1 / (2 * kappa) - 4
    U = synth.unit_gauge(DIMS).numpy()
    S = dirac.site_term(U, kappa, csw)
    for _ in range(6):
        n = [rng.integers(0, DIMS[a]) for a in range(4)]
        p = [2 * np.pi * n[a] / DIMS[a] for a in range(4)]
        if bc_t == 1:
            p[0] = (2 * n[0] + 1) * np.pi / DIMS[0]
        chi = rng.normal(size=4) + 1j * rng.normal(size=4)
        col = rng.normal(size=3) + 1j * rng.normal(size=3)
        psi = plane_wave(DIMS, p, chi, col)
        got = dirac.apply_D(U, S, psi, mu, bc_t)
        want = plane_wave(DIMS, p, free_symbol(p, m, mu) @ chi, col)
        assert np.max(np.abs(got - want)) < 1e-13


@pytest.mark.parametrize("bc_t", [0, 1])
def test_free_field_plane_waves_twisted_boundaries(bc_t):
    """Twisted boundary conditions psi(x + L_mu) = exp(i theta_mu) psi(x): the free plane waves
    have momenta p_mu = (2 pi n_mu + theta_mu) / L_mu (plus pi / L_t with antiperiodic t) and
    the same symbol as without twist."""
    rng = np.random.default_rng(13)
    kappa, csw, mu = 0.13, 1.7, 0.23
    m = 1 / (2 * kappa) - 4
    theta = [0.7, -1.3, 2.1, 0.4]
    U = synth.unit_gauge(DIMS).numpy()
    S = dirac.site_term(U, kappa, csw)
    for _ in range(6):
        n = [rng.integers(0, DIMS[a]) for a in range(4)]
        p = [(2 * np.pi * n[a] + theta[a]) / DIMS[a] for a in range(4)]
        if bc_t == 1:
            p[0] += np.pi / DIMS[0]
        chi = rng.normal(size=4) + 1j * rng.normal(size=4)
        col = rng.normal(size=3) + 1j * rng.normal(size=3)
        psi = plane_wave(DIMS, p, chi, col)
        got = dirac.apply_D(U, S, psi, mu, bc_t, theta)
        want = plane_wave(DIMS, p, free_symbol(p, m, mu) @ chi, col)
        assert np.max(np.abs(got - want)) < 1e-13


def test_twisted_boundaries_equal_boundary_link_phases():
    """A twist angle theta_mu on the fermion hops that wrap is the same operator as the periodic
    one on links U_mu(x) multiplied by exp(i theta_mu) where x_mu = L_mu - 1 (a U(1) factor on the
    links crossing the boundary: every closed loop, so the clover term, is unchanged); and
    Gamma5-hermiticity survives the twist."""
    dims = (4, 2, 4, 2)
    lat = lat_of(dims)
    U = synth.gauge_field(dims, 0.4, seed=7).numpy()
    kappa, csw, mu = 0.125, 1.3, 0.07
    theta = [0.9, -0.4, 1.7, 2.5]
    Uph = U.copy()
    for m_ in range(4):
        edge = [slice(None)] * 4
        edge[dirac.AXIS[m_]] = -1
        Uph[tuple(edge) + (m_,)] *= np.exp(1j * theta[m_])
    S = dirac.site_term(U, kappa, csw)
    assert np.max(np.abs(dirac.site_term(Uph, kappa, csw) - S)) < 1e-13
    psi = synth.gaussian_spinor(dims, seed=8).numpy()
    got = dirac.apply_D(U, S, psi, mu, 0, theta)
    want = dirac.apply_D(Uph, S, psi, mu, 0)
    assert np.max(np.abs(got - want)) < 1e-13
    chi = synth.gaussian_spinor(dims, seed=9).numpy()
    g5 = lambda v: dirac.apply_Gamma5(v)
    lhs = np.vdot(chi, g5(dirac.apply_D(U, S, g5(psi), mu, 0, theta)))
    rhs = np.vdot(dirac.apply_D(U, S, chi, -mu, 0, theta), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert lat == psi.shape[:4]


def test_free_field_spectrum_singular_values():
    """Singular values of the free D(mu): sqrt(M^2 + sum sin^2 p + mu^2), each 12-fold."""
    dims = (4, 2, 2, 4)
    kappa, mu = 0.124, 0.05
    m = 1 / (2 * kappa) - 4
    U = synth.unit_gauge(dims).numpy()
    S = dirac.site_term(U, kappa, 1.0)
    lat = lat_of(dims)
    n = np.prod(lat) * 12
    Dm = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1
        Dm[:, k] = dirac.apply_D(U, S, e.reshape(lat + (4, 3)), mu).ravel()
    sv = np.sort(np.linalg.svd(Dm, compute_uv=False))
    want = []
    for nt in range(dims[0]):
        for nx in range(dims[1]):
            for ny in range(dims[2]):
                for nz in range(dims[3]):
                    p = [2 * np.pi * nt / dims[0], 2 * np.pi * nx / dims[1],
                         2 * np.pi * ny / dims[2], 2 * np.pi * nz / dims[3]]
                    M = m + sum(1 - np.cos(q) for q in p)
                    want += [np.sqrt(M * M + sum(np.sin(q) ** 2 for q in p) + mu * mu)] * 12
    assert np.max(np.abs(sv - np.sort(want))) < 1e-12


def test_constant_links_shift_momenta():
    """All links U_mu = R diag(e^{i theta_mu}) R^dagger: colour eigenvector R e_c sees p -> p + theta_c."""
    rng = np.random.default_rng(5)
    kappa, mu = 0.125, -0.1
    m = 1 / (2 * kappa) - 4
    R = synth.random_gauge_transform((1, 1, 1, 1), seed=11).numpy()[0, 0, 0, 0]
    th = rng.uniform(-1, 1, size=(4, 3))
    th[:, 2] = -th[:, 0] - th[:, 1]
    lat = lat_of(DIMS)
    U = np.zeros(lat + (4, 3, 3), dtype=complex)
    for a in range(4):
        U[..., a, :, :] = R @ np.diag(np.exp(1j * th[a])) @ R.conj().T
    S = dirac.site_term(U, kappa, 2.0)
    for c in range(3):
        n = [rng.integers(0, DIMS[a]) for a in range(4)]
        p = [2 * np.pi * n[a] / DIMS[a] for a in range(4)]
        chi = rng.normal(size=4) + 1j * rng.normal(size=4)
        psi = plane_wave(DIMS, p, chi, R[:, c])
        got = dirac.apply_D(U, S, psi, mu)
        q = [p[a] + th[a, c] for a in range(4)]
        want = plane_wave(DIMS, p, free_symbol(q, m, mu) @ chi, R[:, c])
        assert np.max(np.abs(got - want)) < 1e-13


def abelian_field(dims, nflux):
    """Links diag(e^{i q_c theta_mu(x)}), q = (1, -1, 0), with a constant plaquette angle
    phi_{mu nu} = 2 pi n_{mu nu} / (L_mu L_nu) in every (mu < nu) plane."""
    xs = coords(dims)
    lat = lat_of(dims)
    theta = np.zeros((4,) + lat)
    phis = np.zeros((4, 4))
    for (a, b), n in nflux.items():
        phi = 2 * np.pi * n / (dims[a] * dims[b])
        phis[a, b], phis[b, a] = phi, -phi
        theta[b] += phi * xs[a]
        theta[a] += np.where(xs[a] == dims[a] - 1, -phi * dims[a] * xs[b], 0.0)
    q = np.array([1.0, -1.0, 0.0])
    U = np.zeros(lat + (4, 3, 3), dtype=complex)
    for a in range(4):
        for c in range(3):
            U[..., a, c, c] = np.exp(1j * q[c] * theta[a])
    return U, phis, q


def test_clover_constant_abelian_field():
    """Q_mu_nu = 4 e^{i phi} for a uniform field, so the clover term is
    -(c_sw/2) i sum_{mu<nu} gamma_mu gamma_nu sin(q_c phi_mu_nu) on colour c."""
    kappa, csw = 0.14, 1.3
    m = 1 / (2 * kappa) - 4
    U, phis, q = abelian_field(DIMS, {(0, 1): 1, (0, 3): 2, (1, 2): 1, (2, 3): -1})
    S = dirac.site_term(U, kappa, csw)
    g, _ = dirac.gamma_matrices()
    want = np.zeros((12, 12), dtype=complex)
    for c in range(3):
        blk = (m + 4) * np.eye(4, dtype=complex)
        for a in range(4):
            for b in range(a + 1, 4):
                blk -= 0.5 * csw * 1j * (g[a] @ g[b]) * np.sin(q[c] * phis[a, b])
        for s in range(4):
            for t in range(4):
                want[3 * s + c, 3 * t + c] = blk[s, t]
    assert np.max(np.abs(S - want)) < 1e-13


def test_gauge_covariance():
    dims = (4, 4, 2, 4)
    lat = lat_of(dims)
    U = synth.gauge_field(dims, 0.6, seed=2).numpy()
    gx = synth.random_gauge_transform(dims, seed=9).numpy()
    Ug = np.zeros_like(U)
    for a in range(4):
        Ug[..., a, :, :] = gx @ U[..., a, :, :] @ dirac.dagger(dirac.shift(gx, a, +1))
    psi = synth.gaussian_spinor(dims, seed=4).numpy()
    kappa, csw, mu = 0.13, 1.5755, 0.07
    for bc in (0, 1):
        y = dirac.apply_D(U, dirac.site_term(U, kappa, csw), psi, mu, bc)
        gpsi = np.einsum('...ab,...sb->...sa', gx, psi)
        yg = dirac.apply_D(Ug, dirac.site_term(Ug, kappa, csw), gpsi, mu, bc)
        assert np.max(np.abs(yg - np.einsum('...ab,...sb->...sa', gx, y))) < 1e-12
    assert lat == U.shape[:4]


def test_gamma5_hermiticity_and_norm_identity():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, seed=0).numpy()
    S = dirac.site_term(U, 0.125, 1.0)
    x = synth.gaussian_spinor(dims, seed=1).numpy()
    y = synth.gaussian_spinor(dims, seed=2).numpy()
    mu = 0.01
    for bc in (0, 1):
        lhs = dirac.inner(x, dirac.apply_D(U, S, y, mu, bc))
        rhs = dirac.inner(dirac.apply_Gamma5(dirac.apply_D(U, S, dirac.apply_Gamma5(x), -mu, bc)), y)
        assert abs(lhs - rhs) < 1e-11 * abs(lhs)
        n_mu = dirac.norm(dirac.apply_D(U, S, x, mu, bc)) ** 2
        n_0 = dirac.norm(dirac.apply_D(U, S, x, 0.0, bc)) ** 2
        assert abs(n_mu - (n_0 + mu * mu * dirac.norm(x) ** 2)) < 1e-12 * n_mu


def dense_D(U, S, mu, bc_t=0):
    lat = U.shape[:4]
    n = int(np.prod(lat)) * 12
    Dm = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1
        Dm[:, k] = dirac.apply_D(U, S, e.reshape(lat + (4, 3)), mu, bc_t).ravel()
    return Dm


def test_smallest_singular_value_bounded_by_mu():
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.8, seed=3).numpy()
    kappa = 1 / (2 * (4 - 3.2))  # strongly negative mass: D_W nearly singular
    for mu in (0.05, 0.3):
        Dm = dense_D(U, dirac.site_term(U, kappa, 1.0), mu)
        smin = np.linalg.svd(Dm, compute_uv=False).min()
        assert smin >= abs(mu) * (1 - 1e-12)
        # the eigenvalues of H(mu) = Gamma5 D(mu) are lambda_j + i mu with lambda_j real
        g5 = np.kron(np.ones(16), np.kron([1, 1, -1, -1], np.ones(3)))
        ev = np.linalg.eigvals(g5[:, None] * Dm)
        assert np.max(np.abs(ev.imag - mu)) < 1e-10


def test_even_odd_eigenvalue_relation_csw0():
    """c_sw = 0, mu = 0: lambda_D/(m+4) = 1 -/+ sqrt(1 - lambda_Dhat/(m+4)) (Sec. 2.1)."""
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.5, seed=8).numpy()
    kappa = 0.15
    m = 1 / (2 * kappa) - 4
    Dm = dense_D(U, dirac.site_term(U, kappa, 0.0), 0.0)
    par = np.repeat(dirac.parity(U.shape[:4]).ravel(), 12)
    e, o = par == 0, par == 1
    Dhat = Dm[np.ix_(e, e)] - Dm[np.ix_(e, o)] @ np.linalg.solve(Dm[np.ix_(o, o)], Dm[np.ix_(o, e)])
    lam_hat = np.linalg.eigvals(Dhat)
    lam = np.linalg.eigvals(Dm)
    for lh in lam_hat:
        for sgn in (+1, -1):
            cand = (m + 4) * (1 + sgn * np.sqrt(1 - lh / (m + 4) + 0j))
            assert np.min(np.abs(lam - cand)) < 1e-9


def test_synthetic_links_are_su3():
    """The input generator's exp(i eps H) is special unitary to rounding, for the
    small eps of the gauge fields and eps = 1 of the gauge transformations."""
    import torch
    for eps in (0.12, 0.3, 1.0):
        U = synth.random_hermitian_exp((64, 4), eps, seed=1).numpy()
        uu = U @ dirac.dagger(U)
        assert np.max(np.abs(uu - np.eye(3))) < 1e-14
        assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-14
    # exp(i eps H) = V diag(e^{i eps w}) V^dagger with (w, V) from a library eigensolver
    H = np.array([[1.0, 0.5 - 0.2j, 0.1j], [0.5 + 0.2j, -0.3, 0.4], [-0.1j, 0.4, -0.7]])
    w, Vv = np.linalg.eigh(H)
    want = Vv @ np.diag(np.exp(1j * 0.8 * w)) @ Vv.conj().T
    got = synth.expm_i_hermitian(torch.from_numpy(H)[None], 0.8).numpy()[0]
    assert np.max(np.abs(got - want)) < 1e-14


@pytest.mark.parametrize("bc_t", [0, 1])
def test_slab_decomposed_D_equals_whole_lattice(bc_t):
    """oracle/slabs.py: D evaluated per t-slab with a halo of one layer reproduces the whole-lattice
    oracle D (the clover term included), both time boundary conditions, in-process and in a pool."""
    from oracle import slabs
    from oracle.operators import FineOperator
    dims = (12, 4, 6, 4)
    U = synth.gauge_field(dims, 0.4, seed=21).numpy()
    op = FineOperator(U, 0.13, 1.7, bc_t)
    psis = [synth.gaussian_spinor(dims, seed=22 + r).numpy() for r in range(2)]
    want = [op.apply(p, 0.07) for p in psis]
    for workers, slab in ((0, 3), (2, 4)):
        got = slabs.apply_D_slabs(U, 0.13, 1.7, psis, 0.07, bc_t, slab=slab, workers=workers)
        for g, w in zip(got, want):
            assert np.max(np.abs(g - w)) <= 1e-13 * np.max(np.abs(w))
