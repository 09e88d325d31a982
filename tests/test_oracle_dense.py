"""Brute-force pin of the oracle's D(mu) (Sec. 2.1): the dense matrix assembled entry by entry from the
formula, with explicit site loops and modular coordinate arithmetic (no array shifts), equals the matrix
of the oracle's operator on 2^4 and 4^4 lattices (4^4: 3072 unknowns), periodic and antiperiodic in t.

Per site x: the site block (m + 4) I - c_sw/32 sum_{mu != nu} (gamma_mu gamma_nu) x (Q_mu_nu - Q_nu_mu)
+ i mu gamma5 x I_3, with Q_mu_nu(x) the four plaquette leaves in the mu-nu plane around x, all with
the same orientation; hopping blocks -1/2 (I - gamma_mu) x U_mu(x) to x + mu_hat and
-1/2 (I + gamma_mu) x U_mu(x - mu_hat)^dagger to x - mu_hat, with a sign -1 on hops that wrap in t for
antiperiodic boundaries.  Spin-colour index 3 spin + colour, site index ((t Lz + z) Ly + y) Lx + x.
"""

import numpy as np
import pytest

from oracle import dirac
from oracle.operators import FineOperator
from paper_1610_02370_gb300 import synth


def brute_force_D(U, kappa, csw, mu, dims, bc_t):
    T, X, Y, Z = dims
    L = (T, X, Y, Z)  # extent per direction mu = t, x, y, z
    V = T * X * Y * Z
    g, g5 = dirac.gamma_matrices()
    i4, i3 = np.eye(4), np.eye(3)
    m = 1.0 / (2.0 * kappa) - 4.0

    def index(c):
        t, x, y, z = (c[k] % L[k] for k in range(4))
        return ((t * Z + z) * Y + y) * X + x

    def link(c, d):
        t, x, y, z = (c[k] % L[k] for k in range(4))
        return U[t, z, y, x, d]

    def step(c, d, s):
        c = list(c)
        c[d] += s
        return c

    def leaves(c, a, b):
        """Sum of the four oriented plaquettes in the (a, b) plane that touch site c."""
        dag = lambda A: A.conj().T
        xa, xb = step(c, a, 1), step(c, b, 1)
        xma, xmb = step(c, a, -1), step(c, b, -1)
        xmab = step(xma, b, -1)
        q = link(c, a) @ link(xa, b) @ dag(link(xb, a)) @ dag(link(c, b))
        q = q + link(c, b) @ dag(link(step(xma, b, 1), a)) @ dag(link(xma, b)) @ link(xma, a)
        q = q + dag(link(xma, a)) @ dag(link(xmab, b)) @ link(xmab, a) @ link(xmb, b)
        q = q + dag(link(xmb, b)) @ link(xmb, a) @ link(step(xmb, a, 1), b) @ dag(link(c, a))
        return q

    D = np.zeros((12 * V, 12 * V), dtype=complex)
    for t in range(T):
        for x in range(X):
            for y in range(Y):
                for z in range(Z):
                    c = [t, x, y, z]
                    i = index(c)
                    S = (m + 4.0) * np.eye(12, dtype=complex)
                    for a in range(4):
                        for b in range(4):
                            if a != b:
                                Qab = leaves(c, a, b)
                                S -= csw / 32.0 * np.kron(g[a] @ g[b], Qab - Qab.conj().T)
                    S += 1j * mu * np.kron(g5, i3)
                    D[12 * i:12 * i + 12, 12 * i:12 * i + 12] += S
                    for d in range(4):
                        fwd, bwd = step(c, d, 1), step(c, d, -1)
                        sf = -1.0 if (d == 0 and bc_t == 1 and c[0] == T - 1) else 1.0
                        sb = -1.0 if (d == 0 and bc_t == 1 and c[0] == 0) else 1.0
                        j, k = index(fwd), index(bwd)
                        D[12 * i:12 * i + 12, 12 * j:12 * j + 12] += -0.5 * sf * np.kron(i4 - g[d], link(c, d))
                        D[12 * i:12 * i + 12, 12 * k:12 * k + 12] += (-0.5 * sb *
                                                                       np.kron(i4 + g[d], link(bwd, d).conj().T))
    return D


def oracle_matrix(op, mu):
    shape = op.lat + op.dof
    n = int(np.prod(shape))
    M = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1
        M[:, k] = op.apply(e.reshape(shape), mu).ravel()
    return M


@pytest.mark.parametrize("dims,bc_t", [((2, 2, 2, 2), 0), ((2, 2, 2, 2), 1), ((4, 4, 4, 4), 0), ((4, 4, 4, 4), 1)])
def test_dense_matrix_from_the_formula(dims, bc_t):
    U = synth.gauge_field(dims, 0.3, seed=0).numpy()
    kappa, csw, mu = 0.125, 1.0, 0.01
    op = FineOperator(U, kappa, csw, bc_t)
    want = brute_force_D(U, kappa, csw, mu, dims, bc_t)
    got = oracle_matrix(op, mu)
    assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want))


@pytest.mark.parametrize("bc_t,theta", [(0, None), (1, None), (1, [0.5, -1.2, 0.8, 2.0])])
def test_site_local_evaluation_matches_the_operator(bc_t, theta):
    """oracle/local.py (D psi at chosen sites, for parity on lattices too large for a full oracle
    application) equals the oracle's operator at every site of a 4 x 2 x 4 x 2 lattice and at random
    sites of a 4^4 lattice, for periodic, antiperiodic and twisted boundaries."""
    from oracle import local
    for dims, allsites in (((4, 2, 4, 2), True), ((4, 4, 4, 4), False)):
        U = synth.gauge_field(dims, 0.3, seed=2).numpy()
        psi = synth.gaussian_spinor(dims, seed=3).numpy()
        kappa, csw, mu = 0.13, 1.4, 0.07
        full = dirac.apply_D(U, dirac.site_term(U, kappa, csw), psi, mu, bc_t, theta)
        T, X, Y, Z = dims
        if allsites:
            sites = [(t, x, y, z) for t in range(T) for x in range(X) for y in range(Y) for z in range(Z)]
        else:
            rng = np.random.default_rng(4)
            sites = [tuple(int(rng.integers(0, n)) for n in dims) for _ in range(24)]
        got = local.apply_D_at_sites(U, kappa, csw, psi, mu, sites, bc_t, theta)
        want = np.array([full[t, z, y, x] for (t, x, y, z) in sites])
        assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("bc_t", [0, 1])
def test_sap_cycle_at_blocks_matches_the_whole_lattice_sap(bc_t):
    """oracle/local.py's SAP cycle at chosen blocks (dense block matrices, for parity on lattices too
    large for the whole-lattice oracle) equals the oracle's SAP (one cycle from x = 0, even-odd block MR,
    3 steps) on an 8^4 lattice with 4^4 blocks, at a red and at a black block."""
    from oracle import local, sap
    dims, B = (8, 8, 8, 8), (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, seed=3).numpy()
    b = synth.gaussian_spinor(dims, seed=4).numpy()
    kappa, csw, mu = 0.13, 1.4, 0.05
    full = sap.sap(FineOperator(U, kappa, csw, bc_t), b, mu, B, ncycles=1, nmr=3, eo=True)
    for bc in ((0, 0, 0, 0), (1, 1, 1, 0)):
        got = local.sap_cycle_at_block(U, kappa, csw, b, mu, B, bc, 3, bc_t)
        want = np.array([full[t, z, y, x] for (t, x, y, z) in local.block_sites(B, bc)])
        assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.parametrize("bc_t", [0, 1])
def test_galerkin_columns_at_blocks_match_the_whole_lattice_operator(bc_t):
    """oracle/local.py's Galerkin operator at chosen aggregates (P per aggregate, dense block couplings,
    for parity on lattices too large for the whole-lattice oracle) equals the columns D_c(mu) e_(A, r) of
    the oracle's coarse operator on 8^4 with 2^4 aggregates (4 per direction, so the 8 neighbours are
    distinct), at an interior and at a corner aggregate whose neighbours wrap around; D_c e_(A, r)
    vanishes away from A and its neighbours."""
    from oracle import aggregation, coarse, local
    dims, B, nv, mu = (8, 8, 8, 8), (2, 2, 2, 2), 4, 0.05
    U = synth.gauge_field(dims, 0.3, seed=3).numpy()
    op = FineOperator(U, 0.13, 1.4, bc_t)
    v = synth.gaussian_vectors((nv,) + op.lat + op.dof, seed=5).numpy()
    cop = coarse.build_coarse_operator(op, aggregation.build_P(op, v, B), B)
    for A in ((1, 2, 1, 2), (3, 0, 3, 0)):
        cols = local.coarse_columns_at_block(U, 0.13, 1.4, lambda bc: v[(slice(None),) + local.block_slices(B, bc)],
                                             mu, B, A, bc_t)
        assert len(cols) == 9
        for r in range(2 * nv):
            e = np.zeros(cop.lat + cop.dof, dtype=complex)
            e[A[0], A[3], A[2], A[1], r] = 1
            y = cop.apply(e, mu)
            scale = np.abs(y).max()
            for bc, M in cols.items():
                assert np.abs(M[:, r] - y[bc[0], bc[3], bc[2], bc[1]]).max() <= 1e-13 * scale
                y[bc[0], bc[3], bc[2], bc[1]] = 0
            assert np.abs(y).max() == 0
