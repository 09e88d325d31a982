"""Pins of the oracle's twist that differs on even and odd sites (a library feature of the paper's
appendix, for the Hasenbusch-preconditioned HMC with even-odd preconditioning, where D_hat + i rho
Gamma5_hat is inverted; Sec. 3.1 and the HMC figure).

* The twist pair (mu, mu) is the ordinary twist; the definition i Gamma5 (mu_e P_e + mu_o P_o) holds
  site by site; Gamma5-hermiticity becomes Gamma5 D(mu_e, mu_o) Gamma5 = D(-mu_e, -mu_o)^dagger.
* Its odd-site Schur complement is D_hat(mu_e, mu_e) + i (mu_o - mu_e) Gamma5_hat: an odd-site
  shift is exactly the operator the HMC inverts.
* Galerkin: the coarse operator with the projected parity weight equals the dense P^dagger D P for
  a pair, on two and three levels (the weight Q projects recursively).
* The two-level solve reaches 1e-10 and the dense LU solution for a pair.
"""

import numpy as np
import pytest

from oracle import aggregation, blocks, coarse, dirac, mg, sap
from oracle.operators import FineOperator
from paper_1610_02370_gb300 import synth

DIMS4 = (4, 4, 4, 4)
B2 = (2, 2, 2, 2)
PAIR = (0.03, 0.21)


def dense(apply, shape):
    n = int(np.prod(shape))
    M = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1
        M[:, k] = apply(e.reshape(shape)).ravel()
    return M


def dense_P(op, W, bdims):
    """P as a matrix, columns ordered (aggregate, s, i) with the aggregates in canonical order."""
    nv = W.shape[1]
    cl = blocks.coarse_lat(op.lat, bdims)
    ab = blocks.axis_blocks(op.lat, bdims)
    idx = np.indices(op.lat)
    agg = np.ravel_multi_index([idx[a] // ab[a] for a in range(4)], cl).ravel()
    nd = int(np.prod(op.dof))
    P = np.zeros((int(np.prod(op.lat)) * nd, int(np.prod(cl)) * 2 * nv), dtype=complex)
    for s in range(2):
        for i in range(nv):
            col = W[s, i].reshape(-1, nd)
            for site in range(col.shape[0]):
                P[site * nd:(site + 1) * nd, agg[site] * 2 * nv + s * nv + i] = col[site]
    return P


@pytest.fixture(scope="module")
def fine():
    U = synth.gauge_field(DIMS4, 0.3, seed=0).numpy()
    return FineOperator(U, 0.125, 1.0)


def masks(op):
    par = dirac.parity(op.lat).reshape(op.lat + (1,) * len(op.dof))
    return par == 0, par == 1


def test_pair_definition_reduction_and_gamma5_hermiticity(fine):
    v = synth.gaussian_spinor(DIMS4, seed=1).numpy()
    w = synth.gaussian_spinor(DIMS4, seed=2).numpy()
    E, O = masks(fine)
    assert np.allclose(fine.apply(v, (0.07, 0.07)), fine.apply(v, 0.07), atol=1e-14)
    want = fine.apply(v, 0.0) + dirac.apply_twist(v * E, PAIR[0]) + dirac.apply_twist(v * O, PAIR[1])
    assert np.max(np.abs(fine.apply(v, PAIR) - want)) < 1e-14
    g5 = dirac.apply_Gamma5
    lhs = np.vdot(w, g5(fine.apply(g5(v), PAIR)))
    rhs = np.vdot(fine.apply(w, (-PAIR[0], -PAIR[1])), v)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_schur_complement_of_pair_is_odd_site_shift(fine):
    """D_hat(mu_e, mu_o) = D_oo(mu_o) - D_oe D_ee(mu_e)^-1 D_eo = D_hat(mu_e, mu_e) + i (mu_o - mu_e) Gamma5."""
    E, O = masks(fine)

    def d_hat(v, mu):
        t = fine.site_inv(E * fine.hop(O * v), mu) * E
        return O * fine.site(O * v, mu) - O * fine.hop(t)

    v = synth.gaussian_spinor(DIMS4, seed=3).numpy() * O
    got = d_hat(v, PAIR)
    want = d_hat(v, (PAIR[0], PAIR[0])) + dirac.apply_twist(v, PAIR[1] - PAIR[0])
    assert np.max(np.abs(got - want)) < 1e-13


def test_galerkin_of_pair_is_dense_product(fine):
    nv = 4
    v = synth.gaussian_vectors((nv,) + fine.lat + fine.dof, seed=4).numpy()
    W = aggregation.build_P(fine, v, B2)
    cop = coarse.build_coarse_operator(fine, W, B2)
    P = dense_P(fine, W, B2)
    Df = dense(lambda x: fine.apply(x, PAIR), fine.lat + fine.dof)
    want = P.conj().T @ Df @ P
    got = dense(lambda x: cop.apply(x, PAIR), cop.lat + cop.dof)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    # Q is Hermitian and commutes with Gamma5_c (block diagonal in chirality)
    Q = cop.Q
    assert np.allclose(Q, np.conj(np.swapaxes(Q, -1, -2)), atol=1e-14)
    assert np.allclose(Q * cop.g5c[None, :], Q * cop.g5c[:, None], atol=1e-14)


def test_three_level_galerkin_of_pair():
    """Level 2 = dense P_1^dagger D_1(pair) P_1 with D_1 itself a Galerkin operator: the projected
    parity weight recurses."""
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.3, seed=0).numpy()
    op = FineOperator(U, 0.125, 1.0)
    p = mg.Params(nlevels=3, nv=[2, 2], bdims=[B2, B2])
    lat1 = tuple(n // 2 for n in op.lat)
    v0 = synth.gaussian_vectors((2,) + op.lat + (4, 3), seed=31).numpy()
    v1 = synth.gaussian_vectors((2,) + lat1 + (4,), seed=32).numpy()
    h = mg.hierarchy_from_vectors(op, p, [v0, v1])
    D1, D2 = h.ops[1], h.ops[2]
    P1 = dense_P(D1, h.W[1], B2)
    D1m = dense(lambda x: D1.apply(x, PAIR), D1.lat + D1.dof)
    want = P1.conj().T @ D1m @ P1
    got = dense(lambda x: D2.apply(x, PAIR), D2.lat + D2.dof)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_two_level_solve_with_pair(fine):
    p = mg.Params(nlevels=2, n_setup=2, nv=[8], bdims=[B2], post_smooth=2, nmr=3)
    tv0 = [synth.gaussian_vectors((8,) + fine.lat + fine.dof, seed=21).numpy()]
    h = mg.setup(fine, p, PAIR, tv0)
    b = synth.gaussian_spinor(DIMS4, seed=1).numpy()
    x, info = mg.solve(h, b, PAIR)
    assert info["converged"]
    assert dirac.norm(b - fine.apply(x, PAIR)) <= 1e-10 * dirac.norm(b)
    Dm = dense(lambda y: fine.apply(y, PAIR), fine.lat + fine.dof)
    xs = np.linalg.solve(Dm, b.ravel())
    assert np.linalg.norm(x.ravel() - xs) <= 1e-8 * np.linalg.norm(xs)


def block_sets(lat, bdims, nd):
    """(dofs, colour) of every block, sites in canonical order."""
    cl = blocks.coarse_lat(lat, bdims)
    ab = blocks.axis_blocks(lat, bdims)
    idx = np.indices(lat)
    cidx = [idx[a] // ab[a] for a in range(4)]
    bid = np.ravel_multi_index(cidx, cl).ravel()
    colour = (sum(cidx) % 2).ravel()
    out = []
    for b in range(int(np.prod(cl))):
        sites = np.flatnonzero(bid == b)
        out.append(((sites[:, None] * nd + np.arange(nd)[None, :]).ravel(), colour[sites[0]]))
    return out


def one_sap_cycle_dense(Dm, sets, bv):
    """Red blocks then black, each block solved exactly on the recomputed residual."""
    x = np.zeros_like(bv)
    for colour in (0, 1):
        r = bv - Dm @ x
        for dofs, c in sets:
            if c == colour:
                x[dofs] += np.linalg.solve(Dm[np.ix_(dofs, dofs)], r[dofs])
    return x


@pytest.mark.parametrize("eo", [True, False])
def test_sap_with_pair_equals_dense_block_inverses(fine, eo):
    """SAP (Sec. 2.4) with the twist pair and MR run to convergence equals one red-black cycle of exact
    solves with the diagonal blocks of the dense D(mu_e, mu_o): the smoother sees the pair through its
    site terms (even-odd: A_ee^-1 at mu_e, A_oo at mu_o) and nowhere else."""
    Dm = dense(lambda x: fine.apply(x, PAIR), fine.lat + fine.dof)
    b = synth.gaussian_spinor(DIMS4, seed=41).numpy()
    want = one_sap_cycle_dense(Dm, block_sets(fine.lat, B2, 12), b.ravel())
    got = sap.sap(fine, b, PAIR, B2, ncycles=1, nmr=150, eo=eo).ravel()
    assert np.linalg.norm(got - want) < 1e-10 * np.linalg.norm(want)


def test_coarse_sap_with_pair_equals_dense_block_inverses():
    """The same on a coarse operator carrying a parity weight Q (the level-1 smoother of three levels
    under a twist pair): random nearest-neighbour blocks and a random Hermitian Q that commutes with
    Gamma5_c on a 4^4 coarse lattice, 2^4 blocks, even-odd and full block solves."""
    from oracle.operators import CoarseOperator
    rng = np.random.default_rng(44)
    lat, nv = (4, 4, 4, 4), 2
    n = 2 * nv
    bl = 0.12 * (rng.standard_normal((9,) + lat + (n, n)) + 1j * rng.standard_normal((9,) + lat + (n, n)))
    bl[0] += 1.5 * np.eye(n)
    A = rng.standard_normal(lat + (n, n)) + 1j * rng.standard_normal(lat + (n, n))
    Q = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    Q[..., :nv, nv:] = 0
    Q[..., nv:, :nv] = 0
    cop = CoarseOperator(bl, nv, Q=Q)
    Dm = dense(lambda x: cop.apply(x, PAIR), cop.lat + cop.dof)
    b = rng.standard_normal(lat + (n,)) + 1j * rng.standard_normal(lat + (n,))
    want = one_sap_cycle_dense(Dm, block_sets(lat, B2, n), b.ravel())
    for eo in (True, False):
        got = sap.sap(cop, b, PAIR, B2, ncycles=1, nmr=150, eo=eo).ravel()
        assert np.linalg.norm(got - want) < 1e-10 * np.linalg.norm(want), eo
