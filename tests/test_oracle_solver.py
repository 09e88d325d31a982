"""Pins of the oracle's SAP, aggregation, Galerkin, Krylov and multigrid code.

SAP (Sec. 2.4): with the block MR run to convergence, one cycle equals the
product of dense block inverses applied red then black (on the fine operator,
and on a coarse operator as the smoother of an intermediate level); MR steps satisfy their
defining orthogonality; on a block-diagonal operator one cycle solves exactly.
Aggregation (Sec. 2.3): P^dagger P = I, Gamma5 P = P Gamma5_c, the test vectors
lie in range(P), P equals the Q factor of a library QR per aggregate half.
Galerkin (Sec. 2.3): D_c equals the dense P^dagger D P (+ i mu Gamma5_c),
Gamma5_c-hermiticity, nearest-neighbour sparsity, and the free-field closed
form D_c = m + sum_mu (1 - cos q_mu)/b_mu + i sum_mu gamma_mu sin(q_mu)/b_mu + i mu gamma5.
Krylov (Sec. 2.5): GMRES/FGMRES iterates minimise the residual over their
Krylov space (checked against library least squares), even-odd GMRES solves
the coarse system and its retrieval makes the even rows exact.
Multigrid (Sec. 2.2): the preconditioner's error propagation is
E_SAP^k (I - P D_c^-1 R D); the two-level solve reaches 1e-10 and the dense
solution, for +mu and -mu with one setup.  Three levels (the K-cycle of
Sec. 2.2 / 2.5 with FGMRES on the intermediate level): the level-2 operator is
the dense Galerkin product of the level-1 operator, and the solve reaches 1e-10.
Even-odd CG on the squared reduced operator (the baseline of Sec. 3.1.2): its
adjoint is the true adjoint and it reproduces the dense solution.
"""

import numpy as np
import pytest

from oracle import aggregation, blocks, coarse, dirac, krylov, mg, sap
from oracle.operators import CoarseOperator, FineOperator
from paper_1610_02370_gb300 import synth

DIMS4 = (4, 4, 4, 4)
B2 = (2, 2, 2, 2)


def dense(apply, shape):
    n = int(np.prod(shape))
    M = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1
        M[:, k] = apply(e.reshape(shape)).ravel()
    return M


@pytest.fixture(scope="module")
def fine():
    U = synth.gauge_field(DIMS4, 0.3, seed=0).numpy()
    return FineOperator(U, 0.125, 1.0)


@pytest.fixture(scope="module")
def fine_dense(fine):
    mu = 0.01
    return dense(lambda v: fine.apply(v, mu), fine.lat + fine.dof), mu


def block_index_sets(op, bdims):
    lat = op.lat
    nd = int(np.prod(op.dof))
    cl = blocks.coarse_lat(lat, bdims)
    bid = np.zeros(lat, dtype=int)
    ab = blocks.axis_blocks(lat, bdims)
    idx = np.indices(lat)
    cidx = [idx[a] // ab[a] for a in range(4)]
    bid = np.ravel_multi_index(cidx, cl)
    colour = (sum(cidx) % 2).ravel()
    sets = []
    for b in range(int(np.prod(cl))):
        sites = np.flatnonzero(bid.ravel() == b)
        dofs = (sites[:, None] * nd + np.arange(nd)[None, :]).ravel()
        sets.append((dofs, colour[sites[0]]))
    return sets


def block_inverse_dense(Dm, sets, colour):
    B = np.zeros_like(Dm)
    for dofs, c in sets:
        if c == colour:
            B[np.ix_(dofs, dofs)] = np.linalg.inv(Dm[np.ix_(dofs, dofs)])
    return B


@pytest.mark.parametrize("eo", [True, False])
def test_sap_converged_mr_equals_dense_block_inverses(fine, fine_dense, eo):
    Dm, mu = fine_dense
    sets = block_index_sets(fine, B2)
    Br, Bb = block_inverse_dense(Dm, sets, 0), block_inverse_dense(Dm, sets, 1)
    b = synth.gaussian_spinor(DIMS4, seed=5).numpy()
    bv = b.ravel()
    x1 = Br @ bv
    x2 = x1 + Bb @ (bv - Dm @ x1)
    got = sap.sap(fine, b, mu, B2, ncycles=1, nmr=120, eo=eo).ravel()
    assert np.linalg.norm(got - x2) < 1e-10 * np.linalg.norm(x2)
    # two cycles: error propagator E = (I - Bb D)(I - Br D) applied twice
    xs = np.linalg.solve(Dm, bv)
    E = (np.eye(len(bv)) - Bb @ Dm) @ (np.eye(len(bv)) - Br @ Dm)
    want = xs - E @ (E @ xs)
    got2 = sap.sap(fine, b, mu, B2, ncycles=2, nmr=120, eo=eo).ravel()
    assert np.linalg.norm(got2 - want) < 1e-10 * np.linalg.norm(want)


def dense_mr(A, rhs, nmr):
    """nmr steps of the minimal residual method on the dense system A e = rhs from e = 0."""
    e = np.zeros_like(rhs)
    rho = rhs.copy()
    for _ in range(nmr):
        p = A @ rho
        den = np.vdot(p, p).real
        al = np.vdot(p, rho) / den if den > 0 else 0.0
        e = e + al * rho
        rho = rho - al * p
    return e


@pytest.mark.parametrize("eo", [True, False])
def test_sap_finite_mr_equals_dense_block_computation(fine, fine_dense, eo):
    """One SAP cycle with 3 MR steps per block equals the same steps taken on the dense block
    matrices: red blocks then black on the recomputed residual; per block either MR on the block or,
    even-odd, MR on the Schur complement A_oo - A_oe A_ee^-1 A_eo of the block matrix followed by
    e_e = A_ee^-1 (r_e - A_eo e_o)."""
    Dm, mu = fine_dense
    sets = block_index_sets(fine, B2)
    nd = 12
    par = (np.indices(fine.lat).sum(axis=0) % 2).ravel()
    b = synth.gaussian_spinor(DIMS4, seed=10).numpy()
    bv = b.ravel()
    x = np.zeros_like(bv)
    for colour in (0, 1):
        r = bv - Dm @ x
        for dofs, c in sets:
            if c != colour:
                continue
            A = Dm[np.ix_(dofs, dofs)]
            rb = r[dofs]
            if not eo:
                x[dofs] += dense_mr(A, rb, 3)
                continue
            site_par = par[dofs // nd]
            ev, od = np.flatnonzero(site_par == 0), np.flatnonzero(site_par == 1)
            Aee, Aeo = A[np.ix_(ev, ev)], A[np.ix_(ev, od)]
            Aoe, Aoo = A[np.ix_(od, ev)], A[np.ix_(od, od)]
            Aee_inv = np.linalg.inv(Aee)
            Ahat = Aoo - Aoe @ Aee_inv @ Aeo
            eo_ = dense_mr(Ahat, rb[od] - Aoe @ Aee_inv @ rb[ev], 3)
            ee = Aee_inv @ (rb[ev] - Aeo @ eo_)
            e = np.zeros_like(rb)
            e[ev], e[od] = ee, eo_
            x[dofs] += e
    got = sap.sap(fine, b, mu, B2, ncycles=1, nmr=3, eo=eo).ravel()
    assert np.linalg.norm(got - x) <= 1e-13 * np.linalg.norm(x)


def random_coarse_operator(lat, nv, seed):
    """A coarse operator with the nearest-neighbour block structure of Sec. 2.3 and random
    complex blocks (self blocks shifted to be well conditioned)."""
    rng = np.random.default_rng(seed)
    n = 2 * nv
    shape = (9,) + lat + (n, n)
    bl = 0.12 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    bl[0] += 1.5 * np.eye(n)
    return CoarseOperator(bl, nv)


@pytest.mark.parametrize("eo", [True, False])
def test_sap_on_coarse_operator_equals_dense_block_inverses(eo):
    """The smoother of an intermediate level (three levels): SAP on a coarse operator with 2^4
    blocks of a 4^4 coarse lattice, MR run to convergence, equals red-then-black dense block
    inverses, one and two cycles (its error propagator (I - B_bb D)(I - B_rr D))."""
    cop = random_coarse_operator((4, 4, 4, 4), 2, seed=3)
    mu = 0.05
    Dm = dense(lambda v: cop.apply(v, mu), cop.lat + cop.dof)
    sets = block_index_sets(cop, B2)
    Br, Bb = block_inverse_dense(Dm, sets, 0), block_inverse_dense(Dm, sets, 1)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(cop.lat + cop.dof) + 1j * rng.standard_normal(cop.lat + cop.dof)
    bv = b.ravel()
    x1 = Br @ bv
    x2 = x1 + Bb @ (bv - Dm @ x1)
    got = sap.sap(cop, b, mu, B2, ncycles=1, nmr=120, eo=eo).ravel()
    assert np.linalg.norm(got - x2) < 1e-10 * np.linalg.norm(x2)
    xs = np.linalg.solve(Dm, bv)
    E = (np.eye(len(bv)) - Bb @ Dm) @ (np.eye(len(bv)) - Br @ Dm)
    want = xs - E @ (E @ xs)
    got2 = sap.sap(cop, b, mu, B2, ncycles=2, nmr=120, eo=eo).ravel()
    assert np.linalg.norm(got2 - want) < 1e-10 * np.linalg.norm(want)


def test_mr_steps_are_residual_minimising(fine, fine_dense):
    """Full-block MR: e1 = a1 r with <A r, r - a1 A r> = 0 per block, and the second step
    does the same on the updated residual."""
    Dm, mu = fine_dense
    sets = block_index_sets(fine, B2)
    r = synth.gaussian_spinor(DIMS4, seed=6).numpy()
    e1 = sap.block_solve(fine, r, mu, B2, 0, 1, eo=False).ravel()
    e2 = sap.block_solve(fine, r, mu, B2, 0, 2, eo=False).ravel()
    rv = r.ravel()
    for dofs, c in sets:
        if c != 0:
            assert np.all(e1[dofs] == 0)
            continue
        A = Dm[np.ix_(dofs, dofs)]
        rb = rv[dofs]
        a1 = np.vdot(rb, e1[dofs]) / np.vdot(rb, rb)
        assert np.allclose(e1[dofs], a1 * rb, atol=1e-14)
        p = A @ rb
        assert abs(np.vdot(p, rb - a1 * p)) < 1e-12 * np.linalg.norm(p) * np.linalg.norm(rb)
        rho1 = rb - A @ e1[dofs]
        d = e2[dofs] - e1[dofs]
        a2 = np.vdot(rho1, d) / np.vdot(rho1, rho1)
        assert np.allclose(d, a2 * rho1, atol=1e-13)
        p2 = A @ rho1
        assert abs(np.vdot(p2, rho1 - a2 * p2)) < 1e-12 * np.linalg.norm(p2) * np.linalg.norm(rho1)


def test_sap_block_diagonal_operator_solved_in_one_cycle():
    U = synth.gauge_field(DIMS4, 0.3, seed=1).numpy().copy()
    for mu_ in range(4):
        cut = blocks.crossing_mask(U.shape[:4], B2, mu_, +1)
        U[..., mu_, :, :][cut] = 0.0
    op = FineOperator(U, 0.125, 1.0)
    b = synth.gaussian_spinor(DIMS4, seed=2).numpy()
    for eo in (True, False):
        x = sap.sap(op, b, 0.02, B2, ncycles=1, nmr=150, eo=eo)
        r = b - op.apply(x, 0.02)
        assert dirac.norm(r) < 1e-10 * dirac.norm(b)


@pytest.fixture(scope="module")
def agg(fine):
    nv = 4
    v = synth.gaussian_vectors((nv,) + fine.lat + fine.dof, seed=3).numpy()
    W = aggregation.build_P(fine, v, B2)
    return v, W


def test_P_orthonormal_and_gamma5_compatible(fine, agg):
    v, W = agg
    nv = v.shape[0]
    lat = fine.lat
    for s in range(2):
        for t in range(2):
            for i in range(nv):
                for j in range(nv):
                    g = blocks.block_sum(np.conj(W[s, i]) * W[t, j], lat, B2)
                    assert np.max(np.abs(g - (1.0 if (s, i) == (t, j) else 0.0))) < 1e-13
        for i in range(nv):
            assert np.max(np.abs(dirac.apply_Gamma5(W[s, i]) - (1 - 2 * s) * W[s, i])) == 0
    for i in range(nv):  # test vectors lie in range(P)
        back = aggregation.prolong(W, aggregation.restrict(W, v[i], lat, B2), lat, B2)
        assert np.max(np.abs(back - v[i])) < 1e-12 * np.max(np.abs(v[i]))


def test_P_is_library_QR_per_aggregate_half(fine, agg):
    v, W = agg
    nv = v.shape[0]
    for dofs, _ in block_index_sets(fine, B2):
        for s in range(2):
            chir = np.zeros(12, dtype=bool)
            chir[6 * s:6 * s + 6] = True
            sel = dofs[np.tile(chir, len(dofs) // 12)]
            Vm = np.stack([v[i].ravel()[sel] for i in range(nv)], axis=1)
            Q, R = np.linalg.qr(Vm)
            Q = Q * (np.conj(np.diag(R)) / np.abs(np.diag(R)))[None, :]
            Wm = np.stack([W[s, i].ravel()[sel] for i in range(nv)], axis=1)
            assert np.max(np.abs(Q - Wm)) < 1e-13


def dense_P(op, W, bdims):
    nv = W.shape[1]
    cl = blocks.coarse_lat(op.lat, bdims)
    ncs = int(np.prod(cl))
    sets = block_index_sets(op, bdims)
    nf = int(np.prod(op.lat + op.dof))
    P = np.zeros((nf, ncs * 2 * nv), dtype=complex)
    for a, (dofs, _) in enumerate(sets):
        for s in range(2):
            for i in range(nv):
                P[dofs, a * 2 * nv + s * nv + i] = W[s, i].ravel()[dofs]
    return P


def test_restrict_prolong_are_adjoint_and_match_dense_P(fine, agg):
    v, W = agg
    P = dense_P(fine, W, B2)
    psi = synth.gaussian_spinor(DIMS4, seed=9).numpy()
    c = aggregation.restrict(W, psi, fine.lat, B2)
    assert np.max(np.abs(c.ravel() - P.conj().T @ psi.ravel())) < 1e-12
    cc = synth.gaussian_vectors(c.shape, seed=10).numpy()
    f = aggregation.prolong(W, cc, fine.lat, B2)
    assert np.max(np.abs(f.ravel() - P @ cc.ravel())) < 1e-12


def test_galerkin_equals_dense_product(fine, fine_dense, agg):
    Dm, mu = fine_dense
    v, W = agg
    nv = W.shape[1]
    P = dense_P(fine, W, B2)
    cop = coarse.build_coarse_operator(fine, W, B2)
    shape = cop.lat + cop.dof
    for m in (mu, -0.3):
        Dc = dense(lambda c: cop.apply(c, m), shape)
        D0 = dense(lambda y: fine.apply(y, 0.0), fine.lat + fine.dof)
        ncs = int(np.prod(cop.lat))
        g5c = np.tile(np.concatenate([np.ones(nv), -np.ones(nv)]), ncs)
        want = P.conj().T @ D0 @ P + 1j * m * np.diag(g5c)
        assert np.max(np.abs(Dc - want)) < 1e-13 * np.max(np.abs(want))
        # twist: P^dagger (i m Gamma5) P = i m Gamma5_c exactly
        g5f = np.tile(np.kron([1, 1, -1, -1], np.ones(3)), int(np.prod(fine.lat)))
        assert np.max(np.abs(P.conj().T @ (g5f[:, None] * P) - np.diag(g5c))) < 1e-13
        # Gamma5_c hermiticity: D_c(m)^dagger = Gamma5_c D_c(-m) Gamma5_c
        Dcm = dense(lambda c: cop.apply(c, -m), shape)
        assert np.max(np.abs(Dc.conj().T - g5c[:, None] * Dcm * g5c[None, :])) < 1e-13
    # nearest-neighbour sparsity: coarse sites differing in two directions do not couple
    cl = cop.lat
    n = 2 * nv
    for a in range(ncs):
        ca = np.array(np.unravel_index(a, cl))
        for b in range(ncs):
            cb = np.array(np.unravel_index(b, cl))
            if np.count_nonzero(ca != cb) >= 2:
                assert np.max(np.abs(Dc[a * n:(a + 1) * n, b * n:(b + 1) * n])) == 0


def test_galerkin_with_twisted_boundaries_is_dense_product():
    """Twisted boundaries reach the coarse level through the per-direction hops: D_c = P^dagger D P
    densely, with D the twisted operator (and antiperiodic t on top)."""
    U = synth.gauge_field(DIMS4, 0.3, seed=5).numpy()
    op = FineOperator(U, 0.125, 1.0, 1, theta=[0.6, -0.9, 1.4, 0.3])
    nv = 3
    v = synth.gaussian_vectors((nv,) + op.lat + op.dof, seed=8).numpy()
    W = aggregation.build_P(op, v, B2)
    cop = coarse.build_coarse_operator(op, W, B2)
    mu = 0.04
    P = dense_P(op, W, B2)
    want = P.conj().T @ dense(lambda y: op.apply(y, mu), op.lat + op.dof) @ P
    got = dense(lambda y: cop.apply(y, mu), cop.lat + cop.dof)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


@pytest.mark.parametrize("bc_t", [0, 1])
def test_free_field_coarse_closed_form(bc_t):
    dims = (8, 4, 4, 8)           # T, X, Y, Z
    bd = (2, 2, 4, 4)             # block extents per direction t, x, y, z
    kappa, mu = 0.13, 0.02
    m = 1 / (2 * kappa) - 4
    U = synth.unit_gauge(dims).numpy()
    op = FineOperator(U, kappa, 1.0, bc_t)
    nv = 6
    v = np.zeros((nv,) + op.lat + (4, 3), dtype=complex)
    for k in range(2):
        for c in range(3):
            v[3 * k + c, ..., k, c] = 1.0
            v[3 * k + c, ..., k + 2, c] = 1.0
    W = aggregation.build_P(op, v, bd)
    cop = coarse.build_coarse_operator(op, W, bd)
    cl = cop.lat                  # (NBt, NBz, NBy, NBx)
    nb = (cl[0], cl[3], cl[2], cl[1])  # per direction t, x, y, z
    g, g5 = dirac.gamma_matrices()
    rng = np.random.default_rng(0)
    idx = np.indices(cl)
    X = (idx[0], idx[3], idx[2], idx[1])
    for _ in range(5):
        n = [rng.integers(0, nb[a]) for a in range(4)]
        q = [2 * np.pi * n[a] / nb[a] for a in range(4)]
        if bc_t:
            q[0] = (2 * n[0] + 1) * np.pi / nb[0]
        chi = rng.normal(size=4) + 1j * rng.normal(size=4)
        col = rng.normal(size=3) + 1j * rng.normal(size=3)
        ph = np.exp(1j * sum(q[a] * X[a] for a in range(4)))

        def to_coarse(spinor):
            out = np.zeros(12, dtype=complex)
            for s in range(2):
                for k in range(2):
                    for c in range(3):
                        out[s * 6 + 3 * k + c] = spinor[2 * s + k] * col[c]
            return out
        c = ph[..., None] * to_coarse(chi)[None, None, None, None, :]
        sym = (m + sum((1 - np.cos(q[a])) / bd[a] for a in range(4))) * np.eye(4) \
            + 1j * sum(g[a] * np.sin(q[a]) / bd[a] for a in range(4)) + 1j * mu * g5
        want = ph[..., None] * to_coarse(sym @ chi)[None, None, None, None, :]
        got = cop.apply(c, mu)
        assert np.max(np.abs(got - want)) < 1e-13


def test_gmres_and_fgmres_minimise_over_krylov_space():
    rng = np.random.default_rng(1)
    n, k = 40, 9
    A = 3 * np.eye(n) + rng.normal(size=(n, n)) / np.sqrt(n) + 1j * rng.normal(size=(n, n)) / np.sqrt(n)
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    Mm = np.eye(n) + 0.3 * rng.normal(size=(n, n)) / np.sqrt(n)
    for M in (None, Mm):
        AM = A if M is None else A @ M
        x, info = krylov.fgmres(lambda z: A @ z, b, None if M is None else (lambda z: Mm @ z),
                                restart=k, max_restarts=0, tol=1e-300)
        K = np.stack([np.linalg.matrix_power(AM, j) @ b for j in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        y = np.linalg.lstsq(AM @ Q, b, rcond=None)[0]
        want = Q @ y if M is None else Mm @ (Q @ y)
        assert info['iters'] == k
        assert np.linalg.norm(x - want) < 1e-10 * np.linalg.norm(want)


def small_coarse_operator(seed=0, nv=3, lat=(2, 2, 2, 2)):
    rng = np.random.default_rng(seed)
    n = 2 * nv
    blk = (rng.normal(size=(9,) + lat + (n, n)) + 1j * rng.normal(size=(9,) + lat + (n, n))) * 0.15
    blk[0] += 4.0 * np.eye(n)
    return CoarseOperator(blk, nv)


def test_eo_gmres_solves_and_retrieval_is_exact():
    cop = small_coarse_operator()
    eta = synth.gaussian_vectors(cop.lat + cop.dof, seed=4).numpy()
    mu = 0.05
    Dc = dense(lambda c: cop.apply(c, mu), cop.lat + cop.dof)
    phi, info = krylov.eo_gmres(cop, eta, mu, restart=100, max_restarts=5, tol=1e-13)
    want = np.linalg.solve(Dc, eta.ravel())
    assert np.linalg.norm(phi.ravel() - want) < 1e-11 * np.linalg.norm(want)
    phi1, info1 = krylov.eo_gmres(cop, eta, mu, restart=3, max_restarts=0, tol=1e-1)
    r = (eta.ravel() - Dc @ phi1.ravel()).reshape(eta.shape)
    par = dirac.parity(cop.lat)
    assert np.max(np.abs(r[par == 0])) < 1e-13 * np.max(np.abs(eta))
    assert np.max(np.abs(r[par == 1])) > 1e-6


def test_preconditioner_error_propagation(fine, fine_dense, agg):
    Dm, mu = fine_dense
    v, W = agg
    p = mg.Params(nlevels=2, nv=[v.shape[0]], bdims=[B2], post_smooth=2, nmr=120,
                  coarse_restart=200, coarse_max_restarts=3, coarse_tol=1e-14, delta=5.2)
    h = mg.hierarchy_from_vectors(fine, p, [v])
    b = synth.gaussian_spinor(DIMS4, seed=12).numpy()
    x = h.precondition(0, b, mu).ravel()
    P = dense_P(fine, W, B2)
    D0 = dense(lambda y: fine.apply(y, 0.0), fine.lat + fine.dof)
    nv = v.shape[0]
    g5c = np.tile(np.concatenate([np.ones(nv), -np.ones(nv)]), P.shape[1] // (2 * nv))
    Dc = P.conj().T @ D0 @ P + 1j * p.delta * mu * np.diag(g5c)
    sets = block_index_sets(fine, B2)
    Br, Bb = block_inverse_dense(Dm, sets, 0), block_inverse_dense(Dm, sets, 1)
    E = (np.eye(len(x)) - Bb @ Dm) @ (np.eye(len(x)) - Br @ Dm)
    bv = b.ravel()
    xs = np.linalg.solve(Dm, bv)
    xc = P @ np.linalg.solve(Dc, P.conj().T @ bv)
    want = xs - E @ (E @ (xs - xc))
    assert np.linalg.norm(x - want) < 1e-9 * np.linalg.norm(want)


def test_three_level_preconditioner_with_exact_level1_solve(fine, fine_dense, agg):
    """Three levels with the level-1 FGMRES driven to 1e-14: the level-0 preconditioner equals the
    two-level error propagation with the exact level-1 inverse, E_SAP^k (I - P D_1(mu)^-1 P^dagger D),
    where level 1 (not the coarsest) keeps the twist mu.  Level-1 blocks of single sites on a 2^4
    level-1 lattice keep the dense check small."""
    Dm, mu = fine_dense
    v, W = agg
    nv = v.shape[0]
    B1 = (1, 1, 1, 1)
    p = mg.Params(nlevels=3, nv=[nv, 2], bdims=[B2, B1], post_smooth=2, nmr=120, kcycle_restart=64,
                  kcycle_max_restarts=5, kcycle_tol=1e-14, coarse_restart=60, coarse_max_restarts=2,
                  coarse_tol=1e-6, delta=5.2)
    lat1 = blocks.coarse_lat(fine.lat, B2)
    v1 = synth.gaussian_vectors((2,) + lat1 + (2 * nv,), seed=33).numpy()
    h = mg.hierarchy_from_vectors(fine, p, [v, v1])
    b = synth.gaussian_spinor(DIMS4, seed=12).numpy()
    x = h.precondition(0, b, mu).ravel()
    P = dense_P(fine, W, B2)
    D0 = dense(lambda y: fine.apply(y, 0.0), fine.lat + fine.dof)
    g5c = np.tile(np.concatenate([np.ones(nv), -np.ones(nv)]), P.shape[1] // (2 * nv))
    D1 = P.conj().T @ D0 @ P + 1j * mu * np.diag(g5c)
    sets = block_index_sets(fine, B2)
    Br, Bb = block_inverse_dense(Dm, sets, 0), block_inverse_dense(Dm, sets, 1)
    E = (np.eye(len(x)) - Bb @ Dm) @ (np.eye(len(x)) - Br @ Dm)
    bv = b.ravel()
    xs = np.linalg.solve(Dm, bv)
    xc = P @ np.linalg.solve(D1, P.conj().T @ bv)
    want = xs - E @ (E @ (xs - xc))
    assert np.linalg.norm(x - want) < 1e-9 * np.linalg.norm(want)


def test_two_level_solve_config_4x4x4x4(fine, fine_dense):
    """4^4, eps=0.3, kappa=0.125, c_sw=1.0, mu=0.01: the two-level solve reaches 1e-10 and
    agrees with the dense LU solution; the same setup also solves the -mu flavour."""
    Dm, mu = fine_dense
    p = mg.Params(nlevels=2, n_setup=2, nv=[8], bdims=[B2], post_smooth=2, nmr=3)
    tv0 = [synth.gaussian_vectors((8,) + fine.lat + fine.dof, seed=21).numpy()]
    h = mg.setup(fine, p, mu, tv0)
    b = synth.gaussian_spinor(DIMS4, seed=1).numpy()
    for m in (mu, -mu):
        x, info = mg.solve(h, b, m)
        r = b - fine.apply(x, m)
        assert info['converged']
        assert dirac.norm(r) <= 1e-10 * dirac.norm(b)
        Dmm = Dm if m == mu else dense(lambda y: fine.apply(y, m), fine.lat + fine.dof)
        xs = np.linalg.solve(Dmm, b.ravel())
        assert np.linalg.norm(x.ravel() - xs) <= 1e-8 * np.linalg.norm(xs)
    # setup invariants: orthonormal, Gamma5-compatible P
    W = h.W[0]
    g = blocks.block_sum(np.conj(W[1, 3]) * W[1, 3], fine.lat, B2)
    assert np.max(np.abs(g - 1)) < 1e-13


@pytest.fixture(scope="module")
def three_level():
    """8^4 fine lattice, 2^4 aggregates on both levels: level 1 is 4^4 x 8 dofs, level 2 is 2^4 x 8."""
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.3, seed=0).numpy()
    op = FineOperator(U, 0.125, 1.0)
    mu = 0.01
    p = mg.Params(nlevels=3, n_setup=2, nv=[4, 4], bdims=[B2, B2], post_smooth=2, nmr=3)
    cl = blocks.coarse_lat(op.lat, B2)
    tv0 = [synth.gaussian_vectors((4,) + op.lat + op.dof, seed=31).numpy(),
           synth.gaussian_vectors((4,) + cl + (8,), seed=32).numpy()]
    h = mg.setup(op, p, mu, tv0)
    return op, h, mu


@pytest.mark.slow
def test_three_level_galerkin_is_dense_product(three_level):
    """The level-2 operator equals P_1^dagger D_1 P_1 (+ i delta mu Gamma5 on the coarsest level),
    with D_1 itself a Galerkin operator: the recursion of Sec. 2.3 applied twice."""
    op, h, mu = three_level
    D1, D2 = h.ops[1], h.ops[2]
    W1 = h.W[1]
    mu2 = h.mu_at(2, mu)
    D1m = dense(lambda v: D1.apply(v, mu2), D1.lat + D1.dof)
    n1, n2 = int(np.prod(D1.lat + D1.dof)), int(np.prod(D2.lat + D2.dof))
    Pm = np.zeros((n1, n2), dtype=complex)
    for k in range(n2):
        e = np.zeros(n2, dtype=complex)
        e[k] = 1
        Pm[:, k] = aggregation.prolong(W1, e.reshape(D2.lat + D2.dof), D1.lat, B2).ravel()
    assert np.allclose(Pm.conj().T @ Pm, np.eye(n2), atol=1e-12)
    want = Pm.conj().T @ D1m @ Pm
    got = dense(lambda v: D2.apply(v, mu2), D2.lat + D2.dof)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


@pytest.mark.slow
def test_three_level_solve(three_level):
    """Outer FGMRES with the K-cycle (FGMRES(5) on level 1, even-odd GMRES on level 2) reaches
    the FP64 relative residual 1e-10 for +mu and -mu with one setup."""
    op, h, mu = three_level
    b = synth.gaussian_spinor((8, 8, 8, 8), seed=1).numpy()
    for m in (mu, -mu):
        x, info = mg.solve(h, b, m)
        assert info['converged']
        assert dirac.norm(b - op.apply(x, m)) <= 1e-10 * dirac.norm(b)


def test_eo_cg_adjoint_and_dense_solution(fine, fine_dense):
    """Even-odd CG baseline (Sec. 3.1.2): the operator it squares is applied with its true
    adjoint (<u, D_hat v> = <D_hat^dagger u, v> for random u, v on the odd sites), and the
    solution agrees with the dense LU solve of D(mu) x = b."""
    Dm, mu = fine_dense
    b = synth.gaussian_spinor(DIMS4, seed=7).numpy()
    x, info = krylov.eo_cg(fine, b, mu, tol=1e-13)
    assert info["converged"] and info["iters"] > 0
    xs = np.linalg.solve(Dm, b.ravel())
    assert np.linalg.norm(x.ravel() - xs) <= 1e-8 * np.linalg.norm(xs)
    # adjointness of the two pieces the solver uses, through its own operator object
    par = (np.indices(fine.lat).sum(axis=0) % 2).reshape(fine.lat + (1, 1))
    odd = par == 1
    even = ~odd
    u = synth.gaussian_spinor(DIMS4, seed=8).numpy() * odd
    v = synth.gaussian_spinor(DIMS4, seed=9).numpy() * odd

    def d_hat(w, m):
        t = fine.site_inv(even * fine.hop(w * odd), m) * even
        return odd * fine.site(w * odd, m) - odd * fine.hop(t)

    lhs = np.vdot(u, d_hat(v, mu))
    rhs = np.vdot(fine.gamma5(d_hat(fine.gamma5(u), -mu)), v)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # the recursively updated residual of the squared system fell to the requested 1e-13
    r = np.array(info["residuals"])
    assert np.all(np.isfinite(r)) and r[-1] <= 1e-13 * r[0]
