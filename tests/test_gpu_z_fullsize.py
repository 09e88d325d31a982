"""Parity at the benchmark's full size (32^3 x 64, the propagator workload of bench.py), on outputs the
oracle can compute piece by piece (oracle/local.py): D(mu) at sampled sites, one SAP cycle at sampled
blocks, R, P and the Galerkin coarse operator at sampled aggregates; and properties that hold at any size:
Gamma5-hermiticity of D(mu) and of the coarse operator after the benchmark's setup, R P = I and
R Gamma5 = Gamma5_c R.  The file is named to run after the other GPU test files."""

import numpy as np
import pytest
import torch

from oracle import local
from paper_1610_02370_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = (64, 32, 32, 32)  # T, X, Y, Z
EPS, KAPPA, CSW, MU = 0.12, 0.1372, 1.5755, 0.0015


@pytest.fixture(scope="module")
def lib():
    from paper_1610_02370_gb300 import build
    build.build()
    from paper_1610_02370_gb300 import ddtm
    return ddtm


@pytest.fixture(scope="module")
def full(lib):
    U = synth.gauge_field(DIMS, EPS, seed=0)
    ctx = lib.ddtm_create(DIMS, (4, 4, 4, 4), 0)
    lib.ddtm_load_gauge(ctx, U.cuda(), KAPPA, CSW)
    yield lib, ctx, U
    lib.ddtm_destroy(ctx)


def sampled_sites():
    rng = np.random.default_rng(17)
    T, X, Y, Z = DIMS
    sites = [tuple(int(rng.integers(0, n)) for n in DIMS) for _ in range(56)]
    # the corners of the lattice: every hop of these wraps
    sites += [(t, x, y, z) for t in (0, T - 1) for x in (0, X - 1) for y in (0,) for z in (0, Z - 1)]
    return sites


def test_dirac_full_size_sampled_sites(full):
    lib, ctx, U = full
    x = synth.gaussian_spinor(DIMS, seed=1)
    sites = sampled_sites()
    want = local.apply_D_at_sites(U.numpy(), KAPPA, CSW, x.numpy(), MU, sites)
    idx = tuple(torch.tensor([s[k] for s in sites]) for k in (0, 3, 2, 1))  # (t, z, y, x) array order
    for prec, tol in ((lib.PREC_F64, 1e-13), (lib.PREC_F32, 2e-6), (lib.PREC_F16, 2e-3)):
        y = torch.zeros_like(x).cuda()
        lib.ddtm_apply_D(ctx, y, x.cuda(), 1, MU, prec)
        got = y.cpu()[idx].numpy()
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want)


def g5(v):
    w = v.clone()
    w[..., 2:, :] *= -1
    return w


def test_dirac_full_size_gamma5_hermiticity(full):
    lib, ctx, _ = full
    v = synth.gaussian_spinor(DIMS, seed=2).cuda()
    w = synth.gaussian_spinor(DIMS, seed=3).cuda()
    a = torch.zeros_like(v)
    lib.ddtm_apply_D(ctx, a, g5(v), 1, MU, lib.PREC_F64)
    lhs = torch.vdot(w.flatten(), g5(a).flatten())
    bb = torch.zeros_like(w)
    lib.ddtm_apply_D(ctx, bb, w, 1, -MU, lib.PREC_F64)
    rhs = torch.vdot(bb.flatten(), v.flatten())
    assert abs((lhs - rhs).item()) <= 1e-12 * abs(lhs.item())


@pytest.fixture(scope="module")
def bench_setup(full):
    """The benchmark's setup (Nv = 24, 4^4 aggregates, 6 iterations, FP16 tensor-core coarse operator)."""
    lib, ctx, U = full
    p = lib.ddtm_get_params(ctx)
    p.nv[0] = 24
    p.n_setup = 6
    p.post_smooth = 2
    p.coarse_prec = lib.PREC_F16
    lib.ddtm_set_params(ctx, p)
    lib.ddtm_setup(ctx, MU, 2024)
    return lib, ctx, U


def coarse_shape():
    return tuple(d // 4 for d in (DIMS[0], DIMS[3], DIMS[2], DIMS[1])) + (48,)  # (Tc, Zc, Yc, Xc, 2 Nv)


def test_coarse_operator_full_size_gamma5_hermiticity(bench_setup):
    """After the benchmark's setup: <u, D_c(mu) v> = <Gamma5_c D_c(-mu) Gamma5_c u, v> within the FP16
    storage accuracy."""
    lib, ctx, _ = bench_setup
    u = synth.gaussian_vectors(coarse_shape(), seed=4).cuda()
    v = synth.gaussian_vectors(coarse_shape(), seed=5).cuda()
    g5c = torch.cat([torch.ones(24), -torch.ones(24)]).to(torch.complex128).cuda()
    a = torch.zeros_like(v)
    lib.ddtm_apply_Dc(ctx, 1, a, v, 1, MU)
    lhs = torch.vdot(u.flatten(), a.flatten())
    bq = torch.zeros_like(u)
    lib.ddtm_apply_Dc(ctx, 1, bq, (g5c * u).contiguous(), 1, -MU)
    rhs = torch.vdot((g5c * bq).flatten(), v.flatten())
    scale = torch.linalg.norm(u) * torch.linalg.norm(a)
    assert abs((lhs - rhs).item()) <= 2e-3 * scale.item()


def test_sap_full_size_sampled_blocks(full):
    """One SAP cycle (Sec. 2.4; 3 MR steps per even-odd reduced 4^4 block, red then black) from x = 0 at
    the benchmark's full size, the smoother of the benchmark, against the block-local oracle at two red and
    two black blocks, the lattice's corner blocks among them (their neighbours wrap around), in FP64 /
    FP32 / FP16 storage within 1e-12 / 2e-6 / 2e-3."""
    lib, ctx, U = full
    B = (4, 4, 4, 4)
    b = synth.gaussian_spinor(DIMS, seed=6)
    bl = [(0, 0, 0, 0), (15, 7, 7, 7), (1, 0, 0, 0), (15, 7, 7, 6)]  # red, red, black, black
    assert [sum(c) % 2 for c in bl] == [0, 0, 1, 1]
    want = np.concatenate([local.sap_cycle_at_block(U.numpy(), KAPPA, CSW, b.numpy(), MU, B, c, 3) for c in bl])
    sites = [s for c in bl for s in local.block_sites(B, c)]
    idx = tuple(torch.tensor([s[k] for s in sites]) for k in (0, 3, 2, 1))  # (t, z, y, x) array order
    for prec, tol in ((lib.PREC_F64, 1e-12), (lib.PREC_F32, 2e-6), (lib.PREC_F16, 2e-3)):
        x = torch.zeros_like(b).cuda()
        lib.ddtm_sap(ctx, x, b.cuda(), 1, MU, 1, 3, prec)
        got = x.cpu()[idx].numpy()
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want), prec


def test_transfers_full_size_properties(bench_setup):
    """After the benchmark's setup, properties of the aggregation (Sec. 2.3) that hold at any size:
    R P = I (P has orthonormal columns per aggregate half) and R Gamma5 = Gamma5_c R (P keeps the spin
    chirality), in the FP32 arithmetic of the transfers."""
    lib, ctx, _ = bench_setup
    c = synth.gaussian_vectors(coarse_shape(), seed=7).cuda()
    x = torch.zeros(DIMS[0], DIMS[3], DIMS[2], DIMS[1], 4, 3, dtype=torch.complex128, device="cuda")
    lib.ddtm_prolong(ctx, 0, x, c, 1)
    c2 = torch.zeros_like(c)
    lib.ddtm_restrict(ctx, 0, c2, x, 1)
    assert (torch.linalg.norm(c2 - c) / torch.linalg.norm(c)).item() <= 1e-4
    f = synth.gaussian_spinor(DIMS, seed=8).cuda()
    a, b = torch.zeros_like(c), torch.zeros_like(c)
    lib.ddtm_restrict(ctx, 0, a, g5(f).contiguous(), 1)
    lib.ddtm_restrict(ctx, 0, b, f, 1)
    g5c = torch.cat([torch.ones(24), -torch.ones(24)]).to(torch.complex128).cuda()
    assert (torch.linalg.norm(a - g5c * b) / torch.linalg.norm(b)).item() <= 1e-6


def test_coarse_operator_full_size_sampled_sites(full):
    """The Galerkin coarse operator (Sec. 2.3) at full size, Nv = 24 seeded Gaussian test vectors on 4^4
    aggregates (the benchmark's aggregation, without setup iterations): the columns D_c(mu) e_(A, r), all
    48 of them, on A and its 8 neighbouring coarse sites, at a corner and an interior coarse site, against
    the aggregate-local oracle (oracle/local.py), with FP32 SIMT and FP16 tensor-core coarse storage
    within 1e-5 and 2e-3; and R f = P^dagger f, P c at those aggregates (FP32 P from CGS2 with 24
    vectors per aggregate half, 5e-6)."""
    lib, _, U = full
    B, nv = (4, 4, 4, 4), 24
    NB = (DIMS[0] // 4, DIMS[1] // 4, DIMS[2] // 4, DIMS[3] // 4)
    sampled = [(0, 0, 0, 0), (7, 3, 5, 2)]
    v = synth.gaussian_vectors((nv,) + (DIMS[0], DIMS[3], DIMS[2], DIMS[1], 4, 3), seed=9, device="cuda")
    need = set()
    for A in sampled:
        need.add(A)
        for d in range(4):
            for s in (1, -1):
                bc = list(A)
                bc[d] = (bc[d] + s) % NB[d]
                need.add(tuple(bc))
    vb = {bc: v[(slice(None),) + local.block_slices(B, bc)].cpu().numpy() for bc in need}
    want = {A: local.coarse_columns_at_block(U.numpy(), KAPPA, CSW, vb.__getitem__, MU, B, A) for A in sampled}
    cshape = (NB[0], NB[3], NB[2], NB[1], 2 * nv)
    for cprec, tol in ((lib.PREC_F32, 1e-5), (lib.PREC_F16, 2e-3)):
        ctx = lib.ddtm_create(DIMS, B, 0)
        try:
            lib.ddtm_load_gauge(ctx, U.cuda(), KAPPA, CSW)
            p = lib.ddtm_get_params(ctx)
            p.nv[0] = nv
            p.coarse_prec = cprec
            lib.ddtm_set_params(ctx, p)
            lib.ddtm_set_test_vectors(ctx, 0, v, nv)
            if cprec == lib.PREC_F32:  # R = P^dagger and P at the sampled aggregates (FP32 transfers)
                f = synth.gaussian_spinor(DIMS, seed=10)
                c = synth.gaussian_vectors(cshape, seed=11)
                rc = torch.zeros(cshape, dtype=torch.complex128, device="cuda")
                lib.ddtm_restrict(ctx, 0, rc, f.cuda(), 1)
                pf = torch.zeros_like(f).cuda()
                lib.ddtm_prolong(ctx, 0, pf, c.cuda(), 1)
                rc, pf = rc.cpu().numpy(), pf.cpu().numpy()
                for A in sampled:
                    PA = local.prolongator_at_block(vb[A], B, A)
                    fA = np.concatenate([f.numpy()[t, z, y, x].reshape(12) for (t, x, y, z) in
                                         local.block_sites(B, A)])
                    want_r = PA.conj().T @ fA
                    assert np.linalg.norm(rc[A[0], A[3], A[2], A[1]] - want_r) <= 5e-6 * np.linalg.norm(want_r)
                    want_p = PA @ c.numpy()[A[0], A[3], A[2], A[1]]
                    got_p = np.concatenate([pf[t, z, y, x].reshape(12) for (t, x, y, z) in local.block_sites(B, A)])
                    assert np.linalg.norm(got_p - want_p) <= 5e-6 * np.linalg.norm(want_p)
            for A in sampled:
                x = torch.zeros((2 * nv,) + cshape, dtype=torch.complex128, device="cuda")
                for r in range(2 * nv):
                    x[r, A[0], A[3], A[2], A[1], r] = 1
                y = torch.zeros_like(x)
                lib.ddtm_apply_Dc(ctx, 1, y, x, 2 * nv, MU)
                yh = y.cpu().numpy()
                for bc, M in want[A].items():
                    got = yh[:, bc[0], bc[3], bc[2], bc[1], :].T  # column r = rhs r
                    assert np.linalg.norm(got - M) <= tol * np.linalg.norm(M), (cprec, A, bc)
        finally:
            lib.ddtm_destroy(ctx)
    del v
    torch.cuda.empty_cache()


def test_sap_full_size_batched_12_rhs(full):
    """The SAP cycle in the benchmark's launch configuration: 12 right-hand sides in one batch (one CTA per
    block and right-hand side), FP16 storage, through the field API; the first and the last right-hand
    side at a red and a black corner block against the block-local oracle within 2e-3."""
    lib, ctx, U = full
    B, nrhs = (4, 4, 4, 4), 12
    b = synth.gaussian_spinor(DIMS, seed=12, nrhs=nrhs)
    fb = lib.ddtm_field_create(ctx, lib.PREC_F16, nrhs)
    fx = lib.ddtm_field_create(ctx, lib.PREC_F16, nrhs)
    try:
        lib.ddtm_field_import(ctx, fb, b.cuda())
        lib.ddtm_sap_field(ctx, fx, fb, MU, 1, 3)
        x = torch.zeros_like(b).cuda()
        lib.ddtm_field_export(ctx, fx, x)
        x = x.cpu().numpy()
    finally:
        lib.ddtm_field_destroy(fx)
        lib.ddtm_field_destroy(fb)
    for r in (0, nrhs - 1):
        for c in ((15, 7, 7, 7), (1, 0, 0, 0)):
            want = local.sap_cycle_at_block(U.numpy(), KAPPA, CSW, b[r].numpy(), MU, B, c, 3)
            got = np.array([x[r, t, z, y, xx] for (t, xx, y, z) in local.block_sites(B, c)])
            assert np.linalg.norm(got - want) <= 2e-3 * np.linalg.norm(want), (r, c)


def test_propagator_full_size_oracle_residual_and_deviation(bench_setup):
    """The benchmark's propagator at full size: the 12 point sources solved in one mixed-precision batch
    to 1e-10 (Sec. 2.5 outer FGMRES stopping rule), each residual evaluated with the oracle's FP64 D
    (whole lattice, per t-slab, oracle/slabs.py) <= 1e-10; then the same batch driven to 1e-12 against
    the plain FP64 method driven to 1e-12: solutions within 1e-8 (the bound kappa(D) (tol_a + tol_b)
    allows with sigma_min >= mu)."""
    from oracle import slabs
    lib, ctx, U = bench_setup
    b = synth.point_sources(DIMS, device="cuda")
    x = torch.zeros_like(b)
    info, code = lib.ddtm_solve(ctx, x, b, 12, MU)
    assert code == lib.OK, lib.ddtm_last_error(ctx)
    rr = slabs.relative_residuals(U.numpy(), KAPPA, CSW, b.cpu().numpy(), x.cpu().numpy(), MU, bc_t=0, slab=4,
                                  workers=16)
    assert max(rr) <= 1e-10, rr
    p = lib.ddtm_get_params(ctx)
    tol0 = p.outer_tol
    p.outer_tol = 1e-12
    lib.ddtm_set_params(ctx, p)
    try:
        xm = torch.zeros_like(b)
        info, code = lib.ddtm_solve(ctx, xm, b, 12, MU)
        assert code == lib.OK, lib.ddtm_last_error(ctx)
    finally:
        p.outer_tol = tol0
        lib.ddtm_set_params(ctx, p)
    c64 = lib.ddtm_create(DIMS, (4, 4, 4, 4), 0)
    try:
        lib.ddtm_load_gauge(c64, U.cuda(), KAPPA, CSW)
        q = lib.ddtm_get_params(c64)
        q.nv[0], q.n_setup, q.post_smooth, q.outer_tol = 24, 6, 2, 1e-12
        q.smoother_prec, q.coarse_prec = lib.PREC_F64, lib.PREC_F32
        lib.ddtm_set_params(c64, q)
        lib.ddtm_setup(c64, MU, 2024)
        x64 = torch.zeros_like(b)
        info, code = lib.ddtm_solve(c64, x64, b, 12, MU)
        assert code == lib.OK, lib.ddtm_last_error(c64)
    finally:
        lib.ddtm_destroy(c64)
    dev = [((xm[i] - x64[i]).norm() / x64[i].norm()).item() for i in range(12)]
    assert max(dev) <= 1e-8, dev
