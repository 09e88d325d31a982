"""GPU parity of the three-level hierarchy (Sec. 2.2 K-cycle, Sec. 2.3 recursion) against the CPU
oracle: the level-1 aggregation (P_1 from level-1 test vectors, R_1 = P_1^+), the level-2 Galerkin
operator D_2 = P_1^+ D_1 P_1, and the three-level solve (FGMRES(5) K-cycle on level 1 with the
level-1 SAP smoother, even-odd GMRES on level 2) to FP64 relative residual 1e-10 for +mu and -mu,
its solution against the two-level solution of the same system, and a setup round trip through a file.

The 8^4 lattice with 2^4 aggregates on both levels is the oracle's three-level case (level 1: 4^4
sites x 8 dofs, level 2: 2^4 sites x 8 dofs).  D_2 is summed in FP32 over 16 sites x 4 dofs of the
FP32 D_1, so its tolerance is the one of the level-1 operator (1e-5)."""

import numpy as np
import pytest
import torch

from oracle import aggregation, coarse as ocoarse
from oracle.operators import FineOperator
from paper_1610_02370_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS, B2, EPS, KAPPA, CSW, MU = (8, 8, 8, 8), (2, 2, 2, 2), 0.3, 0.125, 1.0, 0.01


@pytest.fixture(scope="module")
def lib():
    from paper_1610_02370_gb300 import build
    build.build()
    from paper_1610_02370_gb300 import ddtm
    return ddtm


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def three_level_ctx(lib, U, nv=(4, 4), coarse_prec=1, **kw):
    ctx = lib.ddtm_create(DIMS, B2, 0)
    lib.ddtm_load_gauge(ctx, U.cuda(), KAPPA, CSW)
    p = lib.ddtm_get_params(ctx)
    p.n_levels = 3
    p.nv[0], p.nv[1] = nv
    for m in range(4):
        p.block[1][m] = 2
    p.coarse_prec = coarse_prec
    for k, v in kw.items():
        setattr(p, k, v)
    lib.ddtm_set_params(ctx, p)
    return ctx


@pytest.fixture(scope="module")
def case(lib):
    U = synth.gauge_field(DIMS, EPS, seed=0)
    op = FineOperator(U.numpy(), KAPPA, CSW)
    v0 = synth.gaussian_vectors((4,) + op.lat + (4, 3), seed=31)
    W0 = aggregation.build_P(op, v0.numpy(), B2)
    cop1 = ocoarse.build_coarse_operator(op, W0, B2)
    v1 = synth.gaussian_vectors((4,) + cop1.lat + (8,), seed=32)
    W1 = aggregation.build_P(cop1, v1.numpy(), B2)
    cop2 = ocoarse.build_coarse_operator(cop1, W1, B2)
    ctx = three_level_ctx(lib, U)
    lib.ddtm_set_test_vectors(ctx, 0, v0.cuda(), 4)
    lib.ddtm_set_test_vectors(ctx, 1, v1.cuda(), 4)
    yield lib, ctx, op, cop1, W1, cop2
    lib.ddtm_destroy(ctx)


@pytest.mark.parametrize("mu", [0.01, -0.3])
def test_level2_operator_matches_oracle(case, mu):
    lib, ctx, op, cop1, W1, cop2 = case
    x = synth.gaussian_vectors((3,) + cop2.lat + (8,), seed=40)
    y = torch.zeros_like(x).cuda()
    lib.ddtm_apply_Dc(ctx, 2, y, x.cuda(), 3, mu)
    for r in range(3):
        assert relerr(y[r].cpu().numpy(), cop2.apply(x[r].numpy(), mu)) < 1e-5, r


def test_level1_transfers_match_oracle(case):
    lib, ctx, op, cop1, W1, cop2 = case
    v = synth.gaussian_vectors(cop1.lat + (8,), seed=41)
    c = torch.zeros(cop2.lat + (8,), dtype=torch.complex128, device="cuda")
    lib.ddtm_restrict(ctx, 1, c, v.cuda(), 1)
    assert relerr(c.cpu().numpy(), aggregation.restrict(W1, v.numpy(), cop1.lat, B2)) < 5e-6
    e = synth.gaussian_vectors(cop2.lat + (8,), seed=42)
    f = torch.zeros(cop1.lat + (8,), dtype=torch.complex128, device="cuda")
    lib.ddtm_prolong(ctx, 1, f, e.cuda(), 1)
    assert relerr(f.cpu().numpy(), aggregation.prolong(W1, e.numpy(), cop1.lat, B2)) < 5e-6


@pytest.mark.parametrize("coarse_prec", [1, 2])
def test_three_level_solve_both_twists(lib, coarse_prec, tmp_path):
    """GPU setup (2 iterations, level by level), then +mu and -mu solves to 1e-10 (the oracle's
    residual); the solution driven to 1e-12 agrees with the two-level solve driven to 1e-12 within 1e-8;
    a setup saved to a file and loaded into a fresh context gives the bit-identical solution."""
    U = synth.gauge_field(DIMS, EPS, seed=0)
    op = FineOperator(U.numpy(), KAPPA, CSW)
    b = synth.gaussian_spinor(DIMS, seed=1, nrhs=2)
    ctx = three_level_ctx(lib, U, coarse_prec=coarse_prec, n_setup=2, post_smooth=2, nmr=3)
    try:
        lib.ddtm_setup(ctx, MU, 77)
        for m in (MU, -MU):
            x = torch.zeros_like(b).cuda()
            info, code = lib.ddtm_solve(ctx, x, b.cuda(), 2, m)
            assert code == lib.OK, lib.ddtm_last_error(ctx)
            for r in range(2):
                res = np.linalg.norm(b[r].numpy() - op.apply(x[r].cpu().numpy(), m)) / np.linalg.norm(b[r].numpy())
                assert res <= 1e-10, (m, r, res)
        p = lib.ddtm_get_params(ctx)
        p.outer_tol = 1e-12
        lib.ddtm_set_params(ctx, p)
        x3 = torch.zeros_like(b).cuda()
        info, code = lib.ddtm_solve(ctx, x3, b.cuda(), 2, MU)
        assert code == lib.OK
        path = str(tmp_path / "setup3.bin")
        lib.ddtm_save_setup(ctx, path)
        c2 = three_level_ctx(lib, U, coarse_prec=coarse_prec, n_setup=2, post_smooth=2, nmr=3, outer_tol=1e-12)
        try:
            lib.ddtm_load_setup(c2, path)
            xl = torch.zeros_like(b).cuda()
            lib.ddtm_solve(c2, xl, b.cuda(), 2, MU)
            assert torch.equal(xl, x3)
        finally:
            lib.ddtm_destroy(c2)
    finally:
        lib.ddtm_destroy(ctx)
    two = lib.ddtm_create(DIMS, B2, 0)
    try:
        lib.ddtm_load_gauge(two, U.cuda(), KAPPA, CSW)
        q = lib.ddtm_get_params(two)
        q.nv[0], q.n_setup, q.post_smooth, q.outer_tol = 8, 2, 2, 1e-12
        lib.ddtm_set_params(two, q)
        lib.ddtm_setup(two, MU, 78)
        x2 = torch.zeros_like(b).cuda()
        info, code = lib.ddtm_solve(two, x2, b.cuda(), 2, MU)
        assert code == lib.OK
    finally:
        lib.ddtm_destroy(two)
    for r in range(2):
        assert relerr(x3[r].cpu().numpy(), x2[r].cpu().numpy()) <= 1e-8


def test_three_level_parameter_checks(lib):
    U = synth.gauge_field(DIMS, EPS, seed=0)
    ctx = lib.ddtm_create(DIMS, B2, 0)
    try:
        p = lib.ddtm_get_params(ctx)
        p.n_levels = 3
        for m in range(4):
            p.block[1][m] = 4  # 4^4 level-1 lattice: one level-1 block per direction, no red-black colouring
        with pytest.raises(lib.DDTMError) as e:
            lib.ddtm_set_params(ctx, p)
        assert e.value.code == lib.ERR_ARG
        p.n_levels = 4
        with pytest.raises(lib.DDTMError):
            lib.ddtm_set_params(ctx, p)
    finally:
        lib.ddtm_destroy(ctx)


def test_level1_sap_matches_oracle(case):
    """The level-1 smoother (SAP on D_1 with 2^4 blocks of level-1 sites, MR on the full block, red
    then black) against the oracle's SAP with full-block MR on the Galerkin operator D_1."""
    from oracle import sap
    lib, ctx, op, cop1, W1, cop2 = case
    b = synth.gaussian_vectors((2,) + cop1.lat + (8,), seed=43)
    x = torch.zeros_like(b).cuda()
    lib.ddtm_sap_coarse(ctx, 1, x, b.cuda(), 2, MU, 2, 3)
    for r in range(2):
        want = sap.sap(cop1, b[r].numpy(), MU, B2, 2, 3, eo=False)
        assert relerr(x[r].cpu().numpy(), want) < 1e-5, r
