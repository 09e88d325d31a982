"""Coarse stencil on tensor cores (FP16 operand images, FP32 accumulation)
against the oracle's coarse operator D_c (Sec. 2.3), inside the even-odd
coarsest solve (Sec. 2.5) and inside the full two-level solve.

Tolerance.  Each product rounds the operator blocks and the vectors to FP16
(unit roundoff 2^-11 = 4.9e-4) and sums in FP32, so the relative 2-norm error
of D_c x is a few 1e-4; the tests allow 2e-3.  A wrong index, layout or
real/imaginary combination gives errors of order one.

Shapes covered: n = 2 nv = 12 (K padded from 12 to 16), 16, 48 (the propagator
workload's 48 x 48 blocks); R = 1 (N padded to 16), 3 (a partial 8-column
group), 12 and 40 (two column chunks of at most 32 right-hand sides).
"""

import numpy as np
import pytest
import torch

from oracle import aggregation, coarse as ocoarse
from oracle.operators import FineOperator
from paper_1610_02370_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1610_02370_gb300 import build
    build.build()
    from paper_1610_02370_gb300 import ddtm
    return ddtm


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


class Case:
    def __init__(self, ddtm, dims, block, nv, coarse_prec, eps=0.3, kappa=0.13, csw=1.2, seed=0):
        self.dims, self.block, self.nv = dims, block, nv
        self.U = synth.gauge_field(dims, eps, seed=seed)
        self.op = FineOperator(self.U.numpy(), kappa, csw, 0)
        self.v = synth.gaussian_vectors((nv,) + self.op.lat + (4, 3), seed=seed + 50)
        self.ctx = ddtm.ddtm_create(dims, block, 0)
        ddtm.ddtm_load_gauge(self.ctx, self.U.cuda(), kappa, csw)
        p = ddtm.ddtm_get_params(self.ctx)
        p.nv[0] = nv
        p.coarse_prec = coarse_prec
        ddtm.ddtm_set_params(self.ctx, p)
        ddtm.ddtm_set_test_vectors(self.ctx, 0, self.v.cuda(), nv)
        self.W = aggregation.build_P(self.op, self.v.numpy(), block)
        self.cop = ocoarse.build_coarse_operator(self.op, self.W, block)


@pytest.fixture(scope="module", params=[(6, (16, 8, 16, 8)), (8, (16, 8, 16, 8)), (24, (16, 8, 8, 8))],
                ids=["nv6", "nv8", "nv24"])
def tc_case(lib, request):
    nv, dims = request.param
    c = Case(lib, dims, (4, 4, 4, 4), nv, lib.PREC_F16)
    yield c
    lib.ddtm_destroy(c.ctx)


@pytest.mark.parametrize("nrhs", [1, 3, 12, 40])
def test_tc_apply_matches_oracle(lib, tc_case, nrhs):
    c = tc_case
    cl = c.cop.lat
    mu = 0.05
    x = synth.gaussian_vectors((nrhs,) + cl + (2 * c.nv,), seed=7 + nrhs)
    y = torch.zeros_like(x).cuda()
    lib.ddtm_apply_Dc(c.ctx, 1, y, x.cuda(), nrhs, mu)
    y = y.cpu().numpy()
    for r in range(nrhs):
        want = c.cop.apply(x[r].numpy(), mu)
        assert relerr(y[r], want) < 2e-3, (r, relerr(y[r], want))


def test_tc_apply_sign_of_twist(lib, tc_case):
    """+mu and -mu against the same images: the difference is 2 i mu Gamma5_c x."""
    c = tc_case
    cl = c.cop.lat
    x = synth.gaussian_vectors((4,) + cl + (2 * c.nv,), seed=11)
    yp = torch.zeros_like(x).cuda()
    ym = torch.zeros_like(x).cuda()
    lib.ddtm_apply_Dc(c.ctx, 1, yp, x.cuda(), 4, 0.5)
    lib.ddtm_apply_Dc(c.ctx, 1, ym, x.cuda(), 4, -0.5)
    g5 = np.concatenate([np.ones(c.nv), -np.ones(c.nv)])
    want = 2j * 0.5 * g5 * x.numpy()
    # the twist is added in FP32 from the FP32 vector: only the FP16 product differs
    got = (yp - ym).cpu().numpy()
    assert relerr(got, want) < 1e-5


@pytest.fixture(scope="module")
def eo_case(lib):
    c = Case(lib, (8, 8, 8, 8), (4, 4, 4, 4), 8, lib.PREC_F16, seed=3)
    yield c
    lib.ddtm_destroy(c.ctx)


def test_tc_coarse_eo_solve(lib, eo_case):
    """Even-odd coarsest GMRES with the tensor-core Schur complement: the true
    residual with the oracle's FP64 D_c falls to the FP16 operator accuracy, and
    the even rows, rebuilt with the FP32 inverse, vanish to FP32 accuracy."""
    c = eo_case
    cl = c.cop.lat
    muc = 0.5
    b = synth.gaussian_vectors(cl + (2 * c.nv,), seed=6)
    p = lib.ddtm_get_params(c.ctx)
    p.coarse_tol = 1e-5
    p.coarse_restart = 60
    lib.ddtm_set_params(c.ctx, p)
    lib.ddtm_set_test_vectors(c.ctx, 0, c.v.cuda(), c.nv)
    x = torch.zeros_like(b).cuda()
    it, code = lib.ddtm_coarse_solve(c.ctx, x, b.cuda(), muc)
    assert code == lib.OK and it > 0
    xh = x.cpu().numpy()
    r = b.numpy() - c.cop.apply(xh, muc)
    assert np.linalg.norm(r) < 3e-3 * np.linalg.norm(b.numpy())
    par = np.indices(cl).sum(axis=0) % 2
    assert np.linalg.norm(r[par == 0]) < 1e-4 * np.linalg.norm(b.numpy())


@pytest.mark.parametrize("nrhs", [5, 12])
def test_tc_coarse_eo_solve_batch(lib, eo_case, nrhs):
    """The batched coarsest solve (5 right-hand sides padded to 8, and 12):
    every rhs reaches the FP16 operator accuracy against the oracle's D_c."""
    c = eo_case
    cl = c.cop.lat
    muc = 0.5
    b = synth.gaussian_vectors((nrhs,) + cl + (2 * c.nv,), seed=16)
    p = lib.ddtm_get_params(c.ctx)
    p.coarse_tol = 1e-5
    p.coarse_restart = 60
    lib.ddtm_set_params(c.ctx, p)
    lib.ddtm_set_test_vectors(c.ctx, 0, c.v.cuda(), c.nv)
    x = torch.zeros_like(b).cuda()
    it, code = lib.ddtm_coarse_solve_batch(c.ctx, x, b.cuda(), nrhs, muc)
    assert code == lib.OK and it > 0
    xh = x.cpu().numpy()
    for r in range(nrhs):
        res = b[r].numpy() - c.cop.apply(xh[r], muc)
        assert np.linalg.norm(res) < 3e-3 * np.linalg.norm(b[r].numpy()), r


def test_tc_two_level_solve_12rhs(lib):
    """12 right-hand sides through the two-level solve with the tensor-core coarse
    stencil: every system reaches FP64 relative residual 1e-10 (oracle's D), in
    about as many outer iterations as with the FP32 coarse stencil."""
    dims, block, nv, mu = (16, 8, 8, 8), (4, 4, 4, 4), 24, 0.003
    U = synth.gauge_field(dims, 0.2, seed=0)
    op = FineOperator(U.numpy(), 0.1340, 1.5755, 1)
    b = synth.gaussian_spinor(dims, seed=1, nrhs=12)
    iters = {}
    for prec in (lib.PREC_F32, lib.PREC_F16):
        ctx = lib.ddtm_create(dims, block, 1)
        try:
            lib.ddtm_load_gauge(ctx, U.cuda(), 0.1340, 1.5755)
            p = lib.ddtm_get_params(ctx)
            p.nv[0] = nv
            p.n_setup = 3
            p.post_smooth = 2
            p.coarse_prec = prec
            lib.ddtm_set_params(ctx, p)
            lib.ddtm_setup(ctx, mu, 99)
            x = torch.zeros_like(b).cuda()
            info, code = lib.ddtm_solve(ctx, x, b.cuda(), 12, mu)
            assert code == lib.OK, lib.ddtm_last_error(ctx)
            xh = x.cpu().numpy()
            for r in range(12):
                rel = np.linalg.norm(b[r].numpy() - op.apply(xh[r], mu)) / np.linalg.norm(b[r].numpy())
                assert rel <= 1e-10, (prec, r, rel)
            iters[prec] = info.iters
        finally:
            lib.ddtm_destroy(ctx)
    print("outer iterations F32 / F16 coarse:", iters)
    assert iters[lib.PREC_F16] <= iters[lib.PREC_F32] + 3


def test_tc_forced_timeout_reports_status(lib, eo_case):
    """Failure path of the bounded pipeline waits of the tensor-core stencil.
    With the test hook on, the MMA thread of every pass first waits on a barrier
    that nothing completes; the wait runs out after 2 ms, the pass stops (its
    bulk copies awaited, tensor memory freed) and the call reports
    DDTM_ERR_TIMEOUT.  The context stays usable: with the hook off, the same
    call gives the same bits as before the timeout, and matches the oracle."""
    c = eo_case
    cl = c.cop.lat
    nrhs, mu = 12, 0.05
    x = synth.gaussian_vectors((nrhs,) + cl + (2 * c.nv,), seed=21).cuda()
    y0 = torch.zeros_like(x)
    lib.ddtm_apply_Dc(c.ctx, 1, y0, x, nrhs, mu)
    lib.ddtm_set_option(c.ctx, "tc_forced_timeout_us", 2000)
    try:
        assert lib.ddtm_get_option(c.ctx, "tc_forced_timeout_us") == 2000
        y1 = torch.zeros_like(x)
        with pytest.raises(lib.DDTMError) as e:
            lib.ddtm_apply_Dc(c.ctx, 1, y1, x, nrhs, mu)
        assert e.value.code == lib.ERR_TIMEOUT, str(e.value)
    finally:
        lib.ddtm_set_option(c.ctx, "tc_forced_timeout_us", 0)
    assert lib.ddtm_get_option(c.ctx, "tc_forced_timeout_us") == 0
    y2 = torch.zeros_like(x)
    lib.ddtm_apply_Dc(c.ctx, 1, y2, x, nrhs, mu)
    assert torch.equal(y0, y2)
    y2 = y2.cpu().numpy()
    for r in range(nrhs):
        want = c.cop.apply(x[r].cpu().numpy(), mu)
        assert relerr(y2[r], want) < 2e-3, (r, relerr(y2[r], want))
    for bad in (-1, 1000001):
        with pytest.raises(lib.DDTMError):
            lib.ddtm_set_option(c.ctx, "tc_forced_timeout_us", bad)
