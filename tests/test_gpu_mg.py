"""GPU parity of aggregation, the Galerkin coarse operator, the coarsest even-odd
GMRES and the full two-level solve (Sec. 2.2 - 2.6) against the CPU oracle.

* P: both sides orthonormalise each aggregate half by MGS in index order, which
  gives the unique QR factor with positive diagonal, so entries are compared
  (FP32 storage; the GPU starts from FP32-rounded test vectors).
* R, P and D_c applications: relative 2-norm against the oracle with the same
  test vectors.  D_c is summed over 6 V_b terms per entry in FP32, so its
  tolerance is 1e-5 (FP32 storage) and 2e-3 (FP16 storage).
* Solves: final FP64 relative residual <= 1e-10, measured with the oracle's D,
  and the solution within 1e-8 of a dense LU solve where the lattice is small.
"""

import numpy as np
import pytest
import torch

from oracle import aggregation, blocks, coarse as ocoarse, krylov
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


def make_ctx(ddtm, dims, block, U, kappa, csw, nv, bc_t=0, **kw):
    ctx = ddtm.ddtm_create(dims, block, bc_t)
    ddtm.ddtm_load_gauge(ctx, U.cuda(), kappa, csw)
    p = ddtm.ddtm_get_params(ctx)
    p.nv[0] = nv
    for k, v in kw.items():
        setattr(p, k, v)
    ddtm.ddtm_set_params(ctx, p)
    return ctx


class Case:
    def __init__(self, ddtm, dims, block, eps, kappa, csw, nv, coarse_prec, seed=0, bc_t=0):
        self.dims, self.block, self.nv = dims, block, nv
        self.U = synth.gauge_field(dims, eps, seed=seed)
        self.op = FineOperator(self.U.numpy(), kappa, csw, bc_t)
        lat = self.op.lat
        self.v = synth.gaussian_vectors((nv,) + lat + (4, 3), seed=seed + 50)
        self.ctx = make_ctx(ddtm, dims, block, self.U, kappa, csw, nv, bc_t, coarse_prec=coarse_prec)
        ddtm.ddtm_set_test_vectors(self.ctx, 0, self.v.cuda(), nv)
        self.W = aggregation.build_P(self.op, self.v.numpy(), block)
        self.cop = ocoarse.build_coarse_operator(self.op, self.W, block)


@pytest.fixture(scope="module")
def case8(lib):
    c = Case(lib, (8, 8, 8, 8), (4, 4, 4, 4), 0.3, 0.13, 1.2, 6, lib.PREC_F32)
    yield c
    lib.ddtm_destroy(c.ctx)


def test_prolongator_matches_oracle(lib, case8):
    c = case8
    W = torch.zeros((2, c.nv) + c.op.lat + (4, 3), dtype=torch.complex128, device="cuda")
    lib.ddtm_get_prolongator(c.ctx, 0, W)
    assert relerr(W.cpu().numpy(), c.W) < 2e-6


def test_restrict_prolong_match_oracle(lib, case8):
    c = case8
    psi = synth.gaussian_spinor(c.dims, seed=3)
    cl = c.cop.lat
    cv = torch.zeros(cl + (2 * c.nv,), dtype=torch.complex128, device="cuda")
    lib.ddtm_restrict(c.ctx, 0, cv, psi.cuda(), 1)
    want = aggregation.restrict(c.W, psi.numpy(), c.op.lat, c.block)
    assert relerr(cv.cpu().numpy(), want) < 2e-6
    e = synth.gaussian_vectors(cl + (2 * c.nv,), seed=4)
    f = torch.zeros_like(psi).cuda()
    lib.ddtm_prolong(c.ctx, 0, f, e.cuda(), 1)
    want = aggregation.prolong(c.W, e.numpy(), c.op.lat, c.block)
    assert relerr(f.cpu().numpy(), want) < 2e-6


@pytest.fixture(scope="module")
def case24t(lib):
    c = Case(lib, (16, 8, 8, 8), (4, 4, 4, 4), 0.3, 0.13, 1.2, 24, lib.PREC_F32, seed=7)
    yield c
    lib.ddtm_destroy(c.ctx)


@pytest.mark.parametrize("nrhs", [5, 12, 13])
def test_restrict_prolong_batched(lib, case24t, nrhs):
    """Batches of right-hand sides through one restriction / prolongation launch
    (P read once per 6 right-hand sides; 13 = a batch of 12 and a batch of 1):
    each rhs equals, bit for bit, the same rhs transferred alone (same sums in
    the same order), and matches the oracle's R = P^dagger and P (Sec. 2.3)."""
    c = case24t
    cl = c.cop.lat
    psi = synth.gaussian_spinor(c.dims, seed=21, nrhs=nrhs)
    cv = torch.zeros((nrhs,) + cl + (2 * c.nv,), dtype=torch.complex128, device="cuda")
    lib.ddtm_restrict(c.ctx, 0, cv, psi.cuda(), nrhs)
    e = synth.gaussian_vectors((nrhs,) + cl + (2 * c.nv,), seed=22)
    f = torch.zeros_like(psi).cuda()
    lib.ddtm_prolong(c.ctx, 0, f, e.cuda(), nrhs)
    for r in range(nrhs):
        c1 = torch.zeros_like(cv[r:r + 1])
        lib.ddtm_restrict(c.ctx, 0, c1, psi[r:r + 1].contiguous().cuda(), 1)
        assert torch.equal(cv[r:r + 1], c1), r
        f1 = torch.zeros_like(f[r:r + 1])
        lib.ddtm_prolong(c.ctx, 0, f1, e[r:r + 1].contiguous().cuda(), 1)
        assert torch.equal(f[r:r + 1], f1), r
    for r in (0, nrhs - 1):
        want = aggregation.restrict(c.W, psi[r].numpy(), c.op.lat, c.block)
        assert relerr(cv[r].cpu().numpy(), want) < 2e-6
        want = aggregation.prolong(c.W, e[r].numpy(), c.op.lat, c.block)
        assert relerr(f[r].cpu().numpy(), want) < 2e-6


@pytest.mark.parametrize("mu", [0.01, -0.25])
def test_coarse_operator_matches_oracle(lib, case8, mu):
    c = case8
    cl = c.cop.lat
    x = synth.gaussian_vectors((2,) + cl + (2 * c.nv,), seed=5)
    y = torch.zeros_like(x).cuda()
    lib.ddtm_apply_Dc(c.ctx, 1, y, x.cuda(), 2, mu)
    for r in range(2):
        want = c.cop.apply(x[r].numpy(), mu)
        assert relerr(y[r].cpu().numpy(), want) < 1e-5


def test_coarse_operator_fp16_storage(lib):
    c = Case(lib, (8, 8, 8, 8), (4, 4, 4, 4), 0.3, 0.13, 1.2, 6, lib.PREC_F16, seed=2, bc_t=1)
    try:
        cl = c.cop.lat
        x = synth.gaussian_vectors(cl + (2 * c.nv,), seed=5)
        y = torch.zeros_like(x).cuda()
        lib.ddtm_apply_Dc(c.ctx, 1, y, x.cuda(), 1, 0.05)
        assert relerr(y.cpu().numpy(), c.cop.apply(x.numpy(), 0.05)) < 2e-3
    finally:
        lib.ddtm_destroy(c.ctx)


def test_coarse_eo_solve(lib, case8):
    """Tight tolerance: matches the dense solution of the oracle's D_c.  Loose
    tolerance: the retrieval of phi_e makes the even rows of the residual vanish."""
    c = case8
    cl = c.cop.lat
    b = synth.gaussian_vectors(cl + (2 * c.nv,), seed=6)
    muc = 0.5  # well conditioned, so FP32 operator rounding stays below the checks
    n = int(np.prod(cl)) * 2 * c.nv
    Dc = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1
        Dc[:, k] = c.cop.apply(e.reshape(cl + (2 * c.nv,)), muc).ravel()
    p = lib.ddtm_get_params(c.ctx)
    p.coarse_tol = 1e-5
    p.coarse_restart = 60
    lib.ddtm_set_params(c.ctx, p)
    lib.ddtm_set_test_vectors(c.ctx, 0, c.v.cuda(), c.nv)
    x = torch.zeros_like(b).cuda()
    it, code = lib.ddtm_coarse_solve(c.ctx, x, b.cuda(), muc)
    assert code == lib.OK and it > 0
    want = np.linalg.solve(Dc, b.numpy().ravel())
    assert relerr(x.cpu().numpy().ravel(), want) < 1e-4
    p.coarse_tol = 1e-1
    lib.ddtm_set_params(c.ctx, p)
    lib.ddtm_set_test_vectors(c.ctx, 0, c.v.cuda(), c.nv)
    it, code = lib.ddtm_coarse_solve(c.ctx, x, b.cuda(), muc)
    r = (b.numpy().ravel() - Dc @ x.cpu().numpy().ravel()).reshape(b.shape)
    par = np.indices(cl).sum(axis=0) % 2
    assert np.linalg.norm(r[par == 0]) < 1e-4 * np.linalg.norm(b.numpy())
    assert np.linalg.norm(r) <= 0.1 * np.linalg.norm(b.numpy()) * 1.01


def solve_case(lib, dims, block, eps, kappa, csw, mu, nv, n_setup, dense_check, bc_t=0, **kw):
    U = synth.gauge_field(dims, eps, seed=0)
    op = FineOperator(U.numpy(), kappa, csw, bc_t)
    ctx = make_ctx(lib, dims, block, U, kappa, csw, nv, bc_t, n_setup=n_setup, **kw)
    try:
        lib.ddtm_setup(ctx, mu, 1234)
        b = synth.gaussian_spinor(dims, seed=1)
        out = []
        for m in (mu, -mu):
            x = torch.zeros_like(b).cuda()
            info, code = lib.ddtm_solve(ctx, x, b.cuda(), 1, m)
            assert code == lib.OK, lib.ddtm_last_error(ctx)
            xh = x.cpu().numpy()
            r = b.numpy() - op.apply(xh, m)
            rel = np.linalg.norm(r) / np.linalg.norm(b.numpy())
            assert rel <= 1e-10, rel
            assert info.max_relres <= 1e-10
            if dense_check:
                n = int(np.prod(op.lat)) * 12
                D = np.zeros((n, n), dtype=complex)
                for k in range(n):
                    e = np.zeros(n, dtype=complex)
                    e[k] = 1
                    D[:, k] = op.apply(e.reshape(op.lat + (4, 3)), m).ravel()
                xs = np.linalg.solve(D, b.numpy().ravel())
                assert relerr(xh.ravel(), xs) <= 1e-8
            out.append((info.iters, info.coarse_iters, rel))
        return out
    finally:
        lib.ddtm_destroy(ctx)


def test_solve_4x4x4x4(lib):
    """4^4 lattice (eps 0.3, kappa 0.125, c_sw 1.0, mu 0.01), 2^4 aggregates: residual 1e-10
    and the dense LU solution within 1e-8, for +mu and -mu with one setup."""
    res = solve_case(lib, (4, 4, 4, 4), (2, 2, 2, 2), 0.3, 0.125, 1.0, 0.01, 8, 3, True, post_smooth=2, nmr=3)
    print("4^4 solves (iters, coarse iters, relres):", res)


def test_solve_16x16x16x32_fp16_smoother(lib):
    res = solve_case(lib, (32, 16, 16, 16), (4, 4, 4, 4), 0.2, 0.1340, 1.5755, 0.003, 12, 3, False, bc_t=1,
                     post_smooth=3, nmr=4)
    print("16^3x32 solves (iters, coarse iters, relres):", res)


def test_solve_fp64_fine_level(lib):
    """The plain FP64 method (FP64 outer FGMRES cycle and SAP smoother, FP32
    coarse correction): FP64 relative residual 1e-10 for +mu and -mu."""
    res = solve_case(lib, (16, 8, 8, 8), (4, 4, 4, 4), 0.2, 0.134, 1.5755, 0.01, 8, 2, False,
                     smoother_prec=lib.PREC_F64, post_smooth=2, coarse_prec=lib.PREC_F32)
    print("FP64 fine-level solves (iters, coarse iters, relres):", res)


def test_setup_invariants_and_save_load(lib, tmp_path):
    dims, block = (8, 8, 8, 16), (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.2, seed=3)
    op = FineOperator(U.numpy(), 0.134, 1.5755)
    nv = 8
    ctx = make_ctx(lib, dims, block, U, 0.134, 1.5755, nv, n_setup=2)
    ctx2 = make_ctx(lib, dims, block, U, 0.134, 1.5755, nv, n_setup=2)
    try:
        lib.ddtm_setup(ctx, 0.01, 7)
        W = torch.zeros((2, nv) + op.lat + (4, 3), dtype=torch.complex128, device="cuda")
        lib.ddtm_get_prolongator(ctx, 0, W)
        W = W.cpu().numpy()
        for s in range(2):
            for i in range(nv):
                for j in range(nv):
                    g = blocks.block_sum(np.conj(W[s, i]) * W[s, j], op.lat, block)
                    assert np.max(np.abs(g - (i == j))) < 1e-5
            other = W[s][..., 2 * (1 - s):2 * (1 - s) + 2, :]
            assert np.max(np.abs(other)) == 0
        path = str(tmp_path / "setup.bin")
        lib.ddtm_save_setup(ctx, path)
        lib.ddtm_load_setup(ctx2, path)
        b = synth.gaussian_spinor(dims, seed=2).cuda()
        x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
        lib.ddtm_solve(ctx, x1, b, 1, 0.01)
        lib.ddtm_solve(ctx2, x2, b, 1, 0.01)
        assert torch.equal(x1, x2)
        with pytest.raises(lib.DDTMError) as e:
            ctx3 = lib.ddtm_create(dims, block, 0)
            try:
                lib.ddtm_solve(ctx3, x1, b, 1, 0.01)
            finally:
                lib.ddtm_destroy(ctx3)
        assert e.value.code == lib.ERR_STATE
    finally:
        lib.ddtm_destroy(ctx)
        lib.ddtm_destroy(ctx2)


@pytest.fixture(scope="module")
def case24(lib):
    """8^4 lattice, 4^4 aggregates, N_v = 24 (n = 48 dofs per coarse site, the workload's coarse
    block size): FP32 and FP16 coarse storage from the same test vectors."""
    c32 = Case(lib, (8, 8, 8, 8), (4, 4, 4, 4), 0.3, 0.13, 1.2, 24, lib.PREC_F32, seed=4)
    c16 = Case(lib, (8, 8, 8, 8), (4, 4, 4, 4), 0.3, 0.13, 1.2, 24, lib.PREC_F16, seed=4)
    yield c32, c16
    lib.ddtm_destroy(c32.ctx)
    lib.ddtm_destroy(c16.ctx)


@pytest.mark.parametrize("nrhs", [11, 13, 44, 48])
@pytest.mark.parametrize("which", ["f32", "f16"])
def test_coarse_operator_ragged_batches_nv24(lib, case24, nrhs, which):
    """D_c (Sec. 2.3) on batches whose thread shape once exceeded a CTA (n = 48 with 11, 13, 44
    or 48 right-hand sides): every column against the oracle's Galerkin operator."""
    c = case24[0] if which == "f32" else case24[1]
    tol = 1e-5 if which == "f32" else 2e-3
    cl = c.cop.lat
    x = synth.gaussian_vectors((nrhs,) + cl + (2 * c.nv,), seed=40 + nrhs)
    y = torch.zeros_like(x).cuda()
    lib.ddtm_apply_Dc(c.ctx, 1, y, x.cuda(), nrhs, 0.02)
    y = y.cpu().numpy()
    for r in range(nrhs):
        want = c.cop.apply(x[r].numpy(), 0.02)
        assert relerr(y[r], want) < tol, (r, relerr(y[r], want))


def test_solve_fp32_coarse_many_rhs(lib):
    """A 44-rhs batch with the FP32 SIMT coarse stencil (the coarse batch of 44 right-hand sides
    goes through the even-odd coarse kernels in one launch): every solve to 1e-10."""
    dims, block, nv, mu = (8, 8, 8, 8), (4, 4, 4, 4), 24, 0.01
    U = synth.gauge_field(dims, 0.3, seed=0)
    op = FineOperator(U.numpy(), 0.13, 1.2)
    ctx = make_ctx(lib, dims, block, U, 0.13, 1.2, nv, n_setup=2, coarse_prec=lib.PREC_F32, post_smooth=2)
    try:
        lib.ddtm_setup(ctx, mu, 99)
        b = synth.gaussian_spinor(dims, seed=8, nrhs=44)
        x = torch.zeros_like(b).cuda()
        info, code = lib.ddtm_solve(ctx, x, b.cuda(), 44, mu)
        assert code == lib.OK, lib.ddtm_last_error(ctx)
        xh = x.cpu().numpy()
        for r in range(44):
            rel = np.linalg.norm(b[r].numpy() - op.apply(xh[r], mu)) / np.linalg.norm(b[r].numpy())
            assert rel <= 1e-10, (r, rel)
    finally:
        lib.ddtm_destroy(ctx)


def test_error_statuses_noconv_and_oom(lib):
    """DDTM_ERR_NOCONV: an outer iteration budget too small for 1e-10 stops the solve, which still fills
    the report with the achieved residual.  DDTM_ERR_OOM: a device-memory cap below what the setup
    needs fails that call (no cudaMalloc is attempted past the cap) and leaves the context usable."""
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, seed=0)
    ctx = make_ctx(lib, dims, block, U, 0.13, 1.2, 8, n_setup=2, post_smooth=2)
    try:
        lib.ddtm_setup(ctx, 0.01, 5)
        p = lib.ddtm_get_params(ctx)
        p.outer_max_iters = 2
        lib.ddtm_set_params(ctx, p)
        b = synth.gaussian_spinor(dims, seed=1).cuda()
        x = torch.zeros_like(b)
        info, code = lib.ddtm_solve(ctx, x, b, 1, 0.01)
        assert code == lib.ERR_NOCONV
        assert 0 < info.iters <= 2 and 1e-10 < info.max_relres < 1.0
        p.outer_max_iters = 1000
        lib.ddtm_set_params(ctx, p)
        info, code = lib.ddtm_solve(ctx, x, b, 1, 0.01)
        assert code == lib.OK
        used = lib.ddtm_memory_in_use()
        assert used > 0
        lib.ddtm_set_memory_limit(used + 4096)
        try:
            with pytest.raises(lib.DDTMError) as e:
                lib.ddtm_field_create(ctx, lib.PREC_F32, 1)  # one fine field: 8^4 x 12 x 8 bytes > 4 KB
            assert e.value.code == lib.ERR_OOM and "memory limit" in str(e.value)
            assert lib.ddtm_memory_in_use() == used
            # a 3-rhs solve under the cap goes in batches that fit in what the context already holds
            b3 = synth.gaussian_spinor(dims, seed=2, nrhs=3).cuda()
            x3 = torch.zeros_like(b3)
            info, code = lib.ddtm_solve(ctx, x3, b3, 3, 0.01)
            assert code == lib.OK and info.max_relres <= 1e-10
            assert lib.ddtm_memory_in_use() <= used + 4096
        finally:
            lib.ddtm_set_memory_limit(0)
        f = lib.ddtm_field_create(ctx, lib.PREC_F32, 1)
        lib.ddtm_field_destroy(f)
    finally:
        lib.ddtm_destroy(ctx)
