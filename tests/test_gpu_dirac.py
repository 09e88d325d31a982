"""GPU parity of the D(mu) stencil (Sec. 2.1) against the CPU oracle.

Tolerances (relative 2-norm per right-hand side): 1e-13 FP64, 2e-6 FP32 and
2e-3 FP16 storage with FP32 arithmetic.
"""

import numpy as np
import pytest
import torch

from oracle import dirac
from oracle.operators import FineOperator
from paper_1610_02370_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 2e-6, 2: 2e-3}


@pytest.fixture(scope="module")
def lib():
    from paper_1610_02370_gb300 import build
    build.build()
    from paper_1610_02370_gb300 import ddtm
    return ddtm


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def run_case(ddtm, dims, block, eps, kappa, csw, mu, bc_t, nrhs, precs, seed=0, device=True):
    U = synth.gauge_field(dims, eps, seed=seed)
    x = synth.gaussian_spinor(dims, seed=seed + 1, nrhs=nrhs)
    op = FineOperator(U.numpy(), kappa, csw, bc_t)
    ctx = ddtm.ddtm_create(dims, block, bc_t)
    try:
        ddtm.ddtm_load_gauge(ctx, U.cuda() if device else U.numpy(), kappa, csw)
        for m in (mu, -mu):
            ref = np.stack([op.apply(x[r].numpy(), m) for r in range(nrhs)])
            for prec in precs:
                if device:
                    y = torch.zeros_like(x).cuda()
                    ddtm.ddtm_apply_D(ctx, y, x.cuda(), nrhs, m, prec)
                    y = y.cpu().numpy()
                else:
                    y = np.zeros(x.shape, dtype=np.complex128)
                    ddtm.ddtm_apply_D(ctx, y, x.numpy(), nrhs, m, prec)
                for r in range(nrhs):
                    e = relerr(y[r], ref[r])
                    assert e < TOL[prec], (dims, prec, m, r, e)
    finally:
        ddtm.ddtm_destroy(ctx)


@pytest.mark.parametrize("bc_t", [0, 1])
def test_D_parity_4x4x4x4(lib, bc_t):
    """4^4 lattice (2^4 blocks), eps=0.3, kappa=0.125, c_sw=1.0, mu=0.01."""
    run_case(lib, (4, 4, 4, 4), (2, 2, 2, 2), 0.3, 0.125, 1.0, 0.01, bc_t, 2, (0, 1, 2))


def test_D_parity_anisotropic_host_buffers(lib):
    """All extents different, so an axis mix-up between layouts would show; host arrays."""
    run_case(lib, (8, 4, 12, 8), (2, 2, 2, 4), 0.5, 0.131, 1.3, -0.2, 1, 1, (0, 1, 2), device=False)


def test_D_parity_16x16x16x32(lib):
    """16^3 x 32, eps=0.2, kappa=0.1340, c_sw=1.5755, mu=0.003, 4^4 blocks."""
    run_case(lib, (32, 16, 16, 16), (4, 4, 4, 4), 0.2, 0.1340, 1.5755, 0.003, 0, 1, (0, 1, 2))


def test_D_free_field_plane_wave(lib):
    """U = 1: a plane wave maps to [M(p) + i sum gamma sin p + i mu gamma5] times itself."""
    ddtm = lib
    dims = (8, 4, 4, 8)
    kappa, mu = 0.13, 0.05
    m = 1 / (2 * kappa) - 4
    U = synth.unit_gauge(dims)
    ctx = ddtm.ddtm_create(dims, (2, 2, 2, 2), 0)
    try:
        ddtm.ddtm_load_gauge(ctx, U.cuda(), kappa, 1.5)
        T, X, Y, Z = dims
        t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing='ij')
        p = (2 * np.pi * 3 / T, 2 * np.pi / X, 2 * np.pi * 2 / Y, 2 * np.pi * 5 / Z)
        ph = np.exp(1j * (p[0] * t + p[1] * x + p[2] * y + p[3] * z))
        rng = np.random.default_rng(0)
        chi = rng.normal(size=4) + 1j * rng.normal(size=4)
        col = rng.normal(size=3) + 1j * rng.normal(size=3)
        psi = ph[..., None, None] * np.einsum('s,a->sa', chi, col)
        g, g5 = dirac.gamma_matrices()
        sym = (m + sum(1 - np.cos(q) for q in p)) * np.eye(4) + 1j * sum(g[a] * np.sin(p[a]) for a in range(4)) \
            + 1j * mu * g5
        want = ph[..., None, None] * np.einsum('s,a->sa', sym @ chi, col)
        out = torch.zeros(psi.shape, dtype=torch.complex128, device="cuda")
        ddtm.ddtm_apply_D(ctx, out, torch.from_numpy(psi).cuda(), 1, mu, ddtm.PREC_F64)
        assert np.max(np.abs(out.cpu().numpy() - want)) < 1e-13
    finally:
        ddtm.ddtm_destroy(ctx)


def test_D_field_api_matches_canonical_call(lib):
    ddtm = lib
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.3, seed=3).cuda()
    x = synth.gaussian_spinor(dims, seed=4, nrhs=2).cuda()
    ctx = ddtm.ddtm_create(dims, (4, 4, 4, 4), 0)
    try:
        ddtm.ddtm_load_gauge(ctx, U, 0.13, 1.2)
        for prec in (0, 1, 2):
            fx = ddtm.ddtm_field_create(ctx, prec, 2)
            fy = ddtm.ddtm_field_create(ctx, prec, 2)
            ddtm.ddtm_field_import(ctx, fx, x)
            ddtm.ddtm_apply_D_field(ctx, fy, fx, 0.02)
            y1 = torch.zeros_like(x)
            ddtm.ddtm_field_export(ctx, fy, y1)
            y2 = torch.zeros_like(x)
            ddtm.ddtm_apply_D(ctx, y2, x, 2, 0.02, prec)
            torch.cuda.synchronize()
            assert torch.equal(y1, y2)
            ddtm.ddtm_field_destroy(fx)
            ddtm.ddtm_field_destroy(fy)
    finally:
        ddtm.ddtm_destroy(ctx)


def test_errors_state_and_nan(lib):
    ddtm = lib
    dims = (4, 4, 4, 4)
    ctx = ddtm.ddtm_create(dims, (2, 2, 2, 2), 0)
    try:
        x = synth.gaussian_spinor(dims, seed=1).cuda()
        y = torch.zeros_like(x)
        with pytest.raises(ddtm.DDTMError) as e:
            ddtm.ddtm_apply_D(ctx, y, x, 1, 0.1, ddtm.PREC_F32)
        assert e.value.code == ddtm.ERR_STATE
        U = synth.gauge_field(dims, 0.3, seed=0)
        U[1, 2, 3, 0, 2, 1, 1] = float("nan")
        with pytest.raises(ddtm.DDTMError) as e:
            ddtm.ddtm_load_gauge(ctx, U.cuda(), 0.125, 1.0)
        assert e.value.code == ddtm.ERR_NAN
        with pytest.raises(ddtm.DDTMError) as e:
            ddtm.ddtm_apply_D(ctx, y, x, 1, 0.1, 7)
        assert e.value.code == ddtm.ERR_ARG
    finally:
        ddtm.ddtm_destroy(ctx)


@pytest.mark.parametrize("prec", [1, 2])
def test_D_block_kernel_12_rhs_one_launch(lib, prec):
    """The 4^4-block stencil with 12 right-hand sides in one launch (links and clover read once
    per block for all of them), antiperiodic t: every right-hand side against the oracle, and
    bit-equal to 12 single right-hand-side applications."""
    ddtm = lib
    dims, nrhs, mu = (16, 8, 8, 8), 12, 0.0015
    U = synth.gauge_field(dims, 0.12, seed=7)
    op = FineOperator(U.numpy(), 0.1372, 1.5755, 1)
    x = synth.gaussian_spinor(dims, seed=8, nrhs=nrhs)
    ctx = ddtm.ddtm_create(dims, (4, 4, 4, 4), 1)
    try:
        ddtm.ddtm_load_gauge(ctx, U.cuda(), 0.1372, 1.5755)
        fx = ddtm.ddtm_field_create(ctx, prec, nrhs)
        fy = ddtm.ddtm_field_create(ctx, prec, nrhs)
        ddtm.ddtm_field_import(ctx, fx, x.cuda())
        ddtm.ddtm_apply_D_field(ctx, fy, fx, mu)
        y = torch.zeros_like(x).cuda()
        ddtm.ddtm_field_export(ctx, fy, y)
        ddtm.ddtm_field_destroy(fx)
        ddtm.ddtm_field_destroy(fy)
        y1 = torch.zeros_like(x).cuda()
        for r in range(nrhs):
            ddtm.ddtm_apply_D(ctx, y1[r], x[r].cuda(), 1, mu, prec)
        torch.cuda.synchronize()
        assert torch.equal(y, y1)
        y = y.cpu().numpy()
        for r in range(nrhs):
            e = relerr(y[r], op.apply(x[r].numpy(), mu))
            assert e < TOL[prec], (prec, r, e)
    finally:
        ddtm.ddtm_destroy(ctx)
