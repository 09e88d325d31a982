"""Twisted boundary conditions psi(x + L_mu mu_hat) = exp(i theta_mu) psi(x) (a library feature of the
paper's appendix, used with the HMC of Sec. 3.2), applied by the library as phases on the boundary links:
D(mu) against the oracle's D with twisted hops (any order of setting the phases and loading the field,
both time boundary conditions, FP64 / FP32 / FP16 storage, the generic and the 4^4-block stencils), a
two-level solve with twisted boundaries to FP64 relative residual 1e-10, and the return to periodic."""

import numpy as np
import pytest
import torch

from oracle.operators import FineOperator
from paper_1610_02370_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 2e-6, 2: 2e-3}
THETA = (0.3, 1.1, -0.7, 2.0)  # t, x, y, z


@pytest.fixture(scope="module")
def lib():
    from paper_1610_02370_gb300 import build
    build.build()
    from paper_1610_02370_gb300 import ddtm
    return ddtm


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("dims,block,bc_t,phases_first",
                         [((8, 8, 8, 8), (4, 4, 4, 4), 0, True), ((8, 8, 8, 8), (4, 4, 4, 4), 1, False),
                          ((4, 4, 4, 8), (2, 2, 2, 2), 1, True)])
def test_twisted_D_matches_oracle(lib, dims, block, bc_t, phases_first):
    U = synth.gauge_field(dims, 0.3, seed=5)
    x = synth.gaussian_spinor(dims, seed=6)
    op = FineOperator(U.numpy(), 0.13, 1.4, bc_t, theta=THETA)
    ctx = lib.ddtm_create(dims, block, bc_t)
    try:
        if phases_first:
            lib.ddtm_set_boundary_phases(ctx, THETA)
            lib.ddtm_load_gauge(ctx, U.cuda(), 0.13, 1.4)
        else:
            lib.ddtm_load_gauge(ctx, U.cuda(), 0.13, 1.4)
            lib.ddtm_apply_D(ctx, torch.zeros_like(x).cuda(), x.cuda(), 1, 0.02, 1)  # builds an FP32 copy first
            lib.ddtm_set_boundary_phases(ctx, THETA)
        for mu in (0.02, -0.02):
            want = op.apply(x.numpy(), mu)
            for prec in (0, 1, 2):
                y = torch.zeros_like(x).cuda()
                lib.ddtm_apply_D(ctx, y, x.cuda(), 1, mu, prec)
                assert relerr(y.cpu().numpy(), want) < TOL[prec], (prec, mu)
        # back to periodic (antiperiodic t kept)
        lib.ddtm_set_boundary_phases(ctx, (0.0, 0.0, 0.0, 0.0))
        y = torch.zeros_like(x).cuda()
        lib.ddtm_apply_D(ctx, y, x.cuda(), 1, 0.02, 0)
        want = FineOperator(U.numpy(), 0.13, 1.4, bc_t).apply(x.numpy(), 0.02)
        assert relerr(y.cpu().numpy(), want) < 1e-13
    finally:
        lib.ddtm_destroy(ctx)


def test_twisted_two_level_solve(lib):
    dims, mu = (8, 8, 8, 8), 0.01
    U = synth.gauge_field(dims, 0.3, seed=7)
    op = FineOperator(U.numpy(), 0.13, 1.2, 0, theta=THETA)
    ctx = lib.ddtm_create(dims, (4, 4, 4, 4), 0)
    try:
        lib.ddtm_set_boundary_phases(ctx, THETA)
        lib.ddtm_load_gauge(ctx, U.cuda(), 0.13, 1.2)
        p = lib.ddtm_get_params(ctx)
        p.nv[0], p.n_setup, p.post_smooth, p.coarse_prec = 8, 3, 2, lib.PREC_F16
        lib.ddtm_set_params(ctx, p)
        lib.ddtm_setup(ctx, mu, 9)
        b = synth.gaussian_spinor(dims, seed=8, nrhs=2)
        x = torch.zeros_like(b).cuda()
        info, code = lib.ddtm_solve(ctx, x, b.cuda(), 2, mu)
        assert code == lib.OK, lib.ddtm_last_error(ctx)
        for r in range(2):
            res = np.linalg.norm(b[r].numpy() - op.apply(x[r].cpu().numpy(), mu)) / np.linalg.norm(b[r].numpy())
            assert res <= 1e-10, (r, res)
    finally:
        lib.ddtm_destroy(ctx)


def test_setup_update_after_gauge_and_twist_change(lib):
    """The HMC usage of Sec. 3.2: a setup made on one gauge field and twist is updated (test vectors
    kept, one inverse-iteration step) after the field moved by a small random SU(3) rotation and the twist
    changed; the updated hierarchy solves the new system to 1e-10 (the oracle's residual).  Before any
    setup the update is a call-order error."""
    dims = (8, 8, 8, 8)
    U1 = synth.gauge_field(dims, 0.3, seed=20)
    step = synth.random_hermitian_exp(tuple(d for d in (8, 8, 8, 8)) + (4,), 0.05, 21)
    U2 = torch.matmul(step, U1)
    op2 = FineOperator(U2.numpy(), 0.13, 1.2)
    ctx = lib.ddtm_create(dims, (4, 4, 4, 4), 0)
    try:
        lib.ddtm_load_gauge(ctx, U1.cuda(), 0.13, 1.2)
        with pytest.raises(lib.DDTMError) as e:
            lib.ddtm_setup_update(ctx, 0.01, 1)
        assert e.value.code == lib.ERR_STATE
        p = lib.ddtm_get_params(ctx)
        p.nv[0], p.n_setup, p.post_smooth = 8, 3, 2
        lib.ddtm_set_params(ctx, p)
        lib.ddtm_setup(ctx, 0.01, 22)
        lib.ddtm_load_gauge(ctx, U2.cuda(), 0.13, 1.2)
        b = synth.gaussian_spinor(dims, seed=23)
        x = torch.zeros_like(b).cuda()
        with pytest.raises(lib.DDTMError) as e:  # a new gauge field invalidates the hierarchy
            lib.ddtm_solve(ctx, x, b.cuda(), 1, 0.02)
        assert e.value.code == lib.ERR_STATE
        for n_iter in (0, 1):
            lib.ddtm_setup_update(ctx, 0.02, n_iter)
            x = torch.zeros_like(b).cuda()
            info, code = lib.ddtm_solve(ctx, x, b.cuda(), 1, 0.02)
            assert code == lib.OK, lib.ddtm_last_error(ctx)
            res = np.linalg.norm(b.numpy() - op2.apply(x.cpu().numpy(), 0.02)) / np.linalg.norm(b.numpy())
            assert res <= 1e-10, (n_iter, res)
    finally:
        lib.ddtm_destroy(ctx)
