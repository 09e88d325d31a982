"""GPU parity of the even-odd CG baseline (Sec. 3.1.2: CG on the normal equations of the even-odd
reduced operator) against the CPU oracle: the solution of D(mu) x = b within 1e-8 of a dense LU solve
on the 4^4 lattice of the plain-method workload, the true residual measured with the oracle's D on a
larger antiperiodic lattice for +mu and -mu, the CG iteration count against the oracle's even-odd CG
at the same stopping rule, and the non-convergence status."""

import numpy as np
import pytest
import torch

from oracle import krylov
from oracle.operators import FineOperator
from paper_1610_02370_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1610_02370_gb300 import build
    build.build()
    from paper_1610_02370_gb300 import ddtm
    return ddtm


def dense(op, mu):
    n = int(np.prod(op.lat)) * 12
    D = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1
        D[:, k] = op.apply(e.reshape(op.lat + (4, 3)), mu).ravel()
    return D


def test_eo_cg_matches_dense_solution_4x4x4x4(lib):
    dims, mu = (4, 4, 4, 4), 0.01
    U = synth.gauge_field(dims, 0.3, seed=0)
    op = FineOperator(U.numpy(), 0.125, 1.0)
    b = synth.gaussian_spinor(dims, seed=1)
    ctx = lib.ddtm_create(dims, (2, 2, 2, 2), 0)
    try:
        lib.ddtm_load_gauge(ctx, U.cuda(), 0.125, 1.0)
        x = torch.zeros_like(b).cuda()
        info, code = lib.ddtm_eo_cg(ctx, x, b.cuda(), 1, mu, tol=1e-12)
        assert code == lib.OK, lib.ddtm_last_error(ctx)
        xs = np.linalg.solve(dense(op, mu), b.numpy().ravel())
        xh = x.cpu().numpy()
        assert np.linalg.norm(xh.ravel() - xs) <= 1e-8 * np.linalg.norm(xs)
        r = b.numpy() - op.apply(xh, mu)
        assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b.numpy()) * 1.01
        assert abs(info.max_relres - np.linalg.norm(r) / np.linalg.norm(b.numpy())) <= 1e-13
        # the oracle's even-odd CG with the same first stopping rule takes the same number of steps (+-2 for
        # rounding), unless the GPU had to continue for the true residual
        _, oinfo = krylov.eo_cg(op, b.numpy(), mu, tol=1e-12)
        assert info.iters >= oinfo["iters"] - 2
    finally:
        lib.ddtm_destroy(ctx)


def test_eo_cg_true_residual_antiperiodic_both_twists(lib):
    dims = (16, 8, 8, 8)
    U = synth.gauge_field(dims, 0.2, seed=3)
    op = FineOperator(U.numpy(), 0.134, 1.5755, 1)
    b = synth.gaussian_spinor(dims, seed=4, nrhs=2)
    ctx = lib.ddtm_create(dims, (4, 4, 4, 4), 1)
    try:
        lib.ddtm_load_gauge(ctx, U.cuda(), 0.134, 1.5755)
        for mu in (0.003, -0.003):
            x = torch.zeros_like(b).cuda()
            info, code = lib.ddtm_eo_cg(ctx, x, b.cuda(), 2, mu, tol=1e-10)
            assert code == lib.OK, lib.ddtm_last_error(ctx)
            for r in range(2):
                res = np.linalg.norm(b[r].numpy() - op.apply(x[r].cpu().numpy(), mu)) / np.linalg.norm(b[r].numpy())
                assert res <= 1e-10, (mu, r, res)
        x = torch.zeros_like(b).cuda()
        info, code = lib.ddtm_eo_cg(ctx, x, b.cuda(), 2, 0.003, tol=1e-10, max_iter=5)
        assert code == lib.ERR_NOCONV and info.iters == 5 and info.max_relres > 1e-10
    finally:
        lib.ddtm_destroy(ctx)
