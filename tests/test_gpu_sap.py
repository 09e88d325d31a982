"""GPU parity of the red-black SAP smoother (Sec. 2.4) against the CPU oracle.

The smoother is a fixed number of cycles and MR steps, so it is compared
element-wise with the oracle's even-odd block variant, red blocks first:
relative 2-norm 1e-12 in FP64 (several dependent MR steps, each with inner
products summed in a different order), 2e-6 in FP32 and 2e-3 with FP16 storage.
"""

import numpy as np
import pytest
import torch

from oracle import sap as osap
from oracle.operators import FineOperator
from paper_1610_02370_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-6, 2: 2e-3}


@pytest.fixture(scope="module")
def lib():
    from paper_1610_02370_gb300 import build
    build.build()
    from paper_1610_02370_gb300 import ddtm
    return ddtm


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def sap_case(ddtm, dims, block, eps, kappa, csw, mus, bc_t, ncycles, nmr, precs, seed=0):
    U = synth.gauge_field(dims, eps, seed=seed)
    b = synth.gaussian_spinor(dims, seed=seed + 1)
    op = FineOperator(U.numpy(), kappa, csw, bc_t)
    ctx = ddtm.ddtm_create(dims, block, bc_t)
    errs = {}
    try:
        ddtm.ddtm_load_gauge(ctx, U.cuda(), kappa, csw)
        bd = b.cuda()
        for mu in mus:
            ref = osap.sap(op, b.numpy(), mu, block, ncycles, nmr, eo=True)
            for prec in precs:
                x = torch.zeros_like(bd)
                ddtm.ddtm_sap(ctx, x, bd, 1, mu, ncycles, nmr, prec)
                e = relerr(x.cpu().numpy(), ref)
                errs[(mu, prec)] = e
                assert e < TOL[prec], (dims, mu, prec, e)
    finally:
        ddtm.ddtm_destroy(ctx)
    return errs


@pytest.mark.parametrize("bc_t", [0, 1])
def test_sap_parity_4x4x4x4(lib, bc_t):
    sap_case(lib, (4, 4, 4, 4), (2, 2, 2, 2), 0.3, 0.125, 1.0, (0.01, -0.01), bc_t, 2, 4, (0, 1, 2))


def test_sap_parity_16x8x8x8_anisotropic_blocks(lib):
    """16 x 8^3 with 4 x 2 x 4 x 2 blocks: several tiles per colour, unequal block sides."""
    sap_case(lib, (16, 8, 8, 8), (4, 2, 4, 2), 0.3, 0.13, 1.5755, (0.05,), 1, 3, 4, (0, 1, 2))


def test_sap_parity_16x16x16x32(lib):
    """16^3 x 32, eps=0.2, kappa=0.1340, c_sw=1.5755, mu=0.003: 4^4 blocks, 3 cycles x 4 MR."""
    errs = sap_case(lib, (32, 16, 16, 16), (4, 4, 4, 4), 0.2, 0.1340, 1.5755, (0.003,), 0, 3, 4, (0, 1, 2))
    print("SAP 16^3x32 relative errors", errs)


def test_sap_zero_cycles_and_field_api(lib):
    ddtm = lib
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.3, seed=5).cuda()
    b = synth.gaussian_spinor(dims, seed=6, nrhs=2).cuda()
    ctx = ddtm.ddtm_create(dims, (4, 4, 4, 4), 0)
    try:
        ddtm.ddtm_load_gauge(ctx, U, 0.13, 1.0)
        x = torch.ones_like(b)
        ddtm.ddtm_sap(ctx, x, b, 2, 0.1, 0, 3, ddtm.PREC_F32)
        assert torch.count_nonzero(x) == 0
        for prec in (1, 2):
            fb = ddtm.ddtm_field_create(ctx, prec, 2)
            fx = ddtm.ddtm_field_create(ctx, prec, 2)
            ddtm.ddtm_field_import(ctx, fb, b)
            ddtm.ddtm_sap_field(ctx, fx, fb, 0.1, 2, 3)
            x1 = torch.zeros_like(b)
            ddtm.ddtm_field_export(ctx, fx, x1)
            x2 = torch.zeros_like(b)
            ddtm.ddtm_sap(ctx, x2, b, 2, 0.1, 2, 3, prec)
            torch.cuda.synchronize()
            assert torch.equal(x1, x2)
            ddtm.ddtm_field_destroy(fb)
            ddtm.ddtm_field_destroy(fx)
    finally:
        ddtm.ddtm_destroy(ctx)



@pytest.mark.parametrize("nrhs", [3, 5, 12])
def test_sap_batched_rhs_groups(lib, nrhs):
    """A batch of 3, 5 or 12 right-hand sides in one field runs several
    right-hand sides of a block per CTA (one thread group and named barrier
    each, a ragged last group): every rhs of the batch equals, bit for bit, the
    same rhs smoothed alone (same threads, same summation order), and matches
    the oracle's SAP in FP32 and with FP16 storage."""
    ddtm = lib
    dims, block, mu = (8, 8, 8, 8), (4, 4, 4, 4), 0.02
    U = synth.gauge_field(dims, 0.3, seed=11)
    b = synth.gaussian_spinor(dims, seed=12, nrhs=nrhs)
    op = FineOperator(U.numpy(), 0.13, 1.2, 0)
    ctx = ddtm.ddtm_create(dims, block, 0)
    try:
        ddtm.ddtm_load_gauge(ctx, U.cuda(), 0.13, 1.2)
        bd = b.cuda()
        for prec in (1, 2):
            fb = ddtm.ddtm_field_create(ctx, prec, nrhs)
            fx = ddtm.ddtm_field_create(ctx, prec, nrhs)
            ddtm.ddtm_field_import(ctx, fb, bd)
            ddtm.ddtm_sap_field(ctx, fx, fb, mu, 2, 3)
            x = torch.zeros_like(bd)
            ddtm.ddtm_field_export(ctx, fx, x)
            ddtm.ddtm_field_destroy(fb)
            ddtm.ddtm_field_destroy(fx)
            x1 = torch.zeros_like(bd)
            ddtm.ddtm_sap(ctx, x1, bd, nrhs, mu, 2, 3, prec)  # one right-hand side at a time
            torch.cuda.synchronize()
            assert torch.equal(x, x1), prec
            xs = x.cpu().numpy()
            for r in (0, nrhs // 2, nrhs - 1):
                ref = osap.sap(op, b[r].numpy(), mu, block, 2, 3, eo=True)
                assert relerr(xs[r], ref) < TOL[prec], (prec, r, relerr(xs[r], ref))
    finally:
        ddtm.ddtm_destroy(ctx)
