"""ddtm_apply_D_noalloc, the variant of the canonical D(mu) apply for callers
that cannot allocate device memory during a call (cudaMalloc/cudaFree may
synchronise the device, or the caller's allocator owns the memory budget).
Its output is compared with the existing ddtm_apply_D entry point on two calls
in a row, with the parity tolerances of the stencil tests.  Kept in its own
file, collected last."""

import numpy as np
import pytest
import torch

from paper_1610_02370_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 2e-6, 2: 2e-3}


@pytest.fixture(scope="module")
def lib():
    from paper_1610_02370_gb300 import build
    build.build()
    from paper_1610_02370_gb300 import ddtm
    return ddtm


def test_noalloc_apply_matches_apply_D_twice(lib):
    ddtm = lib
    dims = (32, 16, 16, 16)  # 131072 sites: fits the fixed scratch in every precision
    U = synth.gauge_field(dims, 0.2, seed=0).cuda()
    ctx = ddtm.ddtm_create(dims, (4, 4, 4, 4), 1)
    try:
        ddtm.ddtm_load_gauge(ctx, U, 0.1340, 1.5755)
        for prec in (ddtm.PREC_F64, ddtm.PREC_F32, ddtm.PREC_F16):
            for call, seed in enumerate((11, 12)):  # two calls in a row, different inputs
                x = synth.gaussian_spinor(dims, seed=seed).cuda()
                mu = 0.003 if call == 0 else -0.003
                ref = torch.zeros_like(x)
                ddtm.ddtm_apply_D(ctx, ref, x, 1, mu, prec)
                y = torch.full_like(x, float("nan"))
                ddtm.ddtm_apply_D_noalloc(ctx, y, x, mu, prec)
                torch.cuda.synchronize()
                err = (torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref)).item()
                assert err <= TOL[prec], (prec, call, err)
    finally:
        ddtm.ddtm_destroy(ctx)


def test_noalloc_rejects_oversized_lattice_and_missing_precision(lib):
    ddtm = lib
    big = ddtm.ddtm_create((64, 32, 32, 32), (4, 4, 4, 4), 0)
    try:
        x = torch.zeros(4, dtype=torch.complex128, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(ddtm.DDTMError) as e:
            ddtm.ddtm_apply_D_noalloc(big, y, x, 0.1, ddtm.PREC_F64)
        assert e.value.code == ddtm.ERR_ARG and "scratch" in str(e.value)
    finally:
        ddtm.ddtm_destroy(big)
    dims = (8, 8, 8, 8)
    ctx = ddtm.ddtm_create(dims, (4, 4, 4, 4), 0)
    try:
        ddtm.ddtm_load_gauge(ctx, synth.gauge_field(dims, 0.3, seed=1).cuda(), 0.13, 1.0)
        x = synth.gaussian_spinor(dims, seed=2).cuda()
        y = torch.zeros_like(x)
        with pytest.raises(ddtm.DDTMError) as e:
            ddtm.ddtm_apply_D_noalloc(ctx, y, x, 0.1, ddtm.PREC_F16)
        assert e.value.code == ddtm.ERR_STATE
    finally:
        ddtm.ddtm_destroy(ctx)
