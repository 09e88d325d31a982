"""CUDA-graph replay of the coarsest even-odd GMRES iterations (option "graphs"): with graphs the
solves give bit-identical solutions to the direct launches (the same kernels with the same arguments),
graphs are actually cached and replayed, and the library's kernel-launch count (which counts the
kernels inside each replay) is unchanged."""

import pytest
import torch

from paper_1610_02370_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1610_02370_gb300 import build
    build.build()
    from paper_1610_02370_gb300 import ddtm
    return ddtm


@pytest.mark.parametrize("coarse_prec", [1, 2])
def test_graph_replay_is_bit_identical(lib, coarse_prec):
    dims, block, nv, mu = (8, 8, 8, 16), (4, 4, 4, 4), 12, 0.005
    U = synth.gauge_field(dims, 0.2, seed=11)
    ctx = lib.ddtm_create(dims, block, 0)
    try:
        lib.ddtm_load_gauge(ctx, U.cuda(), 0.134, 1.5755)
        p = lib.ddtm_get_params(ctx)
        p.nv[0], p.n_setup, p.post_smooth, p.coarse_prec = nv, 2, 2, coarse_prec
        lib.ddtm_set_params(ctx, p)
        lib.ddtm_setup(ctx, mu, 3)
        b = synth.gaussian_spinor(dims, seed=12, nrhs=4).cuda()
        out = {}
        for graphs in (0, 1):
            lib.ddtm_set_option(ctx, "graphs", graphs)
            for rep in range(3):  # first pass direct, second captures, third replays
                x = torch.zeros_like(b)
                lib.ddtm_timer_reset(ctx)
                info, code = lib.ddtm_solve(ctx, x, b, 4, mu)
                assert code == lib.OK and info.max_relres <= 1e-10
                out[(graphs, rep)] = (x, lib.ddtm_timer_kernel_launches(ctx), info.coarse_iters)
        cached = lib.ddtm_get_option(ctx, "graphs_cached")
        assert cached > 0
        x0, n0, c0 = out[(0, 2)]
        for rep in range(3):
            x1, n1, c1 = out[(1, rep)]
            assert torch.equal(x0, x1), rep
            assert (n1, c1) == (n0, c0), rep
        # releasing the workspace frees the library's buffers and drops the cached graphs; the next
        # solve allocates again and gives the same bits
        before = lib.ddtm_memory_in_use()
        lib.ddtm_release_workspace(ctx)
        assert lib.ddtm_get_option(ctx, "graphs_cached") == 0
        assert lib.ddtm_memory_in_use() < before
        x = torch.zeros_like(b)
        info, code = lib.ddtm_solve(ctx, x, b, 4, mu)
        assert code == lib.OK and torch.equal(x, x0)
    finally:
        lib.ddtm_destroy(ctx)


def test_autotuner_choice_leaves_results_unchanged(lib):
    """The tensor-core pass autotuner (option "autotune") times 1, 2 (and 3) CTAs per SM at the first
    launch of a shape and keeps the fastest; every output comes from the same MMAs in the same order, so
    D_c x is bit-identical with the tuner on and off, and its choice is reported."""
    dims, block, nv = (8, 8, 8, 16), (4, 4, 4, 4), 24
    U = synth.gauge_field(dims, 0.2, seed=13)
    ctx = lib.ddtm_create(dims, block, 0)
    try:
        lib.ddtm_load_gauge(ctx, U.cuda(), 0.134, 1.5755)
        p = lib.ddtm_get_params(ctx)
        p.nv[0], p.coarse_prec = nv, lib.PREC_F16
        lib.ddtm_set_params(ctx, p)
        v = synth.gaussian_vectors((nv, 16, 8, 8, 8, 4, 3), seed=14).cuda()
        lib.ddtm_set_test_vectors(ctx, 0, v, nv)
        x = synth.gaussian_vectors((12, 4, 2, 2, 2, 2 * nv), seed=15).cuda()
        outs = []
        for on in (0, 1, 1):
            lib.ddtm_set_option(ctx, "autotune", on)
            y = torch.zeros_like(x)
            lib.ddtm_apply_Dc(ctx, 1, y, x, 12, 0.03)
            torch.cuda.synchronize()
            outs.append(y)
        assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
        rep = lib.ddtm_autotune_report()
        assert rep and all(v["ctas_per_sm"] >= 1 and len(v["ms"]) >= 1 for v in rep.values())
    finally:
        lib.ddtm_set_option(ctx, "autotune", 1)
        lib.ddtm_destroy(ctx)
