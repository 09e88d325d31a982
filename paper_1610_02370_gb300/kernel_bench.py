"""Small drivers that run one kernel family of libddtm on a synthetic lattice,
for timing and for profiling a single kernel in isolation.

    python -m paper_1610_02370_gb300.kernel_bench coarse --dims 48 24 24 24 --nv 24 --nrhs 12 --reps 4
    python -m paper_1610_02370_gb300.kernel_bench dslash --dims 64 32 32 32 --prec 1 --nrhs 1 --reps 10
    python -m paper_1610_02370_gb300.kernel_bench solve --dims 64 32 32 32 --nrhs 12 --outer-iters 1
    python -m paper_1610_02370_gb300.kernel_bench sap --dims 48 24 24 24 --nrhs 12 --cycles 2
    python -m paper_1610_02370_gb300.kernel_bench csolve --dims 64 32 32 32 --nrhs 12 --ctol 1e-2

``coarse`` builds the aggregation and the Galerkin coarse operator from
Gaussian test vectors (no setup iterations; the second build is timed per
kernel) and applies the coarse operator D_c (Sec. 2.3) to a batch of nrhs
vectors; ``dslash`` applies D(mu) (Sec. 2.1) to one field; ``solve`` runs the
first outer iterations of a batched solve (every kernel of the solve phase);
``sap`` runs the SAP smoother (Sec. 2.4) on a batch of Gaussian right-hand sides;
``csolve`` runs the batched coarsest-level GMRES (Sec. 2.5).
Each prints one JSON line with its times (CUDA events).
"""

import argparse
import json
import statistics

import torch

from . import ddtm, synth


def _events(fn, reps):
    st = torch.cuda.current_stream()
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def coarse(args):
    dims = tuple(args.dims)
    U = synth.gauge_field(dims, args.eps, seed=0, device="cuda")
    ctx = ddtm.ddtm_create(dims, (4, 4, 4, 4), 0)
    try:
        ddtm.ddtm_load_gauge(ctx, U, args.kappa, args.csw)
        p = ddtm.ddtm_get_params(ctx)
        p.nv[0] = args.nv
        p.coarse_prec = args.coarse_prec
        ddtm.ddtm_set_params(ctx, p)
        lat = tuple(dims)
        v = synth.gaussian_vectors((args.nv,) + lat + (4, 3), seed=5, device="cuda")
        ddtm.ddtm_set_test_vectors(ctx, 0, v, args.nv)  # warm-up build (module load, allocation)
        ddtm.ddtm_timer_reset(ctx)
        ddtm.ddtm_timer_enable(ctx, True)
        ddtm.ddtm_set_test_vectors(ctx, 0, v, args.nv)  # aggregation and Galerkin, timed per kernel
        ddtm.ddtm_timer_enable(ctx, False)
        build = {k: round(t["ms"], 3) for k, t in ddtm.ddtm_timer_report(ctx).items()}
        del v
        torch.cuda.empty_cache()
        cl = tuple(d // 4 for d in dims)
        x = synth.gaussian_vectors((args.nrhs,) + cl + (2 * args.nv,), seed=6, device="cuda")
        y = torch.zeros_like(x)
        ms = _events(lambda: ddtm.ddtm_apply_Dc(ctx, 1, y, x, args.nrhs, 0.01), args.reps)
        print(json.dumps({"kernel": "coarse", "dims": dims, "nv": args.nv, "nrhs": args.nrhs,
                          "coarse_prec": args.coarse_prec, "ms_per_call": ms, "build_ms": build}))
    finally:
        ddtm.ddtm_destroy(ctx)


def solve(args):
    """The first outer iterations of a 12-rhs solve on Gaussian test vectors (no
    setup iterations): restriction, coarsest even-odd GMRES (tensor-core
    passes, FP16-basis Gram-Schmidt), prolongation, SAP, FP32 D applications."""
    dims = tuple(args.dims)
    U = synth.gauge_field(dims, args.eps, seed=0, device="cuda")
    ctx = ddtm.ddtm_create(dims, (4, 4, 4, 4), 0)
    try:
        ddtm.ddtm_load_gauge(ctx, U, args.kappa, args.csw)
        p = ddtm.ddtm_get_params(ctx)
        p.nv[0] = args.nv
        p.coarse_prec = args.coarse_prec
        p.outer_restart = max(args.outer_iters, 1)
        p.outer_max_iters = args.outer_iters
        p.post_smooth = 2
        ddtm.ddtm_set_params(ctx, p)
        v = synth.gaussian_vectors((args.nv,) + tuple(dims) + (4, 3), seed=5, device="cuda")
        ddtm.ddtm_set_test_vectors(ctx, 0, v, args.nv)
        del v
        torch.cuda.empty_cache()
        b = synth.point_sources(dims, device="cuda")[: args.nrhs].contiguous()
        x = torch.zeros_like(b)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        info, code = ddtm.ddtm_solve(ctx, x, b, args.nrhs, args.mu)
        e1.record(st)
        e1.synchronize()
        if code not in (ddtm.OK, ddtm.ERR_NOCONV):
            raise ddtm.DDTMError(code, ddtm.ddtm_last_error(ctx))
        print(json.dumps({"kernel": "solve", "dims": dims, "nv": args.nv, "nrhs": args.nrhs,
                          "outer_iters": info.iters, "coarse_iters": info.coarse_iters,
                          "max_relres": info.max_relres, "ms": e0.elapsed_time(e1)}))
    finally:
        ddtm.ddtm_destroy(ctx)


def csolve(args):
    """Batched coarsest-level even-odd GMRES (Sec. 2.5) on nrhs Gaussian coarse
    vectors after an aggregation from Gaussian test vectors: the tensor-core
    Schur complement and the FP16-basis Gram-Schmidt kernels at the sizes of
    the solver's coarse solves (restart 100, tolerance --ctol)."""
    dims = tuple(args.dims)
    U = synth.gauge_field(dims, args.eps, seed=0, device="cuda")
    ctx = ddtm.ddtm_create(dims, (4, 4, 4, 4), 0)
    try:
        ddtm.ddtm_load_gauge(ctx, U, args.kappa, args.csw)
        del U
        p = ddtm.ddtm_get_params(ctx)
        p.nv[0] = args.nv
        p.coarse_prec = args.coarse_prec
        p.coarse_tol = args.ctol
        ddtm.ddtm_set_params(ctx, p)
        v = synth.gaussian_vectors((args.nv,) + tuple(dims) + (4, 3), seed=5, device="cuda")
        ddtm.ddtm_set_test_vectors(ctx, 0, v, args.nv)
        del v
        torch.cuda.empty_cache()
        cl = tuple(d // 4 for d in dims)
        b = synth.gaussian_vectors((args.nrhs,) + cl + (2 * args.nv,), seed=6, device="cuda")
        x = torch.zeros_like(b)
        res = {}
        ms = _events(lambda: res.update(out=ddtm.ddtm_coarse_solve_batch(ctx, x, b, args.nrhs, args.muc)), args.reps)
        print(json.dumps({"kernel": "csolve", "dims": dims, "nv": args.nv, "nrhs": args.nrhs, "ctol": args.ctol,
                          "iters": res["out"][0], "code": res["out"][1], "ms_per_call": ms}))
    finally:
        ddtm.ddtm_destroy(ctx)


def sap(args):
    """SAP smoother (Sec. 2.4) on a batch of nrhs Gaussian right-hand sides from x = 0."""
    dims = tuple(args.dims)
    U = synth.gauge_field(dims, args.eps, seed=0, device="cuda")
    ctx = ddtm.ddtm_create(dims, (4, 4, 4, 4), 0)
    try:
        ddtm.ddtm_load_gauge(ctx, U, args.kappa, args.csw)
        b = synth.gaussian_spinor(dims, seed=1, nrhs=args.nrhs, device="cuda")
        fb = ddtm.ddtm_field_create(ctx, args.sap_prec, args.nrhs)
        fx = ddtm.ddtm_field_create(ctx, args.sap_prec, args.nrhs)
        ddtm.ddtm_field_import(ctx, fb, b)
        del b
        torch.cuda.empty_cache()
        ms = _events(lambda: ddtm.ddtm_sap_field(ctx, fx, fb, args.mu, args.cycles, args.nmr), args.reps)
        print(json.dumps({"kernel": "sap", "dims": dims, "prec": args.sap_prec, "nrhs": args.nrhs, "cycles": args.cycles,
                          "nmr": args.nmr, "ms_per_call": ms}))
        ddtm.ddtm_field_destroy(fx)
        ddtm.ddtm_field_destroy(fb)
    finally:
        ddtm.ddtm_destroy(ctx)


def dslash(args):
    dims = tuple(args.dims)
    U = synth.gauge_field(dims, args.eps, seed=0, device="cuda")
    ctx = ddtm.ddtm_create(dims, (4, 4, 4, 4), 0)
    try:
        ddtm.ddtm_load_gauge(ctx, U, args.kappa, args.csw)
        nr = args.nrhs if args.nrhs > 0 else 1
        x = synth.gaussian_spinor(dims, seed=1, nrhs=nr, device="cuda")
        fx = ddtm.ddtm_field_create(ctx, args.prec, nr)
        fy = ddtm.ddtm_field_create(ctx, args.prec, nr)
        ddtm.ddtm_field_import(ctx, fx, x)
        del x
        ms = _events(lambda: ddtm.ddtm_apply_D_field(ctx, fy, fx, 0.01), args.reps)
        print(json.dumps({"kernel": "dslash", "dims": dims, "prec": args.prec, "nrhs": nr, "ms_per_call": ms}))
        ddtm.ddtm_field_destroy(fx)
        ddtm.ddtm_field_destroy(fy)
    finally:
        ddtm.ddtm_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["coarse", "dslash", "solve", "sap", "csolve"])
    ap.add_argument("--dims", type=int, nargs=4, default=[48, 24, 24, 24])
    ap.add_argument("--eps", type=float, default=0.15)
    ap.add_argument("--kappa", type=float, default=0.137)
    ap.add_argument("--csw", type=float, default=1.5755)
    ap.add_argument("--nv", type=int, default=24)
    ap.add_argument("--nrhs", type=int, default=12)
    ap.add_argument("--coarse-prec", type=int, default=2)
    ap.add_argument("--prec", type=int, default=1)
    ap.add_argument("--reps", type=int, default=4)
    ap.add_argument("--mu", type=float, default=0.0015)
    ap.add_argument("--outer-iters", type=int, default=1)
    ap.add_argument("--sap-prec", type=int, default=2)
    ap.add_argument("--cycles", type=int, default=2)
    ap.add_argument("--nmr", type=int, default=3)
    ap.add_argument("--ctol", type=float, default=1e-2)
    ap.add_argument("--muc", type=float, default=0.0078)
    args = ap.parse_args()
    from . import build
    build.build()
    {"coarse": coarse, "dslash": dslash, "solve": solve, "sap": sap, "csolve": csolve}[args.what](args)


if __name__ == "__main__":
    main()
