#!/usr/bin/env python
"""Benchmark of the GB300 twisted-mass DD-alpha-AMG hot path.

One step = one point-to-all propagator on the 32^3 x 64 workload: adaptive
setup (test vectors, P, Galerkin coarse operator) followed by the solve of the
12 spin-colour point sources to FP64 relative residual 1e-10, all through the
C ABI of libddtm with inputs resident on the device.  The metric is seconds per
12-rhs solve (setup included, lower is better).  Beside it the line carries
the D(mu) stencil bandwidth against the HBM roof, the roofline of the dominant
kernel, an end-to-end number through host buffers, clocks, and the CPU oracle
timed on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

With N > 1 (torchrun) every rank solves its own propagator on its own GPU
(independent replicas: the method's units here are whole propagators) and the
line reports the whole job.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D_TM apply GB/s vs HBM peak; s per 12-rhs solve to 1e-10, mixed vs FP64"
UNIT = "s per 12-rhs solve"

# Workloads: synthetic SU(3) links exp(i eps H) at the lattice sizes and masses
# of the paper's ensembles; multigrid parameters of the two-level set (4^4
# aggregates, Nv = 24, 6 setup iterations) with the smoother of Table 1.
WORKLOADS = {
    "32x32x32x64": dict(dims=(64, 32, 32, 32), eps=0.12, kappa=0.1372, c_sw=1.5755, mu=0.0015),
    "24x24x24x48": dict(dims=(48, 24, 24, 24), eps=0.15, kappa=0.1370, c_sw=1.5755, mu=0.002),
    "16x16x16x32": dict(dims=(32, 16, 16, 16), eps=0.2, kappa=0.1340, c_sw=1.5755, mu=0.003),
    # three levels (4^4 then 2^4 aggregates, N_v = 24 then 32), both twist signs with one setup
    "48x48x48x96": dict(dims=(96, 48, 48, 48), eps=0.1, kappa=0.1373, c_sw=1.5755, mu=0.0009, levels=3, nv1=32,
                        twists=(1, -1)),
}
# Post-smoothing: Table 1 uses 4 SAP cycles, tuned for the real ensemble cA2.09.48.  On these synthetic
# fields the mass lies well below critical and SAP amplifies smooth modes, so the cycle count is tuned as
# the paper does per ensemble: at 24^3x48 one setup then single-rhs solves gave 4 cycles: no convergence
# in 120 iterations; 2 cycles: 22 iterations; 1 cycle: 27 (parameter study recorded with the design notes).
MG = dict(block=(4, 4, 4, 4), nv=24, n_setup=6, post_smooth=2, nmr=3, outer_restart=30, outer_tol=1e-10,
          smoother_prec=2, coarse_prec=2)
NRHS = 12
SEED = 2024

# Algorithmic bytes per site of one D(mu) application: links 4x18 reals (each
# read once), clover 2 x 36 reals, x and y 24 reals each; FP16 adds two 4-byte
# site scales (x and y).
DSLASH_BYTES = {"f64": 1536, "f32": 768, "f16": 392}
S2 = {"f64": 16, "f32": 8, "f16": 4}  # bytes per stored complex number


def dslash_bytes(prec, nrhs):
    """Algorithmic bytes per site of one D(mu) launch over nrhs right-hand sides: links (4 x 18 reals)
    and clover (72 reals) once, x and y (24 reals each, + one 4-byte scale each in FP16) per rhs."""
    s2 = S2[prec]
    nrm = 4 if prec == "f16" else 0
    return (36 + 36) * s2 + nrhs * 2 * (12 * s2 + nrm)


def algorithmic_bytes(name, V, Vb, b, nv, Nc, rhs=1.0):
    """Algorithmic HBM bytes of one launch of kernel ``name`` (every array
    element the kernel must touch, once) carrying ``rhs`` right-hand sides, or
    None if no model applies."""
    n = 2 * nv
    prec = name.rsplit("_", 1)[-1]
    s2 = S2.get(prec)
    face = sum(2.0 / bb for bb in b)  # halo sites per site of a block (both faces, 4 directions)
    if name.startswith("dslash_"):
        return dslash_bytes(prec, rhs) * V
    if name.startswith("sap_half_"):
        half = V / 2
        nrm = 4 if prec == "f16" else 0
        per = (36 + 36 + 36) * s2   # own links, clover, even-site inverses (72 complex per even site): once
        vec = 12 * s2 + nrm         # b
        vec += 2 * (12 * s2 + nrm)  # x read and written on the block
        vec += face * (12 * s2 + nrm)  # neighbour x on the faces
        per += face * 9 * s2 / 2    # links of backward face hops
        return half * (per + rhs * vec)
    if name.startswith("restrict_") or name.startswith("prolong_"):
        pbytes = 4 if (prec == "f16") else 8
        nrm = 4 if prec == "f16" else 0
        fine = V * (12 * s2 + nrm)
        return V * 12 * nv * pbytes + rhs * (fine * (2 if name.startswith("prolong") else 1) + Nc * n * 8)
    if name.startswith("coarse_even_"):
        # 8 hop blocks and the FP32 self-block inverse per even site, read once per batch of NRHS
        d = S2[prec]
        return Nc / 2 * (8 * n * n * d + n * n * 8 + 2 * n * NRHS * 8)
    if name.startswith("coarse_apply_odd_"):
        # self block and 8 hop blocks per odd site; x_o, the even input and y_o
        d = S2[prec]
        return Nc / 2 * (9 * n * n * d + 3 * n * NRHS * 8)
    return None


# DRAM traffic per unit from one ncu capture of the kernel as it stands (profiles/), scaled to a
# launch of the bench workload by the units it processes; remove an entry when its kernel changes.
NCU_TRAFFIC = {
    "sap_half_f16": {"bytes_per_site_rhs": 1.0728e9 / (663552 / 2 * 12), "capture": "k_sap_half_24x24x24x48.md"},
}


def algorithmic_flops(name, V, Vb, b, nv, nmr, rhs_per_launch):
    """Algorithmic FP32 flops of one launch of the compute-bound kernels (None
    otherwise): Galerkin build and Gram-Schmidt per aggregate times the number
    of aggregates; SAP half-sweep (n_MR + 1) D applications of 1920 flops per
    site of the colour, per right-hand side."""
    n = 2 * nv
    Nc = V // Vb
    if name == "galerkin":
        # D applied to the n columns of P on the aggregate and its faces (1920 flops per site),
        # self block: n x n entries of 6 Vb complex products; hop block k: 6 Vb / b_k products
        return Nc * (n * Vb * 1920 + 8 * n * n * 6 * Vb + sum(2 * 8 * n * n * 6 * Vb / bb for bb in b))
    if name == "build_P":
        # two Gram-Schmidt passes over the nv vectors of each aggregate half (6 Vb entries)
        m = 6 * Vb
        return Nc * 2 * 2 * (nv * (nv - 1) / 2 * 16 * m + nv * 8 * m)
    if name.startswith("sap_half_"):
        return rhs_per_launch * (V / 2) * (nmr + 1) * 1920
    return None


def max_over_ranks(value, dist, device):
    """Largest per-rank value over the job (the slowest replica sets the step
    time); ``dist`` is torch.distributed or None for one process."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="32x32x32x64", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cpu-all", action="store_true", help="skip the all-cores oracle timing")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true", help="skip the oracle residual of the full-size solutions")
    ap.add_argument("--study", choices=["eo-cg", "aggregation", "levels", "oracle"], default=None,
                    help="eo-cg: the even-odd CG baseline against DD-alpha-AMG, t_total = t_setup + n_rhs t_solve "
                         "(Sec. 3.1.2, Fig. 3); aggregation: block size x N_v sweep (Sec. 3.3, Table 4)")
    ap.add_argument("--lattices", default=None, help="--study oracle: comma-separated lattices (default: all four)")
    ap.add_argument("--oracle-units", default=None, help=argparse.SUPPRESS)  # child process of the CPU baseline
    return ap.parse_args()


# ---- clocks -----------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---- CPU oracle baseline -------------------------------------------------------------------------
def oracle_unit_times(wl, sample_dims=(16, 8, 8, 8)):
    """Time the oracle's building blocks on a bounded sample lattice with the
    workload's couplings and multigrid parameters; returns seconds per site (or
    per coarse site) of each block."""
    import numpy as np
    from oracle import aggregation, coarse, krylov, sap
    from oracle.operators import FineOperator
    from paper_1610_02370_gb300 import synth

    U = synth.gauge_field(sample_dims, wl["eps"], seed=0).numpy()
    op = FineOperator(U, wl["kappa"], wl["c_sw"])
    V = float(np.prod(op.lat))
    mu = wl["mu"]
    psi = synth.gaussian_spinor(sample_dims, seed=1).numpy()
    out = {}

    def timed(fn, reps=1):
        t = time.perf_counter()
        for _ in range(reps):
            r = fn()
        return (time.perf_counter() - t) / reps, r

    t, _ = timed(lambda: op.apply(psi, mu), 2)
    out["dslash"] = t / V
    blk = MG["block"]

    def half_sweep():
        r = psi - op.apply(psi * 0.5, mu)
        return sap.block_solve(op, r, mu, blk, 0, MG["nmr"])
    t, _ = timed(half_sweep)
    out["sap_half"] = t / V
    v = synth.gaussian_vectors((MG["nv"],) + op.lat + (4, 3), seed=3).numpy()
    t, W = timed(lambda: aggregation.build_P(op, v, blk))
    out["build_P"] = t / V
    t, cop = timed(lambda: coarse.build_coarse_operator(op, W, blk))
    out["galerkin"] = t / V
    t, c = timed(lambda: aggregation.restrict(W, psi, op.lat, blk))
    out["restrict"] = t / V
    t, _ = timed(lambda: aggregation.prolong(W, c, op.lat, blk))
    out["prolong"] = t / V
    Nc = float(np.prod(cop.lat))
    nit = 10
    t, _ = timed(lambda: krylov.eo_gmres(cop, c, 5.2 * mu, restart=nit, max_restarts=0, tol=1e-300))
    out["coarse_iter"] = t / nit / Nc
    out["_sample"] = "x".join(str(d) for d in (sample_dims[1], sample_dims[2], sample_dims[3], sample_dims[0]))
    return out


def oracle_study(only=None):
    """The oracle as it stands, timed directly (no extrapolation) on this host in one process: at
    the four lattices of the parameter sets (4^4 with 2^4 blocks; 16^3x32, 24^3x48 and 32^3x64 with
    4^4 blocks) the construction of the operator (clover term), one application of D(mu) and one SAP
    cycle (red and black half-sweeps, Sec. 2.4) on one Gaussian right-hand side, and on 4^4 the
    plain FP64 GMRES solve to relative residual 1e-10.  Run it with one BLAS / OpenMP thread for a
    single-core figure."""
    import numpy as np
    from oracle import krylov, sap
    from oracle.operators import FineOperator
    from paper_1610_02370_gb300 import synth

    cases = [("4x4x4x4", (4, 4, 4, 4), 0.3, 0.125, 1.0, 0.01, (2, 2, 2, 2), 4)]
    for name, nmr in (("16x16x16x32", 4), ("24x24x24x48", MG["nmr"]), ("32x32x32x64", MG["nmr"])):
        w = WORKLOADS[name]
        cases.append((name, w["dims"], w["eps"], w["kappa"], w["c_sw"], w["mu"], MG["block"], nmr))
    rows = []
    for name, dims, eps, kappa, csw, mu, blk, nmr in cases:
        if only and name not in only:
            continue
        t0 = time.perf_counter()
        op = FineOperator(synth.gauge_field(dims, eps, seed=0).numpy(), kappa, csw)
        t_build = time.perf_counter() - t0
        b = synth.gaussian_spinor(dims, seed=1).numpy()
        t0 = time.perf_counter()
        op.apply(b, mu)
        t_d = time.perf_counter() - t0
        t0 = time.perf_counter()
        sap.sap(op, b, mu, blk, 1, nmr, eo=True)
        t_sap = time.perf_counter() - t0
        row = {"lattice": name, "sites": int(np.prod(dims)), "operator_build_s": t_build, "apply_D_s": t_d,
               "sap_cycle_s": t_sap, "sap_blocks": list(blk), "nmr": nmr}
        if name == "4x4x4x4":
            t0 = time.perf_counter()
            _, info = krylov.gmres(lambda v: op.apply(v, mu), b, 30, 100, 1e-10)
            row.update(gmres_solve_s=time.perf_counter() - t0, gmres_relres=float(info["relres"]),
                       gmres_iters=int(info.get("iters", 0)))
        rows.append(row)
        sys.stderr.write("[oracle] %s\n" % json.dumps(row))
        sys.stderr.flush()
        del op
    print(json.dumps({"study": "oracle", "host": host_cpu(), "threads": os.environ.get("OMP_NUM_THREADS"),
                      "rows": rows}))


def host_cpu():
    """Core count and CPU model of this host, recorded beside the CPU baseline (never raises)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            fields = {}
            for line in f:
                k, sep, v = line.partition(":")
                if sep and v.strip():
                    fields.setdefault(k.strip(), v.strip())
        model = fields.get("model name") or (("CPU part " + fields["CPU part"]) if "CPU part" in fields else None)
    except (OSError, ValueError):
        pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.machine() or "unknown"}


ONE_THREAD = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                "NUMEXPR_NUM_THREADS", "VECLIB_MAXIMUM_THREADS")}


def oracle_unit_times_one_core(workload):
    """oracle_unit_times in a child process whose BLAS / OpenMP pools are
    limited to one thread, so the baseline runs on exactly one host core."""
    env = dict(os.environ, **ONE_THREAD)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-units", workload],
                       capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def host_cores():
    """Host cores this process may run on (its affinity mask, else the CPU count)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


# at most this many oracle processes at once (each imports torch and holds its sample: ~1 GB)
ORACLE_MAX_PROCS = 32


def oracle_unit_times_all_cores(workload, ncores=None):
    """oracle_unit_times in one single-threaded child process per host core (at most ORACLE_MAX_PROCS), all
    running at once: each child times the building blocks under full-node load, so the node does ncores
    units of work in the time one child takes for one.  Returns the children's mean unit times divided by ncores (seconds per
    unit of work with every core busy) and ncores."""
    ncores = ncores or min(host_cores(), ORACLE_MAX_PROCS)
    env = dict(os.environ, **ONE_THREAD)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-units", workload]
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
             for _ in range(ncores)]
    outs, err = [], None
    for p in procs:
        try:
            o, e = p.communicate(timeout=1800)
        except subprocess.TimeoutExpired:
            p.kill()  # this child only
            o, e = p.communicate()
            err = err or "an oracle child timed out"
            continue
        if p.returncode != 0:
            err = err or ("oracle timing failed: " + e[-500:])
            continue
        outs.append(json.loads(o.strip().splitlines()[-1]))
    if err:
        raise RuntimeError(err)
    keys = [k for k in outs[0] if not k.startswith("_")]
    unit = {k: statistics.mean(o[k] for o in outs) / ncores for k in keys}
    unit["_sample"] = outs[0]["_sample"]
    return unit, ncores


def oracle_estimate(unit, counts, V, Nc):
    """Oracle seconds for the GPU step's work: every kernel family's work units
    (right-hand sides or vectors processed, summed over its launches) times the
    oracle's time for one unit, scaled per site.  Returns (seconds, coarse
    rhs-iterations)."""
    def u(prefix):
        return sum(v.get("units", v["launches"]) for k, v in counts.items() if k.startswith(prefix))

    def n(prefix):
        return sum(v["launches"] for k, v in counts.items() if k.startswith(prefix))
    coarse_iters = u("coarse_tc_hop_even") + u("coarse_tc_full")
    if coarse_iters == 0:  # FP32 SIMT coarse stencil: one even-site pass per iteration plus two per solve
        coarse_iters = max(0, u("coarse_even_") - 2 * u("restrict_"))
    t = 0.0
    t += u("dslash_") * unit["dslash"] * V
    t += u("sap_half_") * unit["sap_half"] * V
    t += n("build_P") * unit["build_P"] * V
    t += n("galerkin") * unit["galerkin"] * V
    t += u("restrict_") * unit["restrict"] * V
    t += u("prolong_") * unit["prolong"] * V
    t += coarse_iters * unit["coarse_iter"] * Nc
    return t, coarse_iters


# Work of one step of the default workload (launches and work units per kernel
# family of the library, from a GPU run of this benchmark), used by the
# reference arm, which runs no GPU code.  Updated when the method's iteration
# counts change.
REFERENCE_COUNTS = {
    "dslash_f32": {"launches": 324, "units": 324}, "dslash_f64": {"launches": 24, "units": 24},
    "sap_half_f16": {"launches": 132, "units": 1872}, "build_P": {"launches": 6, "units": 144},
    "galerkin": {"launches": 6, "units": 6}, "restrict_f16": {"launches": 32, "units": 444},
    "prolong_f16": {"launches": 32, "units": 444}, "coarse_tc_hop_even": {"launches": 5340, "units": 71196},
    "coarse_even_f32": {"launches": 64, "units": 888},
}


def reference_arm(args):
    """CPU oracle on a bounded sample, scaled to the workload (see oracle_estimate)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    wl = WORKLOADS[args.workload]
    T, X, Y, Z = wl["dims"]
    V = T * X * Y * Z
    Nc = V // int(np.prod(MG["block"]))
    counts = json.loads(os.environ.get("DDTM_REFERENCE_COUNTS", "null")) or REFERENCE_COUNTS
    # every step times the oracle on all host cores at once (one single-threaded process per core);
    # if that cannot run, on one core
    vals, cores, note = [], 1, None
    for i in range(args.warmup + args.steps):
        try:
            unit, cores = oracle_unit_times_all_cores(args.workload)
        except (RuntimeError, OSError, ValueError, IndexError, KeyError) as e:
            unit, cores, note = oracle_unit_times_one_core(args.workload), 1, "all-cores timing failed: %s" % e
        est, _ = oracle_estimate(unit, counts, V, Nc)
        if i >= args.warmup:
            vals.append(est)
    val = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload + " propagator (12 point sources)", **{k: wl[k] for k in wl},
                       "mg": MG},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "host": host_cpu(),
                             "sample": "oracle building blocks timed on a %s lattice (%s), scaled per site to %s "
                                       "and multiplied by the work units (right-hand sides, vectors) of one GPU "
                                       "step" % (unit["_sample"], "one single-threaded process per host core, all "
                                                 "at once; per-unit time = their mean / cores" if cores > 1 else
                                                 "one single-threaded process", args.workload),
                             **({"note": note} if note else {})},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---- studies (one GPU, not part of the benchmark line) -------------------------------------------
def _mg_ctx(ddtm, dims, U, wl, block=None, nv=None, stream=None):
    ctx = ddtm.ddtm_create(dims, block or MG["block"], 0)
    if stream is not None:
        ddtm.ddtm_set_stream(ctx, stream.cuda_stream)
    p = ddtm.ddtm_get_params(ctx)
    p.nv[0] = nv or MG["nv"]
    for k in ("n_setup", "post_smooth", "nmr", "outer_restart", "outer_tol", "smoother_prec", "coarse_prec"):
        setattr(p, k, MG[k])
    ddtm.ddtm_set_params(ctx, p)
    ddtm.ddtm_load_gauge(ctx, U, wl["kappa"], wl["c_sw"])
    return ctx


def _timed(torch, stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, out


def study(args):
    import torch
    from paper_1610_02370_gb300 import build as _build
    _build.build()
    from paper_1610_02370_gb300 import ddtm, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    wl = WORKLOADS[args.workload]
    dims = wl["dims"]
    mu = wl["mu"]
    U = synth.gauge_field(dims, wl["eps"], seed=0, device="cuda")
    b = synth.point_sources(dims, device="cuda")
    out = {"study": args.study, "workload": args.workload, "mu": mu}
    if args.study == "eo-cg":
        # DD-alpha-AMG: one setup, then the 12 point sources in one batch (warm-up run first)
        ctx = _mg_ctx(ddtm, dims, U, wl, stream=stream)
        x = torch.zeros_like(b)
        ddtm.ddtm_setup(ctx, mu, SEED)
        ddtm.ddtm_solve(ctx, x, b, NRHS, mu)
        t_setup, _ = _timed(torch, stream, lambda: ddtm.ddtm_setup(ctx, mu, SEED))
        t_solve12, (info, code) = _timed(torch, stream, lambda: ddtm.ddtm_solve(ctx, x, b, NRHS, mu))
        ddtm.ddtm_destroy(ctx)
        # even-odd CG (FP64), one point source, to the same true relative residual
        c2 = ddtm.ddtm_create(dims, MG["block"], 0)
        ddtm.ddtm_set_stream(c2, stream.cuda_stream)
        ddtm.ddtm_load_gauge(c2, U, wl["kappa"], wl["c_sw"])
        x1 = torch.zeros_like(b[0])
        t_cg, (cinfo, ccode) = _timed(torch, stream,
                                      lambda: ddtm.ddtm_eo_cg(c2, x1, b[0], 1, mu, MG["outer_tol"], 200000))
        ddtm.ddtm_destroy(c2)
        t_rhs = t_solve12 / NRHS
        out.update({"mg": {"setup_s": t_setup, "solve_12rhs_s": t_solve12, "solve_per_rhs_s": t_rhs,
                           "outer_iters": info.iters, "max_relres": info.max_relres},
                    "eo_cg": {"solve_s": t_cg, "iters": cinfo.iters, "relres": cinfo.max_relres,
                              "converged": ccode == ddtm.OK, "s_per_iter": t_cg / max(cinfo.iters, 1)},
                    "t_total_s": {str(n): {"mg": t_setup + n * t_rhs, "eo_cg": n * t_cg,
                                           "speedup": n * t_cg / (t_setup + n * t_rhs)} for n in (1, 12, 100)},
                    "model": "t_total(n) = t_setup + n t_solve (MG, solve per rhs from the 12-rhs batch) "
                             "against n t_cg (one CG solve per rhs)"})
    elif args.study == "levels":
        # two against three levels (4^4 then 2^4 aggregates, N_v 24 then 32): setup and one 12-rhs solve,
        # with the per-kernel timers on (durations of each kernel family)
        runs = []
        for levels in (2, 3):
            ctx = _mg_ctx(ddtm, dims, U, wl, stream=stream)
            if levels == 3:
                p = ddtm.ddtm_get_params(ctx)
                p.n_levels, p.nv[1] = 3, 32
                for m in range(4):
                    p.block[1][m] = 2
                ddtm.ddtm_set_params(ctx, p)
            x = torch.zeros_like(b)
            ddtm.ddtm_timer_reset(ctx)
            ddtm.ddtm_timer_enable(ctx, True)
            t_setup, _ = _timed(torch, stream, lambda: ddtm.ddtm_setup(ctx, mu, SEED))
            rep_setup = ddtm.ddtm_timer_report(ctx)
            ddtm.ddtm_timer_reset(ctx)
            t_solve, (info, code) = _timed(torch, stream, lambda: ddtm.ddtm_solve(ctx, x, b, NRHS, mu))
            rep_solve = ddtm.ddtm_timer_report(ctx)
            ddtm.ddtm_timer_enable(ctx, False)
            top = lambda rep: {k: round(v["ms"], 1) for k, v in sorted(rep.items(), key=lambda kv: -kv[1]["ms"])[:12]}
            runs.append({"levels": levels, "setup_s": t_setup, "solve_s": t_solve, "outer_iters": info.iters,
                         "coarse_rhs_iters": info.coarse_iters, "max_relres": info.max_relres,
                         "converged": code == ddtm.OK, "setup_top_ms": top(rep_setup), "solve_top_ms": top(rep_solve),
                         "launches_solve": sum(v["launches"] for v in rep_solve.values())})
            ddtm.ddtm_destroy(ctx)
            torch.cuda.empty_cache()
        out["runs"] = runs
    else:
        runs = []
        for block in ((4, 4, 4, 4), (2, 2, 2, 2)):
            for nv in (16, 24, 32):
                ctx = _mg_ctx(ddtm, dims, U, wl, block=block, nv=nv, stream=stream)
                x = torch.zeros_like(b)
                try:
                    ddtm.ddtm_setup(ctx, mu, SEED)
                    ddtm.ddtm_solve(ctx, x, b, NRHS, mu)
                    t_setup, _ = _timed(torch, stream, lambda: ddtm.ddtm_setup(ctx, mu, SEED))
                    t_solve, (info, code) = _timed(torch, stream, lambda: ddtm.ddtm_solve(ctx, x, b, NRHS, mu))
                    runs.append({"block": block, "nv": nv, "setup_s": t_setup, "solve_s": t_solve,
                                 "total_s": t_setup + t_solve, "outer_iters": info.iters,
                                 "coarse_rhs_iters": info.coarse_iters, "max_relres": info.max_relres,
                                 "converged": code == ddtm.OK})
                except ddtm.DDTMError as e:
                    runs.append({"block": block, "nv": nv, "error": str(e)[:200]})
                finally:
                    ddtm.ddtm_destroy(ctx)
                torch.cuda.empty_cache()
        out["runs"] = runs
    print(json.dumps(out))


# ---- our arm ------------------------------------------------------------------------------------
def main():
    args = parse_args()
    if args.oracle_units:
        print(json.dumps(oracle_unit_times(WORKLOADS[args.oracle_units])))
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.study == "oracle":
        oracle_study(args.lattices.split(",") if args.lattices else None)
        return
    if args.study:
        study(args)
        return
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # one process builds (in-tree objects and library are shared by the ranks of a node)
    from paper_1610_02370_gb300 import build as _build
    if local == 0:
        _build.build()
    if dist is not None:
        dist.barrier()
    from paper_1610_02370_gb300 import ddtm, synth

    wl = WORKLOADS[args.workload]
    dims = wl["dims"]
    T, X, Y, Z = dims
    V = T * X * Y * Z
    Vb = int(np.prod(MG["block"]))
    Nc = V // Vb
    stream = torch.cuda.current_stream()

    # measured SIMT arithmetic peaks of this device (FMA throughput, CUDA events), for the ALU rooflines
    f32_peak, _, n_sm = ddtm.ddtm_measure_fma_peak(ddtm.PREC_F32)
    f64_peak, _, _ = ddtm.ddtm_measure_fma_peak(ddtm.PREC_F64)

    ctx = ddtm.ddtm_create(dims, MG["block"], 0)
    ddtm.ddtm_set_stream(ctx, stream.cuda_stream)
    p = ddtm.ddtm_get_params(ctx)
    p.nv[0] = MG["nv"]
    for k in ("n_setup", "post_smooth", "nmr", "outer_restart", "outer_tol", "smoother_prec", "coarse_prec"):
        setattr(p, k, MG[k])
    if wl.get("levels", 2) == 3:
        p.n_levels = 3
        p.nv[1] = wl["nv1"]
        for m in range(4):
            p.block[1][m] = 2
    ddtm.ddtm_set_params(ctx, p)
    twists = wl.get("twists", (1,))
    if len(twists) > 1 or wl.get("levels", 2) == 3:  # the large three-level workload: solver line only
        args.no_fp64 = args.no_oracle_check = args.no_cpu = True

    U = synth.gauge_field(dims, wl["eps"], seed=rank, device="cuda")
    ddtm.ddtm_load_gauge(ctx, U, wl["kappa"], wl["c_sw"])
    b = synth.point_sources(dims, device="cuda")
    x = torch.zeros_like(b)
    mu = wl["mu"]
    info_last = {}

    nstep = [0]

    def step():
        t0 = time.time()
        ddtm.ddtm_setup(ctx, mu, SEED)
        for sgn in twists:  # one setup serves both flavours (+mu and -mu)
            info, code = ddtm.ddtm_solve(ctx, x, b, NRHS, sgn * mu)
            if code != ddtm.OK:
                raise RuntimeError("solve did not converge: " + ddtm.ddtm_last_error(ctx))
            info_last.update(iters=info.iters, restarts=info.restarts, coarse_iters=info.coarse_iters,
                             max_relres=info.max_relres, solve_s=info.solve_s, setup_s=info.setup_s)
            if rank == 0:  # progress on stderr (the JSON line stays alone on stdout)
                sys.stderr.write("[bench] step %d mu %+g: %d outer iterations, %d coarse, relres %.2e, "
                                 "setup %.2f s, solve %.2f s, wall %.1f s\n"
                                 % (nstep[0], sgn * mu, info.iters, info.coarse_iters, info.max_relres,
                                    info.setup_s, info.solve_s, time.time() - t0))
                sys.stderr.flush()
        nstep[0] += 1

    for _ in range(args.warmup):
        step()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- headline: K steps, per-kernel timers off; the library counts its launches meanwhile
    clocks = ClockSampler(local)
    ddtm.ddtm_timer_enable(ctx, False)
    ddtm.ddtm_timer_reset(ctx)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    gpu_launches = ddtm.ddtm_timer_kernel_launches(ctx)  # every library kernel launched in the timed region
    ms = ev0.elapsed_time(ev1)
    t_step = ms / 1000.0 / args.steps
    t_step = max_over_ranks(t_step, dist, "cuda")
    value = t_step / world  # whole job: world propagators per step
    x_timed = x.clone()

    # ---- per-kernel breakdown: one more step of identical work with every launch bracketed by events
    ddtm.ddtm_timer_reset(ctx)
    ddtm.ddtm_timer_enable(ctx, True)
    barrier()
    ei0, ei1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ei0.record(stream)
    step()
    ei1.record(stream)
    barrier()
    ddtm.ddtm_timer_enable(ctx, False)
    counts = ddtm.ddtm_timer_report(ctx)
    instrumented_ms = ei0.elapsed_time(ei1)

    # residual of the timed solutions with the library's FP64 operator (the solver's workspace is
    # released first: on the largest lattices it holds most of the device memory)
    ddtm.ddtm_release_workspace(ctx)
    r = torch.empty_like(x)
    ddtm.ddtm_apply_D(ctx, r, x_timed, NRHS, twists[-1] * mu, ddtm.PREC_F64)
    r = b - r
    relres = float(max((r[i].norm() / b[i].norm()).item() for i in range(NRHS)))
    del r

    # ---- D(mu) stencil on this lattice: 1 rhs per launch (FP16, FP32, FP64) and 12 rhs in one launch
    # (FP16, FP32); inputs far above L2 and L2 flushed between applications
    flush = torch.empty(int(256e6) // 4, dtype=torch.float32, device="cuda")
    dtm = {}
    for prec, tag, nr in ((ddtm.PREC_F16, "f16", 1), (ddtm.PREC_F32, "f32", 1), (ddtm.PREC_F64, "f64", 1),
                          (ddtm.PREC_F16, "f16", NRHS), (ddtm.PREC_F32, "f32", NRHS)):
        fx = ddtm.ddtm_field_create(ctx, prec, nr)
        fy = ddtm.ddtm_field_create(ctx, prec, nr)
        ddtm.ddtm_field_import(ctx, fx, b[:nr].contiguous())
        times = []
        for it in range(13):
            flush.fill_(float(it))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ddtm.ddtm_apply_D_field(ctx, fy, fx, mu)
            e1.record(stream)
            e1.synchronize()
            if it >= 3:
                times.append(e0.elapsed_time(e1))
        tmed = statistics.median(times) / 1000.0
        key = tag if nr == 1 else "%s_%drhs" % (tag, nr)
        nbytes = dslash_bytes(tag, nr) * V
        dtm[key] = {"gbs": nbytes / tmed / 1e9, "ms": tmed * 1e3, "bytes_per_launch": nbytes, "nrhs": nr,
                    "tflops": 1920.0 * V * nr / tmed / 1e12}
        ddtm.ddtm_field_destroy(fx)
        ddtm.ddtm_field_destroy(fy)
    del flush

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_note = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    f32_tf, f64_tf = f32_peak / 1e12, f64_peak / 1e12

    def rhs_per_launch(k):
        v = counts[k]
        return v.get("units", v["launches"]) / v["launches"]

    # algorithmic bytes per launch: stated by the library for the kernels that
    # know their operands (coarse passes, Krylov vectors), modelled here otherwise
    def bytes_per_launch(k):
        v = counts[k]
        if v.get("bytes"):
            return v["bytes"] / v["launches"]
        return algorithmic_bytes(k, V, Vb, MG["block"], MG["nv"], Nc, rhs_per_launch(k))

    def flops_per_launch(k):
        return algorithmic_flops(k, V, Vb, MG["block"], MG["nv"], MG["nmr"], rhs_per_launch(k))

    # dominant kernel of the step and its roofline (durations from the instrumented step)
    kern = sorted(((v["ms"], k) for k, v in counts.items()), reverse=True)
    total_ms = sum(v["ms"] for v in counts.values())
    dom = kern[0][1]
    launches = counts[dom]["launches"]
    avg_s = counts[dom]["ms"] / launches / 1000.0
    nbytes = bytes_per_launch(dom)
    fl = flops_per_launch(dom)
    tr = NCU_TRAFFIC.get(dom)
    traffic = tr["bytes_per_site_rhs"] * (V / 2) * rhs_per_launch(dom) if tr else None
    if fl:
        achieved = fl / avg_s / 1e12
        roofline = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": f32_tf, "unit": "TFLOP/s",
                    "frac": achieved / f32_tf, "traffic": traffic, "traffic_capture": tr["capture"] if tr else None,
                    "share": counts[dom]["ms"] / total_ms, "launches_per_step": launches,
                    "flops_per_launch": fl, "bytes_per_launch": nbytes, "rhs_per_launch": rhs_per_launch(dom),
                    "peak_source": "measured FP32 FMA throughput of this GPU (ddtm_measure_fma_peak, %d SMs)" % n_sm}
    else:
        achieved = nbytes / avg_s / 1e9 if nbytes else None
        roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm if achieved else None, "traffic": traffic,
                    "share": counts[dom]["ms"] / total_ms, "launches_per_step": launches,
                    "bytes_per_launch": nbytes, "peak_source": peak_note}
    roofline["durations"] = "per-launch CUDA events of one instrumented step of the same work after the timed region"
    breakdown = {}
    for k, v in sorted(counts.items(), key=lambda kv: -kv[1]["ms"]):
        nb = bytes_per_launch(k)
        fk = flops_per_launch(k)
        t1 = v["ms"] / v["launches"] / 1000.0
        breakdown[k] = {"ms_per_step": v["ms"], "launches_per_step": v["launches"],
                        "units_per_step": v.get("units", v["launches"]), "share": v["ms"] / total_ms,
                        "gbs": nb / t1 / 1e9 if nb else None, "tflops": fk / t1 / 1e12 if fk else None}

    # end to end through host buffers: gauge upload + setup + solve with pinned host b and x
    e2e = None
    if not args.no_e2e:
        Uh = U.cpu().pin_memory()
        bh = b.cpu().pin_memory()
        xh = torch.zeros_like(bh).pin_memory()
        ts = []
        for _ in range(min(args.steps, 3)):
            barrier()
            t0 = time.perf_counter()
            ddtm.ddtm_load_gauge(ctx, Uh, wl["kappa"], wl["c_sw"])
            ddtm.ddtm_setup(ctx, mu, SEED)
            info, code = ddtm.ddtm_solve(ctx, xh, bh, NRHS, mu)
            barrier()
            ts.append(time.perf_counter() - t0)
        te = max_over_ranks(statistics.median(ts) if ts else float("nan"), dist, "cuda")
        e2e = {"value": te / world, "unit": UNIT, "h2d_bytes_per_step": int(Uh.numel() * 16 + bh.numel() * 16),
               "d2h_bytes_per_step": int(xh.numel() * 16), "steps": len(ts)}
        del Uh, bh, xh

    # the mixed-precision solve driven to 1e-12 (the reference for the solution deviation below)
    x_mix12 = None
    if not args.no_fp64:
        p12 = ddtm.ddtm_get_params(ctx)
        p12.outer_tol = 1e-12
        ddtm.ddtm_set_params(ctx, p12)
        x_mix12 = torch.zeros_like(b)
        ddtm.ddtm_solve(ctx, x_mix12, b, NRHS, mu)
    ddtm.ddtm_destroy(ctx)

    # The plain FP64 method for comparison (FP64 outer FGMRES and SAP smoother, FP32 SIMT coarse
    # operator, one right-hand side per solve): one setup and the 12 point sources solved one after
    # another, all timed.  Then the same method with its 12 solves driven to 1e-12, untimed: the
    # mixed-precision solution at 1e-12 must agree with it within 1e-8.
    fp64 = None
    deviation = None
    if not args.no_fp64:
        c64 = ddtm.ddtm_create(dims, MG["block"], 0)
        ddtm.ddtm_set_stream(c64, stream.cuda_stream)
        p = ddtm.ddtm_get_params(c64)
        p.nv[0] = MG["nv"]
        for k in ("n_setup", "post_smooth", "nmr", "outer_restart", "outer_tol"):
            setattr(p, k, MG[k])
        p.smoother_prec = ddtm.PREC_F64
        p.coarse_prec = ddtm.PREC_F32
        ddtm.ddtm_set_params(c64, p)
        ddtm.ddtm_load_gauge(c64, U, wl["kappa"], wl["c_sw"])
        x64 = torch.zeros_like(b)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(NRHS + 2)]
        iters, relres64, conv = [], [], True
        barrier()
        ev[0].record(stream)
        ddtm.ddtm_setup(c64, mu, SEED)
        ev[1].record(stream)
        for i in range(NRHS):
            info, code = ddtm.ddtm_solve(c64, x64[i], b[i], 1, mu)
            ev[i + 2].record(stream)
            iters.append(info.iters)
            relres64.append(info.max_relres)
            conv = conv and code == ddtm.OK
        barrier()
        t_setup = ev[0].elapsed_time(ev[1]) / 1e3
        t_solves = [ev[i + 1].elapsed_time(ev[i + 2]) / 1e3 for i in range(NRHS)]
        seq = t_setup + sum(t_solves)
        fp64 = {"setup_s": t_setup, "solve_s": t_solves, "iters": iters, "max_relres": max(relres64),
                "converged": conv, "sequential_12_rhs_s": seq,
                "speedup_mixed_batched_vs_fp64_sequential": seq / value,
                "method": "FP64 outer FGMRES and SAP smoother, FP32 SIMT coarse stencil, one rhs per solve; "
                          "setup + the 12 point sources solved one after another, all timed with CUDA events"}
        p.outer_tol = 1e-12
        ddtm.ddtm_set_params(c64, p)
        x64 = torch.zeros_like(b)
        ddtm.ddtm_solve(c64, x64, b, NRHS, mu)  # the 12 sources in one batch of the plain FP64 method
        ddtm.ddtm_destroy(c64)
        dev = [((x_mix12[i] - x64[i]).norm() / x64[i].norm()).item() for i in range(NRHS)]
        deviation = {"max": max(dev), "per_rhs": dev,
                     "method": "mixed-precision batched solve and the plain FP64 method, both to relative "
                               "residual 1e-12; ||x_mixed - x_fp64|| / ||x_fp64|| per point source"}
        del x64, x_mix12

    # the timed solutions' residuals evaluated with the oracle's FP64 D on the host (slabs of t in a
    # pool of spawned processes), independent of the library's operator
    oracle_check = None
    if rank == 0 and not args.no_oracle_check:
        from oracle import slabs
        t0 = time.perf_counter()
        xs = x_timed.cpu().numpy()
        bs = b.cpu().numpy()
        rr = slabs.relative_residuals(U.cpu().numpy(), wl["kappa"], wl["c_sw"], bs, xs, mu, bc_t=0, slab=4,
                                      workers=min(16, host_cores()))
        oracle_check = {"max": max(rr), "per_rhs": rr, "s": time.perf_counter() - t0,
                        "method": "oracle FP64 D (oracle/operators.py) evaluated per t-slab of 4 layers with a "
                                  "halo of 1 (oracle/slabs.py) on the 12 solutions of the last timed step"}
        del xs, bs

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        unit = oracle_unit_times_one_core(args.workload)
        per_step_counts = {k: {"launches": v["launches"], "units": v.get("units", v["launches"])}
                           for k, v in counts.items()}
        est, _ = oracle_estimate(unit, per_step_counts, V, Nc)
        cpu = {"value": est, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
               "extrapolated": True,
               "sample": "oracle building blocks (D, SAP half-sweep, P, Galerkin, R, P, coarse even-odd GMRES "
                         "iteration) timed on a %s lattice with the same couplings and multigrid parameters, scaled "
                         "per site to %s and multiplied by this step's work units (right-hand sides and vectors "
                         "processed per kernel family): an extrapolation, not a timing of the whole workload" % (
                             unit["_sample"], args.workload),
               "unit_s_per_site": {k: v for k, v in unit.items() if not k.startswith("_")}}
        if oracle_check:
            # measured at the workload's full size: the oracle's D on 12 right-hand sides, in parallel slabs
            cpu["measured_full_size"] = {"oracle_D_12rhs_with_site_term_s": oracle_check["s"],
                                         "processes": min(16, host_cores())}
        if not args.no_cpu_all:
            # the same oracle on every host core at once (one single-threaded process per core)
            try:
                unit_all, ncores = oracle_unit_times_all_cores(args.workload)
                est_all, _ = oracle_estimate(unit_all, per_step_counts, V, Nc)
                cpu["all_cores"] = {"value": est_all, "unit": UNIT, "cores": ncores,
                                    "method": "one single-threaded oracle process per host core, all timing the "
                                              "same sample at once; seconds per unit = their mean / cores"}
            except (RuntimeError, OSError, ValueError, IndexError, KeyError) as e:
                cpu["all_cores"] = {"value": None, "error": str(e)[:300]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 outer; f32 arithmetic; f16 storage (smoother fields, coarse tensor-core "
                                          "operands)", "data": "synthetic",
            "config": {"workload": "%s twisted-mass clover propagator, 12 point sources, %s-level DD-alpha-AMG%s"
                                   % (args.workload, "three" if wl.get("levels", 2) == 3 else "two",
                                      ", solved for +mu and -mu after one setup (value: setup + both solves)"
                                      if len(twists) > 1 else ""), "dims_TXYZ": list(dims), **{k: wl[k] for k in wl if k != "dims"},
                       "mg": MG, "nrhs": NRHS, "l2": "working set (test vectors, P, D_c) far above L2",
                       "parallelism": "replicas" if world > 1 else "1 GPU",
                       "timers": "off in the timed region; per-kernel shares from one extra instrumented step"},
            "step": {"setup_s": info_last.get("setup_s"), "solve_s": info_last.get("solve_s"),
                     "outer_iters_max": info_last.get("iters"), "coarse_iters": info_last.get("coarse_iters"),
                     "max_relres": relres, "instrumented_step_ms": instrumented_ms},
            "oracle_relres_max": oracle_check["max"] if oracle_check else None,
            "oracle_relres": oracle_check,
            "solution_deviation_max": deviation["max"] if deviation else None,
            "solution_deviation": deviation,
            "dtm_apply": {"bound": "hbm", "peak": hbm, "unit": "GB/s",
                          "alu_peak_tflops": {"f32": f32_tf, "f64": f64_tf},
                          **{k: {"achieved": v["gbs"], "frac": v["gbs"] / hbm, "ms": v["ms"], "nrhs": v["nrhs"],
                                 "bytes_per_launch": v["bytes_per_launch"], "tflops": v["tflops"],
                                 "alu_frac": v["tflops"] / (f64_tf if k == "f64" else f32_tf)}
                             for k, v in dtm.items()}},
            "peaks": {"f32_fma_tflops": f32_tf, "f64_fma_tflops": f64_tf, "sm_count": n_sm, "hbm_gbs": hbm,
                      "hbm_source": peak_note},
            "roofline": roofline,
            "kernels": breakdown,
            "gpu_launches": gpu_launches,
            "clocks": clk,
            "e2e": e2e,
            "fp64_reference": fp64,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
