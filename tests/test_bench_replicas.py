"""Host logic of the multi-GPU (replica) benchmark path, on CPU with gloo.

With N > 1 every rank solves its own propagator (the method's units are whole
propagators, so the path shards without a data-path collective); the only
communication is the max over ranks of the step time, and only rank 0 prints.
"""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.max_over_ranks(1.5 + rank, dist, "cpu")))
    finally:
        dist.destroy_process_group()


def test_step_time_is_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == {0: 2.5, 1: 2.5}


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25


def test_reference_arm_only_rank0_prints():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


@pytest.mark.slow
def test_reference_arm_line_rank0():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1


def test_host_cpu_record_x86_and_arm(monkeypatch):
    """The CPU baseline's host record reads the model name on x86 hosts and the CPU part on Arm hosts
    (whose /proc/cpuinfo has no model name), and never fails."""
    import builtins
    import io

    sys.path.insert(0, ROOT)
    import bench

    real_open = builtins.open
    samples = {"x86": "processor\t: 0\nmodel name\t: Some CPU @ 2.0GHz\n",
               "arm": "processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\nCPU part\t: 0xd4f\n"}
    for kind, text in samples.items():
        def fake_open(path, *a, text=text, **k):
            if path == "/proc/cpuinfo":
                return io.StringIO(text)
            return real_open(path, *a, **k)
        monkeypatch.setattr(builtins, "open", fake_open)
        rec = bench.host_cpu()
        assert rec["nproc"] == os.cpu_count()
        assert rec["cpu_model"] == ("Some CPU @ 2.0GHz" if kind == "x86" else "CPU part 0xd4f")

    def no_file(path, *a, **k):
        if path == "/proc/cpuinfo":
            raise OSError("no such file")
        return real_open(path, *a, **k)
    monkeypatch.setattr(builtins, "open", no_file)
    assert bench.host_cpu()["cpu_model"]


def test_oracle_estimate_bookkeeping():
    """The CPU estimate multiplies each kernel family's work units of a GPU step by the oracle's time per
    unit: with every unit time 1 it is the sum of the families' units (per site for the fine kernels, per
    coarse site for the coarse iterations), and the coarse rhs-iterations are the tensor-core passes."""
    import bench
    counts = bench.REFERENCE_COUNTS
    unit = {k: 1.0 for k in ("dslash", "sap_half", "build_P", "galerkin", "restrict", "prolong", "coarse_iter")}
    V, Nc = 1000.0, 10.0
    t, iters = bench.oracle_estimate(unit, counts, V, Nc)
    assert iters == counts["coarse_tc_hop_even"]["units"]
    fine_units = (counts["dslash_f32"]["units"] + counts["dslash_f64"]["units"] + counts["sap_half_f16"]["units"]
                  + counts["build_P"]["launches"] + counts["galerkin"]["launches"]
                  + counts["restrict_f16"]["units"] + counts["prolong_f16"]["units"])
    assert t == fine_units * V + iters * Nc
    # each family scales with its own unit time only
    t2, _ = bench.oracle_estimate(dict(unit, galerkin=3.0), counts, V, Nc)
    assert t2 - t == 2.0 * counts["galerkin"]["launches"] * V


def test_oracle_study_times_the_plain_method_on_4x4x4x4():
    """bench.py --study oracle (direct timings of the oracle, no GPU): on the 4^4 parameter set the
    operator build, one D(mu) application, one SAP cycle and the plain FP64 GMRES solve are timed,
    and the solve reaches relative residual 1e-10."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--study", "oracle", "--lattices", "4x4x4x4"],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["study"] == "oracle" and [row["lattice"] for row in out["rows"]] == ["4x4x4x4"]
    row = out["rows"][0]
    for k in ("operator_build_s", "apply_D_s", "sap_cycle_s", "gmres_solve_s"):
        assert row[k] > 0, k
    assert row["gmres_relres"] <= 1e-10 and row["sites"] == 256
