"""Host logic of bench.py without a GPU: the roofline arithmetic on given kernel statistics, the
source check that retires a stale DRAM-traffic figure, and the multi-rank timing of the replicas
mode (every rank solves its own system; the job's step time is the maximum over ranks) with two
gloo ranks on the CPU."""
import hashlib
import math
import multiprocessing as mp
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6785.9}
PIPES = bench.pipe_peaks({"fp64_tflops": 1.25, "fp32_tflops": 78.3})


def _stats():
    # five factor kernels in the order k_pivot, k_panel, k_schur, k_compress, k_redirect
    return {"kernel_ms": [100.0, 50.0, 180.0, 250.0, 40.0], "kernel_launches": [54, 54, 54, 54, 54],
            "kernel_flops": [1e11, 2e11, 3.9e11, 1.6e11, 5e10], "schur_bytes": 1.0e11,
            "compress_proj_flops": 1.2e11, "compress_reorth_flops": 1.0e10}


def test_pipe_peaks_derive_the_double_float_rate_from_the_fp32_rate():
    assert PIPES["dfl"] == 78.3 / 11.0 and PIPES["fp64"] == 1.25 and PIPES["source"].startswith("measured")
    nominal = bench.pipe_peaks(None)
    assert nominal["source"].startswith("nominal") and math.isclose(nominal["fp32"], 152 * 128 * 2 * 2.07e-3)


def test_roofline_picks_the_dominant_kernel_and_divides_by_its_own_peak():
    rf = bench.roofline(_stats(), "mixed_solve", PEAKS, "measured", PIPES)
    assert rf["kernel"] == "k_compress"
    t = 250.0 / 54 / 1000.0
    assert math.isclose(rf["achieved"], 1.6e11 / 54 / t / 1e12, rel_tol=1e-12)
    # two pipes: the projection (1.2e11 flops) and the Gram-Schmidt column work (3e10) in
    # double-float, the re-orthogonalisation (1e10) in FP64; the peak is the rate of that mix with
    # each part at its own pipe's peak
    t_ideal = 1.5e11 / 54 / (PIPES["dfl"] * 1e12) + 0.1e11 / 54 / (PIPES["fp64"] * 1e12)
    assert math.isclose(rf["peak"], 1.6e11 / 54 / t_ideal / 1e12, rel_tol=1e-12)
    assert math.isclose(rf["frac"], rf["achieved"] / rf["peak"])
    assert math.isclose(rf["projection_share_of_flops"], 0.75)
    sc = rf["schur"]
    assert sc["kernel"] == "k_schur" and sc["peak"] == PIPES["dfl"]
    ai = 3.9e11 / 1.0e11
    assert math.isclose(sc["intensity_flop_per_byte"], ai)
    assert math.isclose(sc["attainable"], min(PIPES["dfl"], ai * PEAKS["hbm_gbs"] / 1000.0))
    assert math.isclose(sc["frac_attainable"], sc["achieved"] / sc["attainable"])
    assert math.isclose(sc["algorithmic_gbs"], 1.0e11 / 54 / (180.0 / 54 / 1000.0) / 1e9)
    # no capture of the current sources: no traffic
    assert rf["traffic"] is None and rf["achieved_dram_gbs"] is None


def test_roofline_in_fp64_uses_the_fp64_peak_everywhere():
    rf = bench.roofline(_stats(), "fp64", PEAKS, "measured", PIPES)
    assert rf["peak"] == PIPES["fp64"] and rf["schur"]["peak"] == PIPES["fp64"]
    # the Schur update's ridge lies above the FP64 peak, so the attainable roofline is that peak
    assert rf["schur"]["attainable"] == PIPES["fp64"]


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    """A bounded capture's DRAM bytes per eliminated box, times the boxes of an average launch, while
    the kernel sources hash as they did when it was taken; null once a source differs."""
    csrc = os.path.join(ROOT, "paper_1407_1572_gb300", "csrc")
    files = ["ifmm_factor.cu", "ifmm_common.cuh"]
    now = {f: hashlib.sha256(open(os.path.join(csrc, f), "rb").read()).hexdigest() for f in files}
    monkeypatch.setattr(bench, "TRAFFIC_SRC", now)
    monkeypatch.setattr(bench, "TRAFFIC", {("mixed_solve", "k_compress"): {"bytes_per_box": 3.0e6}})
    assert bench._traffic("mixed_solve", "k_compress", 400.0) == 1.2e9
    assert bench._traffic("fp64", "k_compress", 400.0) is None
    # through the roofline: 54 launches over 21,840 boxes
    rf = bench.roofline(_stats(), "mixed_solve", PEAKS, "measured", PIPES, boxes=21840)
    assert math.isclose(rf["traffic"], 3.0e6 * 21840 / 54)
    assert math.isclose(rf["achieved_dram_gbs"], rf["traffic"] / (250.0 / 54 / 1000.0) / 1e9)
    monkeypatch.setattr(bench, "TRAFFIC_SRC", {f: "0" * 64 for f in files})
    assert bench._traffic("mixed_solve", "k_compress", 400.0) is None


def test_replica_seeds_differ_per_rank_and_the_value_counts_every_rank():
    assert len({bench.replica_seed(1411, r) for r in range(8)}) == 8
    assert math.isclose(bench.whole_job_value(4, 1 << 20, 2000.0), 4 * (1 << 20) / 2.0)
    assert bench.reduce_max_ms(12.5, None, "cpu") == 12.5


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = bench.reduce_max_ms(10.0 + 5.0 * rank, dist, "cpu")
        q.put((rank, ms, bench.whole_job_value(world, 4096, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_step_time():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    assert all(math.isclose(o[2], 2 * 4096 / 0.015) for o in out)


def test_oracle_step_reports_its_phases_and_the_host_cpu():
    w = dict(bench.CPU_SAMPLE, N=1024, depth=2, nrhs=2)
    parts = {}
    dt, err = bench.oracle_step(w, threads=1, parts=parts)
    assert err < 1e-6 and set(parts) == {"t_build_s", "t_factor_s", "t_solve_s", "gmres_iters"}
    assert parts["gmres_iters"] >= 1
    assert math.isclose(parts["t_factor_s"] + parts["t_solve_s"], dt, rel_tol=1e-9)
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()


def test_partition_of_independent_systems_is_complete_and_balanced():
    import random
    rng = random.Random(5)
    work = [rng.randint(2048, 32768) * rng.randint(1, 16) for _ in range(256)]
    assert bench.partition_work(work, 1) == [list(range(256))]     # one rank: every system, in order
    for world in (2, 3, 4, 8):
        parts = bench.partition_work(work, world)
        assert sorted(i for p in parts for i in p) == list(range(256))
        loads = [sum(work[i] for i in p) for p in parts]
        # largest-first greedy: no rank exceeds the least loaded by more than the largest system
        assert max(loads) - min(loads) <= max(work)
        assert bench.partition_work(work, world) == parts            # deterministic


def _batched_rank(rank, world, port, q):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank 0: fast, shallow trees; rank 1: slow, a larger error and deeper trees
        res = bench.aggregate_batched(1.0 + rank, 0.5 + 2 * rank, 1e-8 * (1 + 9 * rank), 3 + rank, 5 + 2 * rank,
                                      dist, "cpu")
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_batched_results_combine_over_two_gloo_ranks():
    assert bench.aggregate_batched(1.0, 2.0, 1e-8, 3, 7, None, "cpu") == (3.0, 1.0, 2.0, 1e-8, 3, 7)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_batched_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, (t, tf, ts, err, dmin, dmax) in out:
        assert (t, tf, ts, dmin, dmax) == (4.5, 2.0, 2.5, 3.0, 7.0)   # slowest rank: 2.0 + 2.5
        assert math.isclose(err, 1e-7)


def test_roofline_reports_every_factor_kernel_against_its_own_peak():
    rf = bench.roofline(_stats(), "mixed_solve", PEAKS, "measured", PIPES)
    fk = rf["factor_kernels"]
    assert list(fk) == ["k_pivot", "k_panel", "k_schur", "k_compress", "k_redirect"]
    st = _stats()
    for i, (name, k) in enumerate(fk.items()):
        t = st["kernel_ms"][i] / 54 / 1000.0
        assert math.isclose(k["achieved"], st["kernel_flops"][i] / 54 / t / 1e12, rel_tol=1e-12)
        assert math.isclose(k["frac"], k["achieved"] / k["peak"], rel_tol=1e-12)
    # pivots in FP64, the products in double-float, the compression on its blend
    assert fk["k_pivot"]["peak"] == PIPES["fp64"]
    assert fk["k_panel"]["peak"] == PIPES["dfl"] and fk["k_redirect"]["peak"] == PIPES["dfl"]
    assert PIPES["fp64"] < fk["k_compress"]["peak"] < PIPES["dfl"]
    assert math.isclose(sum(k["share_of_factor_kernels"] for k in fk.values()), 1.0)
