"""Host logic of the multi-GPU path (replicas: the method's blocks and solves
shard into independent problems, so N GPUs run N copies with no data-path
collective).  Two gloo ranks on the CPU check the max-over-ranks timing, the
whole-job throughput, and that only rank 0 of the reference arm prints."""

import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res == {0: 15.0, 1: 15.0}


def test_replica_throughput_and_single_rank():
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.replica_throughput(4, 1000.0, 2.0) == 2000.0


def test_reference_arm_other_ranks_print_nothing():
    import bench

    class A:
        steps, warmup, config, ref_pairs = 1, 0, "headline", 1

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A(), rank=1, world=2)
    assert buf.getvalue() == ""


def test_reference_arm_line_on_cpu():
    """Rank 0 of the reference arm (the FP64 oracle on the host cores) prints
    one JSON line with the keys the measurement contract names."""
    import json

    import bench

    class A:
        steps, warmup, config, ref_pairs = 1, 0, "headline", 1

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A(), rank=0, world=1)
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ["impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"]:
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "entries/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_adjoint_traffic_model():
    """The layer-fused adjoint's traffic model, counted by hand for a
    three-stage net at 32x32 (E_s = (32 / 2^s)^4, widths 32, 16, 8):
    stage 0: forward 5 passes (input covariance write, two read+write) and
    the pool's read; reverse 2 + 3 + 3 (the last layer reads the pooled
    gradient of stage 1 instead of a stage-0 tensor), q-term partials
    3 x 4 E0 / 32, input adjoints 2 -> 16 E0 + 12 E0 / 32;
    stage 1: pool write, 3 x 2 forward, the next pool's read, reverse
    3 + 3 + 2 and stage 0's pooled-gradient read, partials 3 x 4 E1 / 16 ->
    17 E1 + 12 E1 / 16;  stage 2: pool write, 3 x 2 forward, the readout's
    read, reverse 2 (readout constant) + 3 + 3 and stage 1's pooled-gradient
    read, partials 3 x 4 E2 / 8 -> 17 E2 + 12 E2 / 8."""
    import bench

    E0, E1, E2 = 32 ** 4, 16 ** 4, 8 ** 4
    b = bench.adjoint_layerwise_bytes((3, 3, 3), 32)
    assert b == 4 * (16 * E0 + 12 * E0 // 32 + 17 * E1 + 12 * E1 // 16 + 17 * E2 + 12 * E2 // 8)
    # a single-stage net: input covariance write, readout read, one reverse
    # pass (constant gradient) with its partials, two input adjoints
    assert bench.adjoint_layerwise_bytes((1,), 8) == 4 * ((1 + 1 + 2 + 2) * 8 ** 4 + 4 * 8 ** 4 // 8)
    # one image set without a gradient: one read of the input-covariance
    # gradient instead of two
    b1 = bench.adjoint_layerwise_bytes((3, 3, 3), 32, input_sides=1)
    assert b - b1 == 4 * E0
    r = bench.adjoint_roofline(2.0, 1000, 300, {"hbm_gbs": 5000.0})
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - (b * 1000 + b1 * 300) / 2.0 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 5000.0) < 1e-12


def test_cpu_baseline_line():
    import bench

    d = bench.cpu_baseline_line(160.0, 320, 2.0, 16, 20, 3146752)
    assert d["value"] == 160.0 and d["unit"] == "entries/s" and d["cores"] == 16 and d["kind"] == "oracle"
    assert d["per_core"] == 10.0 and abs(d["workload_extrapolated_s"] - 3146752 / 160.0) < 1e-9
    assert "320 Myrtle-5 32x32" in d["sample"] and "2.0 s" in d["sample"]


def test_headline_traffic_record():
    """The recorded DRAM traffic of the headline's tiled launches is reported
    only for that kernel and workload, and only while the kernel's sources
    hash as they did at the capture."""
    import bench

    v, note = bench.headline_traffic("headline", 3)
    assert (v is None and "changed" in note) or (v > 0 and "ncu" in note)
    assert bench.headline_traffic("small", 3)[0] is None
    assert bench.headline_traffic("headline", 0)[0] is None
