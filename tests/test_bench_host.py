"""Host-side logic of bench.py (no GPU): clock parsing, the roofline record,
the traffic figures tied to the kernel sources, the quality settings."""
import json
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_parses_nvidia_smi_lines():
    c = bench.ClockSampler(0)
    c.proc = _FakeProc()
    c.lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    out = c.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["source"] == "nvidia-smi"


def test_roofline_record(monkeypatch):
    monkeypatch.setattr(bench, "sm_count", lambda: 152)   # no device here: the GB300's SM count
    tr = types.SimpleNamespace(n=1000, H=720, W=1280)
    st = {"render_backward": 0.1, "project_gaussians": 0.04, "render_sampled": 0.05}
    info = {"evals_per_step": 1.0e6, "visible": 500, "touched": 200, "n_isect": 5000, "P": 61200}
    peaks = {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0}
    clocks = {"sm_mhz": 2000.0}
    r = bench.roofline(st, info, peaks, "measured", clocks, tr)
    assert r["kernel"] == "render_backward" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    alu = 152 * 128 * 2 * 2000.0e6 / 1e12
    assert r["peak"] == pytest.approx(alu)
    assert r["achieved"] == pytest.approx(1.0e6 * bench.FLOPS_BWD / 1e12 / 1e-4)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    info.update(walked_per_step=2.5e6, maybe_stopped=0.01)
    f = bench.roofline(st, info, peaks, "measured", clocks, tr, dom="render_sampled")
    # an alpha test per position walked, a blend per position up to n_last
    assert f["achieved"] == pytest.approx((2.5e6 * bench.FLOPS_ALPHA + 1.0e6 * bench.FLOPS_BLEND) / 1e12 / 0.05e-3)
    p = bench.roofline(st, info, peaks, "measured", clocks, tr, dom="project_gaussians")
    assert p["bound"] == "hbm" and p["unit"] == "GB/s" and p["peak"] == 6000.0
    byts = tr.n * (44 + 48) + info["visible"] * 192
    assert p["achieved"] == pytest.approx(byts / 0.04e-3 / 1e9)
    assert p["frac"] == pytest.approx(p["achieved"] / 6000.0)


def test_traffic_figures_follow_their_sources(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    rel = os.path.relpath(src, bench.ROOT)
    rec = {"s": {"kernel": "k", "bytes_per_launch": 123.0, "sources": [rel],
                 "sources_sha256": bench.source_digest([rel])}}
    tf = tmp_path / "traffic.json"
    tf.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tf))
    assert bench.measured_traffic("s") == 123.0
    assert bench.measured_traffic("other") is None
    src.write_text("kernel v2")          # the kernel changed since the counters were taken
    assert bench.measured_traffic("s") is None


def test_quality_settings_unique():
    args = types.SimpleNamespace(fraction=1.0, rate=0.1)
    s = bench.quality_settings(args)
    assert s == [(1.0, 0.1), (1.0, bench.PIXEL_RATE), (0.5, 0.1)]
    args = types.SimpleNamespace(fraction=0.2, rate=bench.PIXEL_RATE)
    assert len(bench.quality_settings(args)) == 4


def _replica_rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r timed its 10 steps in 20 + 5 r ms: the job is bound by the slowest
    v = bench.replica_throughput(20.0 + 5.0 * rank, 10, world, dist)
    out[rank] = v
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    """The N > 1 path of the bench (independent replicas, max over ranks) on
    two CPU processes."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_replica_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    want = 2 * 10 / (25.0e-3)
    assert out[0] == pytest.approx(want) and out[1] == pytest.approx(want)
    assert bench.replica_throughput(20.0, 10, 1) == pytest.approx(10 / 20e-3)
