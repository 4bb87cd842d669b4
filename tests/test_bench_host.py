"""Host logic of bench.py without a GPU: the slowest-rank reduction under torch.distributed
(two gloo ranks on CPU), the reference arm's JSON line, and the clock-sample summary."""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.init_dist(world, "gloo")
    t = bench.reduce_max(1.5 + rank, world)
    bench.barrier(world)
    out.put((rank, t))
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 2.5, 1: 2.5}


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_clock_summary_flags_throttle_reasons():
    sys.path.insert(0, ROOT)
    import bench
    cs = bench.ClockSampler(0)
    cs.rows = [["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Active"],
               ["0", "1980", "2070", "950", "0x4", "Not Active", "Active", "Not Active", "Not Active"],
               ["0", "2010", "2070", "940", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = cs.summary()
    assert s["sm_mhz"] == 2010 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_recorded_traffic_only_for_the_sources_it_was_measured_on(tmp_path, monkeypatch):
    """The roofline's `traffic` comes from the committed ncu summary only while the kernel
    sources hash to the value recorded with it; otherwise it is reported as null."""
    sys.path.insert(0, ROOT)
    import bench
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"c2/f32": {"bytes_per_launch": 304.7e6, "source_hash": "abc"},
         "c3/f32": {"bytes_per_launch": 2797e6, "source_hash": "old"}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.recorded_traffic("c2", "f32") == pytest.approx(304.7e6)
    assert bench.recorded_traffic("c3", "f32") is None        # measured on other sources
    assert bench.recorded_traffic("c2", "f16") is None        # never measured


def test_committed_traffic_entries_are_well_formed():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    for key in ("c2/f32", "c3/f32"):
        e = d[key]
        assert e["bytes_per_launch"] > 0 and len(e["source_hash"]) == 16
        assert sum(e["kernels"].values()) == pytest.approx(e["bytes_per_launch"], rel=1e-3)
