"""Multi-rank bench logic on CPU with gloo (world size 2): replicas with no
data-path collective, max-over-ranks timing and whole-job throughput; the
reference arm prints on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=2)
    ms = [10.0, 12.5][rank]          # rank 1 is the slower replica
    e2e = [2.0, 1.5][rank]
    out = bench.aggregate(ms, e2e, steps=100, e2e_steps=50, ws=2)
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_takes_the_slowest_rank():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, e2e_s, value, e2e_value = res[r]
        assert ms == 12.5 and e2e_s == 2.0
        assert value == pytest.approx(2 * 100 / 12.5e-3)
        assert e2e_value == pytest.approx(2 * 50 / 2.0)


def test_single_rank_aggregate_is_local():
    sys.path.insert(0, ROOT)
    import bench
    ms, e2e_s, value, e2e_value = bench.aggregate(4.0, 1.0, 10, 5, 1)
    assert (ms, e2e_s) == (4.0, 1.0) and value == pytest.approx(2500.0) and e2e_value == 5.0


def test_reference_arm_silent_on_other_ranks(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        workload, steps, warmup = "qbd_L64_m8", 3, 3
    bench.run_reference(A())
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank0(monkeypatch, capsys):
    """The reference arm (the oracle on the host cores) prints the contract's
    JSON line on rank 0: impl, metric, unit, the timing keys, cpu_baseline and
    an e2e with zero transfer bytes."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")

    class A:
        workload, steps, warmup, dtype = "qbd_L64_m8", 3, 1, "f64"
    bench.run_reference(A())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == "qbd_L64_m8"


def test_clock_sampler_reports_median_clock_and_throttle_reasons(tmp_path, monkeypatch):
    """The clock record of the bench line: median SM clock under load, the
    maximum, and every throttle reason that was active in any sample (a fake
    nvidia-smi on PATH stands in for the GPU machine's)."""
    import time
    sys.path.insert(0, ROOT)
    import bench
    fake = tmp_path / "nvidia-smi"
    argf = tmp_path / "args"
    fake.write_text("#!/bin/sh\n"
                    f"echo \"$@\" > {argf}\n"
                    "echo '2070, 2070, 500.1, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '1980, 2070, 610.5, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "echo '2070, 2070, 590.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ.get('PATH', '')}")
    # the timed GPU is named by UUID: nvidia-smi's own indices ignore
    # CUDA_VISIBLE_DEVICES, so ordinal 0 of this process may be another GPU
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "GPU-1234abcd-0000-1111-2222-333344445555")
    sel = bench.gpu_id(0)
    assert sel == "GPU-1234abcd-0000-1111-2222-333344445555"
    s = bench.ClockSampler(sel)
    s.start()
    for _ in range(100):
        if len(s.rows) >= 3:
            break
        time.sleep(0.05)
    out = s.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    assert out["power_w_max"] == 610.5
    assert out["gpu"] == sel
    assert argf.read_text().split()[:2] == ["-i", sel]
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "3,5")
    assert bench.gpu_id(1) == "5"
