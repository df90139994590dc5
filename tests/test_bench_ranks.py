"""Host logic of bench.py on the CPU: the multi-replica timing on gloo ranks
(world size 2: every rank sees the slowest replica's time, and the job rate
counts all replicas' units over it), the reference arm's JSON line, and the
parsing of the clocks sampled during the timed region."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mine = 1.5 + rank  # rank 1 is the slow replica
    t = bench.max_over_ranks(mine, dist, "cpu")
    q.put((rank, t, bench.job_rate(100, t, ws), bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    ps = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate, env in out:
        assert t == 2.5
        assert rate == pytest.approx(2 * 100 / 2.5)
        assert env == (2, rank, rank)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.job_rate(10, 2.0, 1) == 5.0


def test_reference_arm_line_on_cpu():
    """The reference arm (the oracle on the host) prints one JSON line with the
    contract's keys; a rank other than 0 exits without work."""
    import json
    import subprocess
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "20000",
           "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out1 = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert out1.returncode == 0 and out1.stdout.strip() == ""


def test_clock_sampler_parses_a_fake_nvidia_smi(tmp_path, monkeypatch):
    """The clocks record of the bench line: median SM clock, the highest
    maximum, and every throttle reason seen Active, read from nvidia-smi's CSV
    (a stand-in script on PATH; unparsable lines are skipped)."""
    sys.path.insert(0, ROOT)
    import bench
    lines = [
        "0, 1900, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1950, 2070, 1100.4, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1200.0, 0x8, Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    (tmp_path / "out.csv").write_text("\n".join(lines) + "\n")
    fake = tmp_path / "nvidia-smi"
    fake.write_text(f"#!/bin/sh\ncat '{tmp_path / 'out.csv'}'\nexec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    cs = bench.ClockSampler(0)
    cs.start()
    import time
    time.sleep(0.5)
    rec = cs.stop()
    assert rec == {"sm_mhz": 1950.0, "sm_max_mhz": 2070.0,
                   "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 3}


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))
    cs = bench.ClockSampler(0)
    cs.start()
    assert cs.stop() is None


def test_algorithmic_bytes_per_unit():
    """The bytes each kernel group must move, per the units it processes:
    per point, per leaf, per cell of the pyramid and per non-zero of P."""
    sys.path.insert(0, ROOT)
    import bench
    n, nnz, L = 1000, 90_000, 4
    leaves, cells = 4 ** L, sum(4 ** l for l in range(L + 1))
    b = bench.group_bytes(n, nnz, L)
    assert b["k_update"] == 72 * n
    assert b["k_snap_hist"] == 44 * n + 20 * min(n, leaves)
    assert b["k_pyr_pass"] == 24 * leaves + 20 * cells + 20 * min(n, leaves)
    b2 = bench.group_bytes(n, nnz, L, 100, 60)
    assert b2["k_pyr_pass"] == 24 * leaves + 4 * cells + 16 * 100 + 20 * 60
    assert b2["k_snap_hist"] == 44 * n + 20 * 60
    assert b["k_perm_scatter"] == 20 * n
    assert b["k_bh_traverse"] == 24 * n + 20 * cells
    assert b["k_attract"] == 8 * nnz + 8 * (n + 1) + 20 * n
    assert b["k_zsum"] == 4 * n
    assert b["k_relabel"] == (16 * nnz + 56 * n) / bench.RELABEL_EVERY
