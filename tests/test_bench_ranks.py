"""Host logic of bench.py, on CPU: on the N > 1 path, replicas on two gloo
ranks combine their timings as the slowest rank's time and the sum of their
work, and the reference arm runs on rank 0 only; the ncu traffic table is
well formed and goes stale (None) when a kernel's source changes."""
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
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0, 14.0][rank]
    work = [100.0, 250.0][rank]
    e2e = [12.0, 11.0][rank]
    out = bench.combine_ranks(dist, torch, torch.device("cpu"), ms, work, e2e)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_replicas_combine_max_time_and_summed_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert res[r] == (14.0, 350.0, 12.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


@pytest.mark.parametrize("table", ["traffic.txt", "issue.txt"])
def test_ncu_table_rows_and_staleness(tmp_path, monkeypatch, table):
    """profiles/traffic.txt (DRAM bytes) and profiles/issue.txt (warp
    instructions): every row names a kernel class of the library, a per-site
    unit and an existing source file; bench.table_per_launch scales the
    per-site value to a launch while the source is unchanged and reports None
    once the file's hash differs from the one captured."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2407_08092_gb300 import build
    build.build()   # the class names come from the library (a no-op when it is up to date)
    from paper_2407_08092_gb300 import lqdd
    classes = {lqdd.lq_kernel_class_name(c) for c in range(lqdd.LQ_K_COUNT)}
    rows = [ln.split() for ln in open(os.path.join(ROOT, "profiles", table)) if ln.strip() and ln[0] != "#"]
    assert rows
    for name, per_unit, unit, src, digest in rows:
        assert name in classes, name
        assert unit in ("V", "Vh") and float(per_unit) > 0 and len(digest) == 16
        assert os.path.exists(os.path.join(ROOT, "paper_2407_08092_gb300", "csrc", src))
    # the live table: bytes per launch proportional to the sites (None when stale)
    name, per_unit, unit, src, _ = rows[0]
    got = bench.table_per_launch(table, name, 2 * 1024)
    if got is not None:
        assert got == pytest.approx(float(per_unit) * (2048 if unit == "V" else 1024))
    # a copy of the tree whose source file no longer matches: None
    fake = tmp_path / "root"
    (fake / "profiles").mkdir(parents=True)
    (fake / "paper_2407_08092_gb300" / "csrc").mkdir(parents=True)
    (fake / "profiles" / table).write_text(f"{name} {per_unit} {unit} {src} 0123456789abcdef\n")
    (fake / "paper_2407_08092_gb300" / "csrc" / src).write_text("// changed\n")
    monkeypatch.setattr(bench, "ROOT", str(fake))
    assert bench.table_per_launch(table, name, 2048) is None
