"""CPU tests of the benchmark's multi-rank path: replicas on 2 gloo ranks
reduce their timings to the maximum, and the whole-job rate counts every
rank's units over that time; the reference arm runs on rank 0 only."""
import importlib.util
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    b = _bench()
    t, e = b.max_over_ranks([1.0 + rank, 5.0 - rank], dist, "cpu")
    q.put((rank, t, e, b.job_throughput(8 * 3, ws, t)))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, e, v in out:
        assert t == 2.0 and e == 5.0          # slowest rank's time on every rank
        assert v == 8 * 3 * 2 / 2.0            # both ranks' layers over that time


def test_single_process_identity():
    b = _bench()
    assert b.max_over_ranks([0.25, 3.0], None, "cpu") == [0.25, 3.0]
    assert b.job_throughput(16, 1, 0.5) == 32.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup = 2, 1, 0
    assert b.run_reference(A()) == 0
    assert capsys.readouterr().out == ""


def test_traffic_record_follows_kernel_sources(tmp_path, monkeypatch):
    """A DRAM-traffic record is scaled to a launch only while its source hash
    matches the reverse-pass sources; an edit to any of them, an unknown
    kernel or a missing record reports no traffic rather than a stale
    figure.  Checked on a copy of the sources, with a record written for it."""
    import json
    b = _bench()
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for k in ("rev_mid_tma_kernel", "rev_pass_kernel", "rev_pass_half_kernel", "final_pass_half_kernel"):
        assert 0.9 < d[k]["dram_bytes"] / d[k]["alg_bytes"] < 1.1
    root = tmp_path / "repo"
    src = root / "paper_2606_26297_b300" / "csrc"
    src.mkdir(parents=True)
    for name in ("kernels_adjoint.cu", "kernels_rev_half.cu", "pass_half.cuh", "pass_body.cuh", "pass_common.cuh",
                 "tma_util.cuh", "qaoa_internal.h"):
        (src / name).write_bytes(open(os.path.join(ROOT, "paper_2606_26297_b300", "csrc", name), "rb").read())
    monkeypatch.setattr(b, "ROOT", str(root))
    assert b._traffic("rev_pass_kernel", 1000.0) is None  # no record
    (root / "profiles").mkdir()
    rec = {"rev_pass_kernel": {"dram_bytes": 980.0, "alg_bytes": 1000, "source_hash": b._kernel_source_hash()}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert b._traffic("rev_pass_kernel", 5000.0) == pytest.approx(4900.0)
    assert b._traffic("no_such_kernel", 5000.0) is None
    (src / "pass_half.cuh").write_bytes((src / "pass_half.cuh").read_bytes() + b"\n")
    assert b._traffic("rev_pass_kernel", 5000.0) is None
