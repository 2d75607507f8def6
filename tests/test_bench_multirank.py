"""bench.py host logic: the multi-rank timing rule on CPU ranks (gloo, world
size 2: every rank reports the slowest rank's time, a single process is
unaffected) and the reference arm's JSON line and rank handling."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    q.put((rank, bench.max_over_ranks(10.0 + 5.0 * rank, device="cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(3.25, device="cpu") == 3.25


def _reference_line(monkeypatch, capsys, env):
    import json

    import bench
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    calls = []

    def fake_sample(n, inner):
        calls.append((n, inner))
        return 1000, 0.5, 3

    monkeypatch.setattr(bench, "oracle_sample", fake_sample)
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"])
    assert bench.main() == 0
    out = capsys.readouterr().out.strip()
    return (json.loads(out) if out else None), calls


def test_reference_arm_line(monkeypatch, capsys):
    """The reference arm's JSON line (the oracle timed on the host, here with
    its sample replaced by a fixed 1000 unknowns in 0.5 s): the ours-arm keys,
    impl, cpu_baseline and a zero-copy e2e, warm-up samples untimed."""
    line, calls = _reference_line(monkeypatch, capsys, {"RANK": "0", "WORLD_SIZE": "1"})
    assert len(calls) == 3 and calls[0] == (12, "amg")
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] == 2000.0 and line["ms_per_step"] == 500.0 and line["unit"] == "DOFs/s"
    assert line["higher_is_better"] is True and line["vs_baseline"] is None and line["n_gpus"] == 1
    assert line["config"]["workload"] == "hex128-k1-fgmres30-blocktri-amg-fp64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == 2000.0 and cb["sample"]
    assert line["e2e"] == {"value": 2000.0, "unit": "DOFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    """Under a multi-rank launch only rank 0 runs the oracle and prints."""
    line, calls = _reference_line(monkeypatch, capsys, {"RANK": "1", "WORLD_SIZE": "2"})
    assert line is None and calls == []
