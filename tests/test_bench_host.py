"""Host logic of bench.py's multi-process path (replicas, max over ranks),
checked with world_size-2 gloo process groups on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, values, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.max_over_ranks(values[rank])
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    values = [12.5, 40.25]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, values, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 40.25


def test_single_rank_identity_and_throughput():
    assert bench.max_over_ranks(3.5) == 3.5
    # two replicas of 2.652 GB each, 10 steps in 100 ms (slowest rank) -> 530.4 GB/s
    assert bench.job_throughput(2.652e9, 10, 100.0, 2) == pytest.approx(530.4)


def test_reference_arm_other_ranks_do_nothing(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    bench.run_reference(A())
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("kind,count", [("batch", 2048), ("serve", 400)])
def test_solves_cpu_baseline_reports_its_sample(kind, count):
    """The batch and serving CPU baselines solve a prefix of the same request
    list with the oracle and say how much they solved."""
    r = bench.solves_cpu_baseline(kind, count, 0.05)
    assert r["kind"] == "oracle" and r["unit"] == "solves/s" and r["value"] > 0 and r["cores"] >= 1
    assert f"of the {count} {kind} requests in list order" in r["sample"]
    assert len(r["_energies"]) >= 1 and all(isinstance(e, float) for e in r["_energies"])


def test_agreement_of_gpu_and_oracle_energies():
    d, n = bench.agreement([-1.0, None, 2.0, 5.0], [-1.0 - 2e-12, -3.0, 2.0 + 4e-12])
    assert n == 2 and d == pytest.approx(2e-12, rel=1e-3)
    assert bench.agreement([None], [1.0]) == (None, 0)


def test_attach_solve_baselines(monkeypatch):
    def fake(kind, count, budget):
        return {"value": 1.0, "unit": "solves/s", "_energies": [-2.0, -3.0 + 3e-12]}
    monkeypatch.setattr(bench, "solves_cpu_baseline", fake)
    line = {"batch": {"_energies": [-2.0, -3.0, -4.0]}}
    bench.attach_solve_baselines(line, 2048, 400, 1.0)
    cb = line["batch"]["cpu_baseline"]
    assert "_energies" not in cb and cb["compared"] == 2 and cb["max_rel_diff_vs_gpu"] == pytest.approx(1e-12)
    assert "serve" not in line
