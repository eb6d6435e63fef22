"""The N > 1 path of bench.py (independent replicas, no data-path collective)
on CPU: two gloo ranks exercise the host-side pieces the GPU job uses —
per-rank inputs, the max-over-ranks time and the whole-job value — and the
reference arm's rank gating."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402

WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, port: int, out_dir: str) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(WORLD))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        wl = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
        u0 = bench.make_u0(wl, bench.replica_seed(0, rank))
        # the slowest rank's time is the job's time: rank r reports 10 + r ms
        ms = bench.max_over_ranks(10.0 + rank, dist, "cpu")
        # every rank solved its own instance: gather a checksum of each input
        sums = [torch.zeros(1, dtype=torch.float64) for _ in range(WORLD)]
        dist.all_gather(sums, torch.tensor([float(np.sum(u0 * np.arange(u0.size)))], dtype=torch.float64))
        dof = wl["nx"] * wl["ny"] * wl["nt"]
        value = bench.whole_job_value(WORLD, dof, ms * 1e-3)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.array([ms, value, dof] + [float(t.item()) for t in sums]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_max_and_distinct_inputs(tmp_path):
    mp.start_processes(_worker, args=(_free_port(), str(tmp_path)), nprocs=WORLD, join=True, start_method="spawn")
    r0, r1 = (np.load(tmp_path / f"rank{r}.npy") for r in range(WORLD))
    assert r0[0] == r1[0] == 11.0                       # max over ranks
    assert r0[1] == r1[1] == WORLD * r0[2] / 11e-3      # all ranks' DOF over the slowest time
    assert r0[3] != r0[4] and r0[3] == r1[3] and r0[4] == r1[4]   # distinct per-rank inputs, seen alike


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.replica_seed(7, 0) == 7 and bench.replica_seed(7, 3) == 10


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    # ranks other than 0 return at once, printing nothing and running no oracle
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "run_cpu_worker", lambda *a, **k: called.append(a))

    class A:
        warmup, steps, workload, alpha, cpu_budget, seed, gpus = 3, 2, bench.DEFAULT_WORKLOAD, 1e-2, 1.0, 0, 2

    bench.main_reference(A())
    assert called == [] and capsys.readouterr().out == ""
