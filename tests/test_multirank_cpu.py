"""The benchmark's multi-GPU path on the CPU: two `gloo` ranks exercise the same host logic
(max over ranks, barrier, one problem per rank, whole-job throughput) that bench.py runs
over NCCL with one rank per GPU.  The path shards independent problems (weak scaling), so
there is no data-path collective to test."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_1609_07758_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms_local = 10.0 + 5.0 * rank                  # the slower rank sets the job's time
    ms = bench.max_over_ranks(ms_local, w)
    bench.barrier(w)
    f = inputs.smooth_sine_rhs(bench.rank_seed(r), 2, 8)
    value = bench.job_throughput(100, w, ms)
    np.save(os.path.join(out_dir, f"rank{r}.npy"), np.array([r, w, local, ms, value, float(np.abs(f).sum())]))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time_and_solve_different_problems(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    a = np.load(tmp_path / "rank0.npy")
    b = np.load(tmp_path / "rank1.npy")
    assert (a[0], a[1], a[2]) == (0, 2, 0) and (b[0], b[1], b[2]) == (1, 2, 1)
    assert a[3] == b[3] == 15.0                                # max over ranks
    assert a[4] == b[4] == pytest.approx(2 * 100 / 0.015)      # whole-job throughput
    assert a[5] != b[5]                                        # one problem per rank


def _partition_rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import paper_1609_07758_gb300 as hofem
    from paper_1609_07758_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = inputs.batch_problems(4)
    part_of, cost = hofem.batch_partition(probs, hofem.HOFEM_FP32_REFINED, world)
    mine = [i for i, p in enumerate(part_of) if p == rank]
    counts = torch.zeros(len(probs), dtype=torch.int64)
    counts[mine] = 1
    dist.all_reduce(counts)                         # how many ranks took each problem
    load = torch.tensor([sum(cost[i] for i in mine)], dtype=torch.float64)
    loads = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(loads, load)
    np.save(os.path.join(out_dir, f"part{rank}.npy"),
            np.concatenate([counts.numpy().astype(float), [l.item() for l in loads], [max(cost)]]))
    dist.destroy_process_group()


def test_batch_partition_over_two_gloo_ranks_assigns_each_problem_once_and_balances_cost(tmp_path):
    """hofem_batch_partition of the 512-problem batch: both ranks compute the same split
    (host-only, deterministic), every problem lands on exactly one rank, and the ranks'
    predicted work differs by at most one problem's (longest processing time first)."""
    import torch.multiprocessing as mp
    from paper_1609_07758_gb300 import binding
    if not os.path.exists(binding.library_path()):
        pytest.skip("libhofem.so is not built")
    port = _free_port()
    mp.start_processes(_partition_rank, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    a, b = np.load(tmp_path / "part0.npy"), np.load(tmp_path / "part1.npy")
    assert np.array_equal(a, b)
    counts, loads, cmax = a[:512], a[512:514], a[514]
    assert np.all(counts == 1)
    assert abs(loads[0] - loads[1]) <= cmax
    assert max(loads) / min(loads) < 1.02
