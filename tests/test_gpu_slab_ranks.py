"""The slab decomposition of one problem run as separate processes, each holding its slab in
device memory and running its sweeps, block copies and slab residual through the C ABI
(paper_1609_07758_gb300/slab.py, GpuOps).  The two ranks share the one GPU of this run, so
their exchanges go through `gloo` on host copies of the packs (HostComm below): no kernel of
one rank waits on a kernel of the other, as an NCCL all-to-all between two processes on one
GPU would.  The gathered slabs are compared with the plan's own undivided solve.
"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_07758_gb300 import build as b
    b.build()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class HostComm:
    """all_to_all of device packs through gloo: copy to the host, exchange, copy back."""

    def all_to_all(self, send, send_counts, recv_counts, ops):
        import torch.distributed as dist
        s = send.cpu()
        r = torch.empty(sum(recv_counts), dtype=s.dtype)
        dist.all_to_all_single(r, s, recv_counts, send_counts)
        return r.to(send.device)


CASES = {
    # (N, element counts, order, lengths, dtype name, corrections, ranks)
    "2d_n9_refined": (2, [64, 48], 9, [1.0, 1.3], "HOFEM_FP32_REFINED", 2, 2),
    "3d_n3_fp64": (3, [8, 6, 5], 3, [1.0, 0.8, 1.2], "HOFEM_FP64", 0, 3),
}


def _rhs(case):
    N, Ks, n = CASES[case][:3]
    return np.random.default_rng(12).standard_normal([1] + [n * K - 1 for K in Ks])


def _rank(rank, world, port, case, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import paper_1609_07758_gb300 as hofem
    from paper_1609_07758_gb300 import slab
    N, Ks, n, Xs, dt, corr, _ = CASES[case]
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    M = tuple(n * K - 1 for K in Ks)
    L = slab.SlabLayout.by_elements(M, Ks[0], n, world)
    plan = hofem.Plan(N, Ks, n, Xs, getattr(hofem, dt))
    solver = slab.SlabSolver(L, rank, slab.GpuOps(plan), 1)
    start, rows = L.rows[rank]
    f = torch.from_numpy(np.ascontiguousarray(_rhs(case)[:, start:start + rows])).cuda()
    u = torch.empty_like(f)
    if corr:
        solver.solve_refined(f, u, HostComm(), corr)
    else:
        solver.solve(f, u, HostComm())
    torch.cuda.synchronize()
    np.save(os.path.join(out_dir, f"{case}_u{rank}.npy"), u.cpu().numpy())
    plan.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", list(CASES))
def test_slab_solve_over_processes_matches_the_undivided_solve(tmp_path, case):
    import torch.multiprocessing as mp
    import paper_1609_07758_gb300 as hofem
    N, Ks, n, Xs, dt, corr, world = CASES[case]
    mp.start_processes(_rank, args=(world, _free_port(), case, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    u = np.concatenate([np.load(tmp_path / f"{case}_u{k}.npy") for k in range(world)], axis=1)
    plan = hofem.Plan(N, Ks, n, Xs, getattr(hofem, dt))
    if corr:
        plan.set_refinement(corr)
    fd = torch.from_numpy(_rhs(case)).cuda()
    ud = torch.empty_like(fd)
    plan.solve(fd, ud, 1)
    torch.cuda.synchronize()
    ref = ud.cpu().numpy()
    plan.close()
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    assert err <= 1e-13, err
