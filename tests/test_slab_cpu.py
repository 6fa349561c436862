"""The slab decomposition of one problem (paper_1609_07758_gb300/slab.py) on the CPU.

Two and three `gloo` ranks each hold a slab of x_1 rows and run SlabSolver with the same
block geometry and the same two all-to-all exchanges the GPUs run over NCCL.  The per-rank
operations here are the oracle's plain dense mode products (S along one axis of a block,
the division by the eigenvalue sums at offset columns) and numpy block copies, so the test
checks the decomposition itself -- slabs, chunks, offsets, pack and unpack layouts, the
exchange counts -- against the oracle's undivided solve.  The GPU operations behind the
same interface are tested against the oracle in tests/test_gpu_slab.py.
"""
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


class OracleOps:
    """hofem_sweep / hofem_copy_block semantics written with the oracle's dense matrices."""

    def __init__(self, specs, alpha):
        self.specs, self.alpha = specs, alpha
        self.S = [s.dense_S() for s in specs]

    @staticmethod
    def _view(t, count):
        return t.numpy().reshape(-1)[:count]

    def sweep(self, axis, mode, x, y, outer, inner, offset=0):
        M = self.specs[axis].M
        xa = self._view(x, outer * M * inner).reshape(outer, M, inner).copy()
        S, norm = self.S[axis], self.specs[axis].norm
        if mode in (0, 1):      # direct transform: (x, s_q) / ||s_q||^2 along the axis
            xa = np.einsum("ojl,jq->oql", xa, S) / norm[None, :, None]
        if mode == 1:           # division by the eigenvalue sums at columns offset + l
            rest = np.zeros(int(np.prod([s.M for s in self.specs[1:]])))
            if len(self.specs) == 2:
                rest += self.specs[1].lam
            else:
                rest += (self.specs[1].lam[:, None] + self.specs[2].lam[None, :]).reshape(-1)
            cols = rest[offset:offset + inner]
            xa = xa / (self.specs[0].lam[None, :, None] + cols[None, None, :] + self.alpha)
        if mode in (1, 2):      # inverse transform: sum_q x_q s_q
            xa = np.einsum("oql,jq->ojl", xa, S)
        self._view(y, outer * M * inner)[:] = xa.reshape(-1)

    def copy_block(self, src, src_off, dst, dst_off, batch, rows, cols, src_ld, dst_ld, src_bs, dst_bs):
        s, d = src.numpy().reshape(-1), dst.numpy().reshape(-1)
        for b in range(batch):
            for r in range(rows):
                i, j = src_off + b * src_bs + r * src_ld, dst_off + b * dst_bs + r * dst_ld
                d[j:j + cols] = s[i:i + cols]

    def empty(self, count, like):
        return torch.zeros(count, dtype=torch.float64)

    # hofem_residual_slab with intermediates of this class's own choosing: t0 = u with the mass
    # matrices of x_2..x_N, t1 = the rest of the operator along x_2..x_N; the sweep along x_1
    # then adds s_1 A_1 t0 + C_1 t1 over the slab's rows, read from the rows with their halo
    def set_operator(self, ns, Ks, Xs, alpha):
        from oracle import assemble
        self.ns, self.Ks, self.alpha_op = ns, Ks, alpha
        self.mats = [assemble.global_1d_sparse(n, K) for n, K in zip(ns, Ks)]
        self.sc = [4.0 * (K / X) ** 2 for K, X in zip(Ks, Xs)]

    def residual_slab(self, stage, e0, e1, a, b, f, out0, out1, nrhs):
        from oracle.assemble import _mode_product
        N, n0, K0 = len(self.Ks), self.ns[0], self.Ks[0]
        M = [m[0].shape[0] for m in self.mats]
        rows = min(e1 * n0, M[0]) - e0 * n0
        pre, post = (1 if e0 > 0 else 0), (n0 if e1 < K0 else 0)
        ext = pre + rows + post
        plane = int(np.prod(M[1:]))
        if stage == 0:
            u = self._view(a, nrhs * rows * plane).reshape([nrhs, rows] + M[1:])
            t0 = u
            for m in range(1, N):
                t0 = _mode_product(t0, self.mats[m][1], m + 1)
            t1 = self.alpha_op * t0
            for i in range(1, N):
                t = u
                for m in range(1, N):
                    t = _mode_product(t, self.mats[m][0] if m == i else self.mats[m][1], m + 1)
                t1 = t1 + self.sc[i] * t
            for arr, val in ((out0, t0), (out1, t1)):
                v = self._view(arr, nrhs * ext * plane).reshape(nrhs, ext, plane)
                v[:, pre:pre + rows] = val.reshape(nrhs, rows, plane)
            return
        q0 = e0 * n0 - pre
        hi = min(q0 + ext, M[0])
        A0, C0 = (m.tocsr()[e0 * n0:e0 * n0 + rows, q0:hi] for m in self.mats[0])
        t0 = self._view(a, nrhs * ext * plane).reshape(nrhs, ext, plane)[:, :hi - q0]
        t1 = self._view(b, nrhs * ext * plane).reshape(nrhs, ext, plane)[:, :hi - q0]
        r = np.stack([self.sc[0] * (A0 @ t0[q]) + C0 @ t1[q] for q in range(nrhs)])
        if f is not None:
            r = self._view(f, nrhs * rows * plane).reshape(nrhs, rows, plane) - r
        self._view(out0, nrhs * rows * plane)[:] = r.reshape(-1)

    def axpy(self, y, c, x, count):
        self._view(y, count)[:] += c * self._view(x, count)


CASES = {
    "2d": dict(ns=[3, 2], Ks=[8, 6], Xs=[1.0, 1.5], alpha=0.0, nrhs=2),
    "3d": dict(ns=[2, 3, 2], Ks=[5, 3, 4], Xs=[1.0, 0.7, 1.2], alpha=0.5, nrhs=2),
}


def _rank_main(rank, world, port, case, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from oracle import spectrum
    from paper_1609_07758_gb300 import slab
    c = CASES[case]
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = [spectrum.spectrum(n, K, X) for n, K, X in zip(c["ns"], c["Ks"], c["Xs"])]
    M = tuple(s.M for s in specs)
    layout = slab.SlabLayout(M, world)
    f = np.random.default_rng(7).standard_normal((c["nrhs"],) + M)
    start, rows = layout.rows[rank]
    f_local = torch.from_numpy(np.ascontiguousarray(f[:, start:start + rows]))
    u_local = torch.zeros_like(f_local)
    solver = slab.SlabSolver(layout, rank, OracleOps(specs, c["alpha"]), c["nrhs"])
    solver.solve(f_local, u_local, slab.TorchComm())
    np.save(os.path.join(out_dir, f"{case}_u{rank}.npy"), u_local.numpy())
    dist.destroy_process_group()


def _residual_rank(rank, world, port, case, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from oracle import spectrum
    from paper_1609_07758_gb300 import slab
    c = CASES[case]
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = [spectrum.spectrum(n, K, X) for n, K, X in zip(c["ns"], c["Ks"], c["Xs"])]
    M = tuple(s.M for s in specs)
    layout = slab.SlabLayout.by_elements(M, c["Ks"][0], c["ns"][0], world)
    ops = OracleOps(specs, c["alpha"])
    ops.set_operator(c["ns"], c["Ks"], c["Xs"], c["alpha"])
    rng = np.random.default_rng(9)
    f = rng.standard_normal((c["nrhs"],) + M)
    u = rng.standard_normal((c["nrhs"],) + M)
    start, rows = layout.rows[rank]
    fl = torch.from_numpy(np.ascontiguousarray(f[:, start:start + rows]))
    ul = torch.from_numpy(np.ascontiguousarray(u[:, start:start + rows]))
    solver = slab.SlabSolver(layout, rank, ops, c["nrhs"])
    r = torch.zeros_like(fl)
    solver.residual(fl, ul, r, slab.TorchComm())        # r = f - A u on the slab
    v = torch.zeros_like(fl)
    solver.solve_refined(fl, v, slab.TorchComm(), 2)    # refined solve (exact inner solves here)
    np.save(os.path.join(out_dir, f"{case}_r{rank}.npy"), r.numpy())
    np.save(os.path.join(out_dir, f"{case}_v{rank}.npy"), v.numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("2d", 2), ("2d", 3), ("3d", 3)])
def test_slab_residual_and_refined_solve_over_gloo_ranks_match_the_oracle(tmp_path, case, world):
    """The slab residual's halo exchange (the previous slab's last row, the next slab's first n
    rows of both intermediates) against the oracle's operator on the whole grid, and the refined
    slab solve against the oracle's solve."""
    import torch.multiprocessing as mp
    from oracle import assemble, solve as osolve
    port = _free_port()
    mp.start_processes(_residual_rank, args=(world, port, case, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    c = CASES[case]
    M = tuple(n * K - 1 for n, K in zip(c["ns"], c["Ks"]))
    rng = np.random.default_rng(9)
    f = rng.standard_normal((c["nrhs"],) + M)
    u = rng.standard_normal((c["nrhs"],) + M)
    r = np.concatenate([np.load(tmp_path / f"{case}_r{k}.npy") for k in range(world)], axis=1)
    ref = f - assemble.apply_operator(u, c["ns"], c["Ks"], c["Xs"], c["alpha"])
    assert np.linalg.norm(r - ref) <= 1e-13 * np.linalg.norm(ref)
    v = np.concatenate([np.load(tmp_path / f"{case}_v{k}.npy") for k in range(world)], axis=1)
    vref = osolve.solve_tensor(f, c["ns"], c["Ks"], c["Xs"], c["alpha"])
    assert np.linalg.norm(v - vref) <= 1e-12 * np.linalg.norm(vref)


@pytest.mark.parametrize("case,world", [("2d", 2), ("2d", 3), ("3d", 2), ("3d", 3)])
def test_slab_solve_over_gloo_ranks_matches_the_oracle(tmp_path, case, world):
    import torch.multiprocessing as mp
    from oracle import solve as osolve
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, case, str(tmp_path)), nprocs=world, start_method="spawn",
                       join=True)
    c = CASES[case]
    u = np.concatenate([np.load(tmp_path / f"{case}_u{r}.npy") for r in range(world)], axis=1)
    M = tuple(n * K - 1 for n, K in zip(c["ns"], c["Ks"]))
    f = np.random.default_rng(7).standard_normal((c["nrhs"],) + M)
    ref = osolve.solve_tensor(f, c["ns"], c["Ks"], c["Xs"], c["alpha"])
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    assert err < 1e-12, err


def test_layout_splits_and_exchange_counts_are_consistent():
    from paper_1609_07758_gb300 import slab
    assert slab.split(10, 3) == [(0, 4), (4, 3), (7, 3)]
    L = slab.SlabLayout((23, 17, 5), 3)
    # what rank r sends to d is what d receives from r, in both exchanges
    for r in range(3):
        for d in range(3):
            assert L.send_counts_1(r, 2)[d] == L.recv_counts_1(d, 2)[r]
    assert sum(sum(L.send_counts_1(r, 2)) for r in range(3)) == 2 * 23 * 17 * 5
    with pytest.raises(ValueError):
        slab.SlabLayout((23, 2), 3)
