"""One problem split over several GPUs by slabs of x_1 (algorithm (a), Sect. 2 par. 4).

The transforms along x_2..x_N are local to a slab of x_1 rows; the fused sweep along x_1
(direct transform, division by the eigenvalue sums, inverse transform) needs whole x_1
lines.  So each rank

1. transforms its slab along x_N, .., x_2 (``hofem_sweep`` forward),
2. packs, for every rank d, its rows restricted to d's chunk of the x_2 index
   (``hofem_copy_block``), and exchanges the packs with one all-to-all,
3. stacks the received row blocks into whole x_1 lines over its own x_2 chunk and runs
   the fused sweep on them, its columns offset by the chunk's start in the x_2..x_N plane,
4. sends every rank's rows back with a second all-to-all, and
5. transforms its slab back along x_2, .., x_N.

Two all-to-alls per solve, each moving (P - 1) / P of the array.  The arithmetic runs in
the library (``hofem_sweep``, ``hofem_copy_block``); this module only computes the block
geometry and calls the exchange.  ``SlabSolver.solve`` drives one rank with a collective
(``TorchComm``: ``torch.distributed.all_to_all_single``, NCCL on GPUs); the three phases
are also public, so that one process can drive several slabs phase by phase.

Scope: plans in FP64 (and unrefined FP32); refinement with a distributed residual is not
part of this module.
"""
from dataclasses import dataclass

from . import binding


def split(count, parts):
    """Balanced contiguous split of range(count) into `parts` (start, size) pieces."""
    q, r = divmod(int(count), int(parts))
    out, start = [], 0
    for i in range(parts):
        size = q + (1 if i < r else 0)
        out.append((start, size))
        start += size
    return out


@dataclass
class SlabLayout:
    """Slabs of x_1 rows (the data's home) and chunks of the x_2 index (the fused phase)."""
    M: tuple
    parts: int

    def __post_init__(self):
        if len(self.M) not in (2, 3):
            raise ValueError("N must be 2 or 3")
        if self.parts < 1 or self.parts > min(self.M[0], self.M[1]):
            raise ValueError("parts must be between 1 and min(M_1, M_2)")
        self.rows = split(self.M[0], self.parts)
        self.cols = split(self.M[1], self.parts)
        self.tail = 1 if len(self.M) == 2 else self.M[2]     # elements per x_2 index

    def slab_shape(self, rank, nrhs):
        return (nrhs, self.rows[rank][1]) + tuple(self.M[1:])

    def chunk_width(self, rank):
        """Elements of one x_1 row inside rank's x_2 chunk."""
        return self.cols[rank][1] * self.tail

    def send_counts_1(self, rank, nrhs):
        return [nrhs * self.rows[rank][1] * self.chunk_width(d) for d in range(self.parts)]

    def recv_counts_1(self, rank, nrhs):
        return [nrhs * self.rows[s][1] * self.chunk_width(rank) for s in range(self.parts)]


class GpuOps:
    """The per-rank operations on device arrays, through the C ABI."""

    def __init__(self, plan, stream=None):
        self.plan, self.stream = plan, stream

    def sweep(self, axis, mode, x, y, outer, inner, offset=0):
        binding.hofem_sweep(self.plan.handle, axis, mode, x, y, outer, inner, offset, self.stream)

    def copy_block(self, src, src_off, dst, dst_off, batch, rows, cols, src_ld, dst_ld, src_bs, dst_bs):
        binding.hofem_copy_block(src.data_ptr() + 8 * src_off, dst.data_ptr() + 8 * dst_off, batch, rows, cols,
                                 src_ld, dst_ld, src_bs, dst_bs, self.stream)

    def empty(self, count, like):
        import torch
        return torch.empty(count, dtype=torch.float64, device=like.device)


class TorchComm:
    """All-to-all through torch.distributed (NCCL for device tensors, gloo for host ones)."""

    def __init__(self, group=None):
        self.group = group

    def all_to_all(self, send, send_counts, recv_counts, ops):
        import torch.distributed as dist
        recv = ops.empty(sum(recv_counts), send)
        dist.all_to_all_single(recv, send, recv_counts, send_counts, group=self.group)
        return recv


class SlabSolver:
    """u = A^{-1} f for the slab of rank `rank` (f, u: (nrhs, rows, M_2[, M_3]) FP64)."""

    def __init__(self, layout, rank, ops, nrhs=1):
        self.L, self.rank, self.ops, self.nrhs = layout, rank, ops, nrhs

    # phase 1: local forward sweeps, pack for the first exchange
    def forward(self, f, u):
        L, r, ops, q = self.L, self.rank, self.ops, self.nrhs
        M, N = L.M, len(L.M)
        rows = L.rows[r][1]
        plane = M[1] * L.tail
        if N == 3:
            ops.sweep(2, binding.HOFEM_SWEEP_FORWARD, f, u, q * rows * M[1], 1)
            ops.sweep(1, binding.HOFEM_SWEEP_FORWARD, u, u, q * rows, M[2])
        else:
            ops.sweep(1, binding.HOFEM_SWEEP_FORWARD, f, u, q * rows, 1)
        send = ops.empty(q * rows * plane, u)
        off = 0
        for d in range(L.parts):
            cw = L.chunk_width(d)
            ops.copy_block(u, L.cols[d][0] * L.tail, send, off, q, rows, cw, plane, cw, rows * plane, rows * cw)
            off += q * rows * cw
        return send

    # phase 2: whole x_1 lines over this rank's x_2 chunk, the fused sweep, pack back
    def fused(self, recv):
        L, r, ops, q = self.L, self.rank, self.ops, self.nrhs
        cw = L.chunk_width(r)
        M0 = L.M[0]
        y = ops.empty(q * M0 * cw, recv)
        off = 0
        for s in range(L.parts):
            start, rows = L.rows[s]
            ops.copy_block(recv, off, y, start * cw, q, rows, cw, cw, cw, rows * cw, M0 * cw)
            off += q * rows * cw
        ops.sweep(0, binding.HOFEM_SWEEP_FUSED, y, y, q, cw, L.cols[r][0] * L.tail)
        send = ops.empty(q * M0 * cw, y)
        off = 0
        for d in range(L.parts):
            start, rows = L.rows[d]
            ops.copy_block(y, start * cw, send, off, q, rows, cw, cw, cw, M0 * cw, rows * cw)
            off += q * rows * cw
        return send

    # phase 3: unpack this rank's rows, local inverse sweeps
    def inverse(self, recv, u):
        L, r, ops, q = self.L, self.rank, self.ops, self.nrhs
        M, N = L.M, len(L.M)
        rows = L.rows[r][1]
        plane = M[1] * L.tail
        off = 0
        for s in range(L.parts):
            cw = L.chunk_width(s)
            ops.copy_block(recv, off, u, L.cols[s][0] * L.tail, q, rows, cw, cw, plane, rows * cw, rows * plane)
            off += q * rows * cw
        if N == 3:
            ops.sweep(1, binding.HOFEM_SWEEP_INVERSE, u, u, q * rows, M[2])
            ops.sweep(2, binding.HOFEM_SWEEP_INVERSE, u, u, q * rows * M[1], 1)
        else:
            ops.sweep(1, binding.HOFEM_SWEEP_INVERSE, u, u, q * rows, 1)

    def solve(self, f, u, comm):
        L, r, q = self.L, self.rank, self.nrhs
        send = self.forward(f, u)
        recv = comm.all_to_all(send, L.send_counts_1(r, q), L.recv_counts_1(r, q), self.ops)
        send = self.fused(recv)
        recv = comm.all_to_all(send, L.recv_counts_1(r, q), L.send_counts_1(r, q), self.ops)
        self.inverse(recv, u)
