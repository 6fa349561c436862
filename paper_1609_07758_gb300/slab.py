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

Refined solves (``SlabSolver.solve_refined``) add the FP64 residual of each slab
(``hofem_residual_slab``): the operator's sweeps along x_N .. x_2 are local; the sweep along
x_1 needs the previous slab's last row and the next slab's first n rows of its two
intermediate arrays, which one more (small) all-to-all exchanges; slabs then hold whole
elements along x_1 (``SlabLayout.by_elements``).  The correction solves run the plan's
low-precision sweeps through the same two-exchange path, and ``hofem_axpy`` adds them to u.
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

    @classmethod
    def by_elements(cls, M, K0, n0, parts):
        """Slabs of whole elements along x_1 (needed by the slab residual): slab r owns elements
        e_r .. e_{r+1} - 1, i.e. the dof rows e_r n0 .. min(e_{r+1} n0, M_1) - 1."""
        L = cls(tuple(M), parts)
        if parts > K0:
            raise ValueError("parts must not exceed the elements along x_1")
        L.elems = [(s, s + c) for s, c in split(K0, parts)]
        L.rows = [(e0 * n0, min(e1 * n0, M[0]) - e0 * n0) for e0, e1 in L.elems]
        if min(c for _, c in L.rows) < 1:
            raise ValueError("every slab needs at least one row")
        L.K0, L.n0 = K0, n0
        return L

    def lead_rows(self, rank):
        """The rows a slab sends to the previous one: its first n0, or all it has (the last
        element's right node is the Dirichlet boundary)."""
        return min(self.n0, self.rows[rank][1])

    def halo(self, rank):
        """(rows before, rows after) of a slab's halo for the operator along x_1."""
        e0, e1 = self.elems[rank]
        return (1 if e0 > 0 else 0), (self.n0 if e1 < self.K0 else 0)

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

    def residual_slab(self, stage, e0, e1, a, b, f, out0, out1, nrhs):
        binding.hofem_residual_slab(self.plan.handle, stage, e0, e1, a, b, f, out0, out1, 0, nrhs, self.stream)

    def axpy(self, y, c, x, count):
        binding.hofem_axpy(y, c, x, count, self.stream)

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

    # ---- the slab residual r = f - A u (layout from SlabLayout.by_elements)
    def _ext_rows(self):
        pre, post = self.L.halo(self.rank)
        return pre, self.L.rows[self.rank][1], post

    def residual_local(self, u):
        """Stage 0: the two intermediates, owned rows filled; returns (t0, t1, halo pack)."""
        L, r, ops, q = self.L, self.rank, self.ops, self.nrhs
        pre, rows, post = self._ext_rows()
        plane = L.M[1] * L.tail
        ext = pre + rows + post
        t0, t1 = ops.empty(q * ext * plane, u), ops.empty(q * ext * plane, u)
        e0, e1 = L.elems[r]
        ops.residual_slab(0, e0, e1, u, None, None, t0, t1, q)
        # pack by destination: the first rows for rank r - 1, then the last row for rank r + 1
        up, down = (1 if r + 1 < L.parts else 0), (L.lead_rows(r) if r > 0 else 0)
        send = ops.empty(2 * q * (up + down) * plane, u)
        off = 0
        if down:
            for t in (t0, t1):
                ops.copy_block(t, pre * plane, send, off, q, down, plane, plane, plane, ext * plane, down * plane)
                off += q * down * plane
        if up:
            for t in (t0, t1):
                ops.copy_block(t, (pre + rows - 1) * plane, send, off, q, 1, plane, plane, plane, ext * plane, plane)
                off += q * plane
        return t0, t1, send

    def halo_counts(self):
        """(send, recv) counts of the halo exchange, per rank."""
        L, r, q = self.L, self.rank, self.nrhs
        plane = L.M[1] * L.tail
        send = [0] * L.parts
        recv = [0] * L.parts
        if r > 0:
            send[r - 1] = 2 * q * L.lead_rows(r) * plane     # my first rows: its 'after' halo
            recv[r - 1] = 2 * q * plane                      # its last row: my 'before' halo
        if r + 1 < L.parts:
            send[r + 1] = 2 * q * plane
            recv[r + 1] = 2 * q * L.lead_rows(r + 1) * plane
        return send, recv

    def residual_last(self, t0, t1, recv, f, out):
        """Stage 1: unpack the halo rows, the sweep along x_1: out = f - A u on the slab."""
        L, r, ops, q = self.L, self.rank, self.ops, self.nrhs
        pre, rows, post = self._ext_rows()
        plane = L.M[1] * L.tail
        ext = pre + rows + post
        off = 0
        if r > 0:                                       # from rank r - 1: its last row, both arrays
            for t in (t0, t1):
                ops.copy_block(recv, off, t, 0, q, 1, plane, plane, plane, plane, ext * plane)
                off += q * plane
        if r + 1 < L.parts:                             # from rank r + 1: its first rows
            lead = L.lead_rows(r + 1)
            for t in (t0, t1):
                ops.copy_block(recv, off, t, (pre + rows) * plane, q, lead, plane, plane, plane, lead * plane,
                               ext * plane)
                off += q * lead * plane
        e0, e1 = L.elems[r]
        ops.residual_slab(1, e0, e1, t0, t1, f, out, None, q)

    def residual(self, f, u, out, comm):
        t0, t1, send = self.residual_local(u)
        sc, rc = self.halo_counts()
        recv = comm.all_to_all(send, sc, rc, self.ops)
        self.residual_last(t0, t1, recv, f, out)

    def solve_refined(self, f, u, comm, corrections):
        """u = A^{-1} f: the plan's low-precision solve, then `corrections` steps of
        r = f - A u (FP64, slab residual), delta = solve(r), u += delta."""
        self.solve(f, u, comm)
        r = self.ops.empty(u.numel(), u)
        d = self.ops.empty(u.numel(), u)
        for _ in range(corrections):
            self.residual(f, u, r, comm)
            self.solve(r, d, comm)
            self.ops.axpy(u, 1.0, d, u.numel())
