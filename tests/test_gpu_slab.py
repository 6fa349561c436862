"""GPU parity of the slab decomposition of one problem (paper_1609_07758_gb300/slab.py):
hofem_sweep on blocks of lines (with the fused sweep's column offset) and hofem_copy_block
for the exchange packs, on one GPU.  P slabs are driven phase by phase in one process; the
all-to-all between phases is emulated by concatenating the device packs (what
torch.distributed.all_to_all_single delivers), since this run has one GPU.  The result is
compared with the oracle element by element and with the plan's own single-GPU solve.
"""
import numpy as np
import pytest

from oracle import solve as osolve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_07758_gb300 import build as b
    b.build()
    import paper_1609_07758_gb300 as hofem
    return hofem.load_library()


def _exchange(sends, counts_of):
    """recv[r] = concatenation over s of the part of sends[s] addressed to r."""
    P = len(sends)
    recvs = []
    for r in range(P):
        parts = []
        for s in range(P):
            c = counts_of(s)
            off = sum(c[:r])
            parts.append(sends[s][off:off + c[r]])
        recvs.append(torch.cat(parts))
    return recvs


def slab_solve(plan, f, parts, nrhs):
    from paper_1609_07758_gb300 import slab
    M = tuple(f.shape[1:])
    L = slab.SlabLayout(M, parts)
    ops = slab.GpuOps(plan)
    solvers = [slab.SlabSolver(L, r, ops, nrhs) for r in range(parts)]
    fl = [f[:, s:s + n].contiguous() for s, n in L.rows]
    ul = [torch.empty_like(x) for x in fl]
    sends = [sv.forward(fl[r], ul[r]) for r, sv in enumerate(solvers)]
    recvs = _exchange(sends, lambda s: L.send_counts_1(s, nrhs))
    sends = [sv.fused(recvs[r]) for r, sv in enumerate(solvers)]
    recvs = _exchange(sends, lambda s: L.recv_counts_1(s, nrhs))
    for r, sv in enumerate(solvers):
        sv.inverse(recvs[r], ul[r])
    torch.cuda.synchronize()
    return torch.cat(ul, dim=1)


@pytest.mark.parametrize("ns,Ks,Xs,alpha,nrhs,parts", [
    ([3, 3], [16, 12], [1.0, 1.4], 0.0, 2, 2),
    ([4, 2], [9, 13], [1.2, 0.8], 1.0, 1, 3),
    ([2, 3, 2], [6, 5, 7], [1.0, 0.9, 1.3], 0.0, 2, 2),
    ([3, 2, 4], [5, 6, 4], [0.8, 1.0, 1.1], 0.5, 1, 3),
])
def test_slab_solve_matches_oracle(ns, Ks, Xs, alpha, nrhs, parts):
    import paper_1609_07758_gb300 as hofem
    N = len(Ks)
    M = [n * K - 1 for n, K in zip(ns, Ks)]
    plan = hofem.Plan(N, Ks, list(ns), Xs, hofem.HOFEM_FP64, alpha)
    f = np.random.default_rng(3).standard_normal([nrhs] + M)
    fd = torch.from_numpy(f).cuda()
    u = slab_solve(plan, fd, parts, nrhs).cpu().numpy()
    ref = osolve.solve_tensor(f, ns, Ks, Xs, alpha)
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    assert err <= 1e-12, err
    plan.close()


@pytest.mark.parametrize("dtype,tol,parts", [("HOFEM_FP64", 1e-13, 4), ("HOFEM_FP32", 1e-5, 3)])
def test_slab_solve_matches_single_gpu_solve_n9_k64(dtype, tol, parts):
    """2D n = 9, K = 64 (575^2 unknowns; the register-sweep shape is n = 9 at K = 1024 only,
    so this runs the general sweeps) against hofem_solve of the same plan."""
    import paper_1609_07758_gb300 as hofem
    plan = hofem.Plan(2, [64, 64], 9, [1.0, 1.0], getattr(hofem, dtype))
    M = 575
    f = torch.randn(1, M, M, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    u_ref = torch.empty_like(f)
    plan.solve(f, u_ref, 1)
    u = slab_solve(plan, f, parts, 1)
    err = float(torch.linalg.vector_norm(u - u_ref) / torch.linalg.vector_norm(u_ref))
    assert err <= tol, err
    plan.close()


def test_block_sweep_rejects_bad_blocks():
    import paper_1609_07758_gb300 as hofem
    from paper_1609_07758_gb300 import binding
    plan = hofem.Plan(2, [8, 8], 2, [1.0, 1.0], hofem.HOFEM_FP64)
    x = torch.zeros(15 * 15, dtype=torch.float64, device="cuda")
    with pytest.raises(hofem.HofemError):      # the fused sweep runs along axis 0 only
        plan.sweep(1, hofem.HOFEM_SWEEP_FUSED, x, x, 15, 1)
    with pytest.raises(hofem.HofemError):      # columns beyond the x_2 plane
        plan.sweep(0, hofem.HOFEM_SWEEP_FUSED, x, x, 1, 10, 8)
    with pytest.raises(hofem.HofemError):      # an empty or out-of-range element stretch
        binding.hofem_residual_slab(plan.handle, 1, 5, 5, x, x, None, x, None, 0, 1)
    with pytest.raises(hofem.HofemError):
        binding.hofem_residual_slab(plan.handle, 0, 6, 9, x, None, None, x, x, 0, 1)
    plan.close()


def _slab_plans(N, Ks, n, Xs, dtype, parts, alpha=0.0):
    """One plan per slab, as every GPU of a split problem holds its own."""
    import paper_1609_07758_gb300 as hofem
    return [hofem.Plan(N, Ks, n, Xs, dtype, alpha) for _ in range(parts)]


def _emulated(L, solvers):
    """Run the slab residual and the refined slab solve phase by phase over all slabs."""
    def residual(fs, us, rs):
        packs = [sv.residual_local(us[k]) for k, sv in enumerate(solvers)]
        recvs = _exchange([p[2] for p in packs], lambda k: solvers[k].halo_counts()[0])
        for k, sv in enumerate(solvers):
            sv.residual_last(packs[k][0], packs[k][1], recvs[k], fs[k], rs[k])

    def solve(fs, us):
        q = solvers[0].nrhs
        sends = [sv.forward(fs[k], us[k]) for k, sv in enumerate(solvers)]
        recvs = _exchange(sends, lambda k: L.send_counts_1(k, q))
        sends = [sv.fused(recvs[k]) for k, sv in enumerate(solvers)]
        recvs = _exchange(sends, lambda k: L.recv_counts_1(k, q))
        for k, sv in enumerate(solvers):
            sv.inverse(recvs[k], us[k])

    def solve_refined(fs, us, corrections):
        solve(fs, us)
        rs = [torch.empty_like(u) for u in us]
        ds = [torch.empty_like(u) for u in us]
        for _ in range(corrections):
            residual(fs, us, rs)
            solve(rs, ds)
            for k, sv in enumerate(solvers):
                sv.ops.axpy(us[k], 1.0, ds[k], us[k].numel())

    return residual, solve_refined


@pytest.mark.parametrize("N,Ks,n,Xs,alpha,nrhs,parts", [
    (2, [12, 9], 3, [1.0, 1.3], 0.0, 2, 3),
    (2, [10, 10], 4, [1.0, 1.0], 0.0, 1, 4),          # uniform scale, last slab one element
    (2, [7, 8], 2, [0.9, 1.1], 1.5, 1, 2),
    (3, [6, 5, 4], 2, [1.0, 0.8, 1.2], 0.0, 2, 3),
    (3, [5, 5, 5], 3, [1.0, 1.0, 1.0], 0.5, 1, 2),    # uniform scale with alpha
])
def test_slab_residual_matches_the_plans_residual(N, Ks, n, Xs, alpha, nrhs, parts):
    import paper_1609_07758_gb300 as hofem
    from paper_1609_07758_gb300 import slab
    M = [n * K - 1 for K in Ks]
    L = slab.SlabLayout.by_elements(tuple(M), Ks[0], n, parts)
    plans = _slab_plans(N, Ks, n, Xs, hofem.HOFEM_FP64, parts, alpha)
    solvers = [slab.SlabSolver(L, k, slab.GpuOps(plans[k]), nrhs) for k in range(parts)]
    residual, _ = _emulated(L, solvers)
    g = torch.Generator("cuda").manual_seed(2)
    f = torch.randn([nrhs] + M, dtype=torch.float64, device="cuda", generator=g)
    u = torch.randn([nrhs] + M, dtype=torch.float64, device="cuda", generator=g)
    fs = [f[:, s:s + c].contiguous() for s, c in L.rows]
    us = [u[:, s:s + c].contiguous() for s, c in L.rows]
    rs = [torch.empty_like(x) for x in fs]
    residual(fs, us, rs)
    r_ref = torch.empty_like(f)
    plans[0].residual(f, u, r_ref, nrhs)
    torch.cuda.synchronize()
    r = torch.cat(rs, dim=1)
    err = float(torch.linalg.vector_norm(r - r_ref) / torch.linalg.vector_norm(r_ref))
    assert err <= 1e-14, err
    for p in plans:
        p.close()


@pytest.mark.parametrize("N,Ks,n,Xs,nrhs,parts", [
    (2, [16, 12], 3, [1.0, 1.4], 2, 3),
    (3, [6, 5, 7], 2, [1.0, 0.9, 1.3], 1, 2),
])
def test_refined_slab_solve_matches_oracle_and_the_plans_solve(N, Ks, n, Xs, nrhs, parts):
    import paper_1609_07758_gb300 as hofem
    from paper_1609_07758_gb300 import slab
    M = [n * K - 1 for K in Ks]
    L = slab.SlabLayout.by_elements(tuple(M), Ks[0], n, parts)
    plans = _slab_plans(N, Ks, n, Xs, hofem.HOFEM_FP32_REFINED, parts)
    solvers = [slab.SlabSolver(L, k, slab.GpuOps(plans[k]), nrhs) for k in range(parts)]
    _, solve_refined = _emulated(L, solvers)
    f = np.random.default_rng(4).standard_normal([nrhs] + M)
    fd = torch.from_numpy(f).cuda()
    fs = [fd[:, s:s + c].contiguous() for s, c in L.rows]
    us = [torch.empty_like(x) for x in fs]
    solve_refined(fs, us, 2)
    plans[0].set_refinement(2)
    u_ref = torch.empty_like(fd)
    plans[0].solve(fd, u_ref, nrhs)
    torch.cuda.synchronize()
    u = torch.cat(us, dim=1)
    err = float(torch.linalg.vector_norm(u - u_ref) / torch.linalg.vector_norm(u_ref))
    assert err <= 1e-13, err
    ref = osolve.solve_tensor(f, [n] * N, Ks, Xs, 0.0)
    err_o = np.linalg.norm(u.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err_o <= 1e-12, err_o
    for p in plans:
        p.close()


def test_refined_slab_solve_n9_k1024_register_sweeps():
    """The benchmark's grid (2D n = 9, K = 1024, register sweeps) in 4 slabs, 2 corrections,
    against the plan's own refined solve."""
    import paper_1609_07758_gb300 as hofem
    from paper_1609_07758_gb300 import inputs, slab
    K, n, parts = 1024, 9, 4
    M = [n * K - 1] * 2
    L = slab.SlabLayout.by_elements(tuple(M), K, n, parts)
    plans = _slab_plans(2, [K, K], n, [1.0, 1.0], hofem.HOFEM_FP32_REFINED, parts)
    solvers = [slab.SlabSolver(L, k, slab.GpuOps(plans[k]), 1) for k in range(parts)]
    _, solve_refined = _emulated(L, solvers)
    fd = torch.from_numpy(inputs.smooth_sine_rhs(2, n, K)).cuda()
    fs = [fd[:, s:s + c].contiguous() for s, c in L.rows]
    us = [torch.empty_like(x) for x in fs]
    solve_refined(fs, us, 2)
    plans[0].set_refinement(2)
    u_ref = torch.empty_like(fd)
    plans[0].solve(fd, u_ref, 1)
    torch.cuda.synchronize()
    u = torch.cat(us, dim=1)
    err = float(torch.linalg.vector_norm(u - u_ref) / torch.linalg.vector_norm(u_ref))
    assert err <= 1e-13, err
    for p in plans:
        p.close()
