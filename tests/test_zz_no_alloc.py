"""hofem_apply_static: the operator apply for callers that cannot allocate device memory.

Such callers (a framework allocator that forbids raw cudaMalloc, a real-time loop that
cannot take cudaMalloc's synchronisation) get the same r = A u as hofem_apply, computed
with intermediates in a fixed device array inside the library.  This file is collected
last so that a run stopping at the first failure has run every other test; it passes
alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_07758_gb300 import build as b
    b.build()
    import paper_1609_07758_gb300 as hofem
    return hofem.load_library()


def _plan(lib, N, n, K, X, alpha):
    plan = ctypes.c_void_p()
    assert lib.hofem_plan(N, (ctypes.c_int * N)(*K), n, (ctypes.c_double * N)(*X), 0, alpha,
                          ctypes.byref(plan)) == 0
    return plan


@pytest.mark.parametrize("N,n,K,X,alpha,nrhs", [
    (2, 4, [32, 64], [1.0, 1.5], 0.5, 2),
    (3, 3, [8, 16, 8], [1.0, 1.0, 2.0], 0.0, 1),
])
def test_static_apply_matches_allocating_apply_twice(lib, N, n, K, X, alpha, nrhs):
    from paper_1609_07758_gb300.binding import hofem_info

    # the static path runs on a plan of its own that never reserves workspace, so an
    # allocation on that path would show as workspace_bytes > 0; the allocating apply runs
    # on a second plan
    p_sta = _plan(lib, N, n, K, X, alpha)
    p_ref = _plan(lib, N, n, K, X, alpha)
    Ms = [n * k - 1 for k in K]
    rng = np.random.default_rng(11)
    try:
        for call in range(2):                        # two calls in a row, different inputs
            u = torch.from_numpy(rng.standard_normal([nrhs] + Ms)).cuda()
            r_ref = torch.zeros_like(u)
            r_sta = torch.full_like(u, float("nan"))
            assert lib.hofem_apply_static(p_sta, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(r_sta.data_ptr()),
                                          nrhs, None) == 0
            torch.cuda.synchronize()
            info = hofem_info()
            assert lib.hofem_get_info(p_sta, ctypes.byref(info)) == 0
            assert info.workspace_bytes == 0
            assert lib.hofem_apply(p_ref, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(r_ref.data_ptr()),
                                   nrhs, None) == 0
            torch.cuda.synchronize()
            a, b = r_sta.cpu().numpy(), r_ref.cpu().numpy()
            err = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert err <= 1e-13, (call, err)
    finally:
        lib.hofem_destroy(p_sta)
        lib.hofem_destroy(p_ref)


def test_static_apply_rejects_problems_above_its_limit(lib):
    K = (ctypes.c_int * 2)(1024, 1024)
    X = (ctypes.c_double * 2)(1.0, 1.0)
    plan = ctypes.c_void_p()
    assert lib.hofem_plan(2, K, 2, X, 0, 0.0, ctypes.byref(plan)) == 0   # 2047^2 > 2,097,152
    try:
        u = torch.zeros(1, 2047, 2047, dtype=torch.float64, device="cuda")
        r = torch.zeros_like(u)
        st = lib.hofem_apply_static(plan, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(r.data_ptr()), 1, None)
        assert st == 1
        assert b"static scratch" in lib.hofem_last_error()
    finally:
        lib.hofem_destroy(plan)
