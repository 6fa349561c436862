"""Batched solves (hofem_batch_*): problems of uneven N, K, n, X, alpha and nrhs in one
captured CUDA graph, each against the oracle's tensor-product solve; graph reuse and
recapture; the autotuner's launch shapes give the same solutions."""
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


def H():
    import paper_1609_07758_gb300 as hofem
    return hofem


PROBLEMS = [
    {"N": 2, "K": (37, 48), "n": 2, "X": (1.3, 0.7), "alpha": 0.0, "nrhs": 2},
    {"N": 2, "K": (64, 64), "n": 3, "X": (1.0, 1.0), "alpha": 1.5, "nrhs": 1},
    {"N": 2, "K": (33, 20), "n": 5, "X": (2.5, 0.6), "alpha": 0.0, "nrhs": 3},
    {"N": 3, "K": (6, 5, 9), "n": 3, "X": (1.0, 1.0, 1.0), "alpha": 0.0, "nrhs": 1},
    {"N": 2, "K": (100, 7), "n": 8, "X": (4.0, 0.5), "alpha": 0.0, "nrhs": 2},
    {"N": 3, "K": (8, 8, 8), "n": 2, "X": (1.0, 1.0, 1.0), "alpha": -1.0, "nrhs": 2},
    {"N": 2, "K": (2, 3), "n": 1, "X": (1.0, 1.0), "alpha": 0.0, "nrhs": 1},
    {"N": 2, "K": (127, 32), "n": 4, "X": (0.9, 3.1), "alpha": 0.0, "nrhs": 1},
]


def rhs(i, q):
    rng = np.random.default_rng([7, i])
    return rng.standard_normal((q["nrhs"],) + tuple(q["n"] * k - 1 for k in q["K"]))


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("dtype,tol", [(0, 1e-12), (4, 1e-12), (5, 1e-12), (6, 1e-12), (1, 1e-5)])
def test_batch_matches_oracle(dtype, tol):
    b = H().Batch(PROBLEMS, dtype)
    fs = [rhs(i, q) for i, q in enumerate(PROBLEMS)]
    fd = [torch.from_numpy(f).cuda() for f in fs]
    ud = [torch.zeros_like(f) for f in fd]
    b.solve(fd, ud)
    torch.cuda.synchronize()
    for i, q in enumerate(PROBLEMS):
        ref = osolve.solve_tensor(fs[i], [q["n"]] * q["N"], list(q["K"]), list(q["X"]), q["alpha"])
        err = rel_l2(ud[i].cpu().numpy(), ref)
        assert err <= tol, (i, err)
    info = b.info()
    assert info.count == len(PROBLEMS) and info.captures == 1 and info.graph_nodes > 0
    assert info.unknowns == sum(q["nrhs"] * int(np.prod([q["n"] * k - 1 for k in q["K"]])) for q in PROBLEMS)


def test_batch_graph_reuse_recapture_and_tuning():
    b = H().Batch(PROBLEMS, H().HOFEM_FP32_REFINED)
    fd = [torch.from_numpy(rhs(i, q)).cuda() for i, q in enumerate(PROBLEMS)]
    u1 = [torch.zeros_like(f) for f in fd]
    b.solve(fd, u1)
    b.solve(fd, u1)                                   # same pointers: the graph is relaunched
    torch.cuda.synchronize()
    assert b.info().captures == 1
    u2 = [torch.zeros_like(f) for f in fd]
    b.solve(fd, u2)                                   # new pointers: recaptured
    torch.cuda.synchronize()
    assert b.info().captures == 2
    for x, y in zip(u1, u2):
        assert torch.equal(x, y)
    b.tune()
    assert b.info().tune_ms > 0 and b.plan_info(0).tuned_shapes > 0
    u3 = [torch.zeros_like(f) for f in fd]
    b.solve(fd, u3)
    torch.cuda.synchronize()
    assert b.info().captures == 3
    for x, y in zip(u1, u3):
        assert float(torch.linalg.vector_norm(x - y) / torch.linalg.vector_norm(y)) <= 1e-12


def test_batch_rejects_aliased_and_null_pointers():
    b = H().Batch(PROBLEMS[:2], H().HOFEM_FP32_REFINED)
    fd = [torch.from_numpy(rhs(i, q)).cuda() for i, q in enumerate(PROBLEMS[:2])]
    with pytest.raises(H().HofemError):
        b.solve(fd, fd)
