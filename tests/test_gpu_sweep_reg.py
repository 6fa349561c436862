"""GPU parity of the register-resident FP32 sweep (the warp-FFT kernel instantiated for
(n, K) = (9, 1024), (4, 128), (8, 64)) against the oracle, element by element.

The transform hook runs W lines per CTA over a number of lines that leaves the last tile
ragged; the solves run it on contiguous and strided axes, several right-hand sides,
mixed orders per axis, next to axes on the general kernel, unrefined (FP32, 1e-5) and
refined (1e-12).  HOFEM_SWEEP_REG=0 forces the general kernel on the same plan, which both
paths are also compared against.
"""
import numpy as np
import pytest

from oracle import solve as osolve, spectrum

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


def H():
    import paper_1609_07758_gb300 as hofem
    return hofem


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel_l2(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return (np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)).max()


def transforms(plan, y, c, lines, M):
    out = torch.zeros(lines, M, dtype=torch.float64, device="cuda")
    plan.transform1d(0, 0, dev(y), out, lines)
    torch.cuda.synchronize()
    fwd = out.cpu().numpy()
    plan.transform1d(0, 1, dev(c), out, lines)
    torch.cuda.synchronize()
    return fwd, out.cpu().numpy()


@pytest.mark.parametrize("n,K,lines,W", [(9, 1024, 5, 4), (9, 1024, 3, 4), (4, 128, 37, 16), (8, 64, 21, 16)])
def test_register_sweep_transforms_match_oracle(monkeypatch, n, K, lines, W):
    X = 1.3
    plan = H().Plan(2, [K, K], n, [X, X], H().HOFEM_FP32)
    s = spectrum.spectrum(n, K, X)
    S = s.dense_S()
    M = n * K - 1
    rng = np.random.default_rng(n * 100 + K)
    y = rng.standard_normal((lines, M))
    c = rng.standard_normal((lines, M))
    fac = np.sqrt(s.norm / K)
    fwd, inv = transforms(plan, y, c, lines, M)
    assert plan.info().lines_per_cta[0] == W
    ref_f, ref_i = s.forward(y, S) * fac, s.inverse(c / fac, S)
    e_f, e_i = rel_l2(fwd, ref_f), rel_l2(inv, ref_i)
    print(f"n {n} K {K} W {W}: forward {e_f:.2e}, inverse {e_i:.2e}")
    assert e_f <= 3e-6 and e_i <= 3e-6
    # the general kernel on the same plan agrees to FP32 rounding
    monkeypatch.setenv("HOFEM_SWEEP_REG", "0")
    fwd0, inv0 = transforms(plan, y, c, lines, M)
    assert rel_l2(fwd0, ref_f) <= 3e-6 and rel_l2(inv0, ref_i) <= 3e-6
    assert rel_l2(fwd, fwd0) <= 4e-6 and rel_l2(inv, inv0) <= 4e-6


REG_SOLVES = [
    # N, orders per axis, K, X, alpha, nrhs
    (2, [4, 4], [128, 128], [1.0, 2.5], 0.5, 3),      # both axes: contiguous and strided, ragged tiles
    (2, [8, 8], [64, 64], [0.7, 1.0], 0.0, 2),
    (2, [4, 8], [128, 64], [1.0, 1.0], 0.0, 1),       # two instantiations, M = 511 on both axes
    (2, [9, 9], [1024, 16], [1.0, 0.5], 0.0, 1),      # fused sweep on K = 1024; general kernel on axis 1
    (2, [9, 9], [16, 1024], [1.0, 1.0], 0.0, 2),      # K = 1024 contiguous: first and last sweeps
    (3, [4, 4, 4], [128, 8, 128], [1.0, 1.0, 0.8], 0.0, 1),    # 3D: strided middle axis on the general kernel
    (3, [4, 4, 4], [16, 128, 16], [1.0, 1.2, 1.0], 0.25, 1),   # 3D: K = 128 on the strided middle axis
]


@pytest.mark.parametrize("dtype,tol", [(1, 1e-5), (4, 1e-12)])
@pytest.mark.parametrize("N,ns,K,X,alpha,nrhs", REG_SOLVES)
def test_solves_on_register_sweeps_match_oracle(dtype, tol, N, ns, K, X, alpha, nrhs):
    plan = H().Plan(N, K, ns if len(set(ns)) > 1 else ns[0], X, dtype, alpha)
    Ms = [n * k - 1 for n, k in zip(ns, K)]
    rng = np.random.default_rng(sum(Ms) + nrhs)
    f = rng.standard_normal([nrhs] + Ms)
    ref = osolve.solve_tensor(f, ns, K, X, alpha)
    fd = dev(f)
    ud = torch.zeros_like(fd)
    plan.solve(fd, ud, nrhs)
    torch.cuda.synchronize()
    err = rel_l2(ud.cpu().numpy(), ref)
    print(f"dtype {dtype} orders {ns} K {K}: rel L2 {err:.2e}, {plan.info().iterations} steps")
    assert err <= tol, err
    assert np.array_equal(fd.cpu().numpy(), f)
