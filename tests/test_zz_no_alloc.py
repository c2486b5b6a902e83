"""The allocation-free MLP backward (amg_mlp_backward_noalloc) against the
allocating one (amg_mlp_backward), through the C ABI.

Callers that cannot allocate device memory (during stream capture, inside
real-time or embedding hosts, or with the device memory handed to another
framework) use the variant whose scratch is a fixed device array.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1403_1649_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1649_gb300 import amg, build
    build.build()
    return torch, amg


def _features(amg, A):
    h = amg.Hierarchy(A, alpha=0.25, seed=1)
    f = np.zeros((A.n, 16), np.float32)
    assert amg.lib().amg_features(h.h, 0, f.ctypes.data, None) == 0
    return f


@pytest.mark.parametrize("m", [38, 45])  # 1444 rows, and 2025 rows (near the 2048-row limit)
def test_noalloc_backward_matches_allocating_backward_twice(env, m):
    torch, amg = env
    L = amg.lib()
    feat = _features(amg, P.fem2d(m, 21))
    n = feat.shape[0]
    rng = np.random.default_rng(m)
    dev = torch.device("cuda")
    w = torch.from_numpy((rng.normal(size=5443) * 0.3).astype(np.float32)).to(dev)
    f = torch.from_numpy(feat.reshape(-1)).to(dev)
    dout = torch.from_numpy(rng.normal(size=3 * n).astype(np.float32)).to(dev)
    ref = torch.zeros(5443, dtype=torch.float64, device=dev)
    assert L.amg_mlp_backward(n, w.data_ptr(), f.data_ptr(), dout.data_ptr(), ref.data_ptr(), None) == 0
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    assert np.abs(r).max() > 0
    for _ in range(2):  # the fixed array keeps the previous call's contents
        got = torch.full((5443,), np.nan, dtype=torch.float64, device=dev)
        assert L.amg_mlp_backward_noalloc(n, w.data_ptr(), f.data_ptr(), dout.data_ptr(), got.data_ptr(),
                                          None) == 0
        torch.cuda.synchronize()
        g = got.cpu().numpy()
        assert np.allclose(g, r, rtol=1e-12, atol=1e-12 * np.abs(r).max())


def test_noalloc_backward_rejects_too_many_rows(env):
    torch, amg = env
    L = amg.lib()
    n = 2049
    dev = torch.device("cuda")
    w = torch.zeros(5443, dtype=torch.float32, device=dev)
    f = torch.zeros(16 * n, dtype=torch.float32, device=dev)
    dout = torch.zeros(3 * n, dtype=torch.float32, device=dev)
    out = torch.zeros(5443, dtype=torch.float64, device=dev)
    rc = L.amg_mlp_backward_noalloc(n, w.data_ptr(), f.data_ptr(), dout.data_ptr(), out.data_ptr(), None)
    assert rc == amg.AMG_ERR_BAD_INPUT
    assert "2048" in amg.amg_last_error()
