"""Learned polynomial smoother on the GPU against the oracle: features (exact),
MLP forward (FP32 rounding), MLP backward and the two-grid loss gradient, and the
trained network's gain over damped Jacobi."""
import ctypes as C

import numpy as np
import pytest

from paper_1403_1649_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle
    from paper_1403_1649_gb300 import amg, build
    build.build()
    oracle.build()
    return torch, amg, oracle


def two_level(amg, A, **kw):
    return amg.Hierarchy(A, alpha=0.25, seed=1, coarse_max=16, max_levels=2, omega_mode=1, omega=2.0 / 3.0, **kw)


def gradient_term_magnitudes(w, feat, dout):
    """Per parameter, the sum over rows of |term| of its gradient (W1[64][16] b1
    W2[64][64] b2 W3[3][64] b3), from an FP64 forward and backward pass."""
    o = 0
    W1 = w[o:o + 1024].reshape(64, 16); o += 1024
    b1 = w[o:o + 64]; o += 64
    W2 = w[o:o + 4096].reshape(64, 64); o += 4096
    b2 = w[o:o + 64]; o += 64
    W3 = w[o:o + 192].reshape(3, 64)
    h1 = np.tanh(feat @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    dz2 = (dout @ W3) * (1 - h2 * h2)
    dz1 = (dz2 @ W2) * (1 - h1 * h1)
    a = np.abs
    return np.concatenate([(a(dz1).T @ a(feat)).ravel(), a(dz1).sum(0), (a(dz2).T @ a(h1)).ravel(), a(dz2).sum(0),
                           (a(dout).T @ a(h2)).ravel(), a(dout).sum(0)])


def test_features_bit_exact(env):
    torch, amg, oracle = env
    for A in (P.fem2d(40, 3), P.varcoef3d(12, 2, block=4)):
        g = amg.Hierarchy(A, alpha=0.25, seed=1)
        for k in range(g.nlevels):
            L = g.level(k)
            f = np.zeros((L["n"], 16), np.float32)
            assert amg.lib().amg_features(g.h, k, f.ctypes.data, None) == 0
            ref = oracle.features(P.CSR(L["n"], L["rowptr"], L["col"], L["val"]), level=k)
            assert np.array_equal(f, ref), k


def test_mlp_forward_and_backward(env):
    torch, amg, oracle = env
    rng = np.random.default_rng(0)
    w32 = (rng.normal(size=oracle.NPARAM) * 0.3).astype(np.float32)
    w16 = w32.astype(np.float16)
    feat = oracle.features(P.fem2d(30, 4))
    n = feat.shape[0]
    dev = torch.device("cuda")
    fd = torch.from_numpy(feat).to(dev)
    out = torch.zeros(n * 3, dtype=torch.float32, device=dev)
    w16d = torch.from_numpy(w16.view(np.uint16).astype(np.int16)).to(dev)
    assert amg.lib().amg_mlp_forward(n, C.c_void_p(w16d.data_ptr()), C.c_void_p(fd.data_ptr()),
                                     C.c_void_p(out.data_ptr()), None) == 0
    torch.cuda.synchronize()
    ref = oracle.mlp_forward(w16.view(np.uint16), feat)
    assert np.allclose(out.cpu().numpy().reshape(n, 3), ref, rtol=1e-5, atol=1e-5)
    # backward: d<dout, MLP(feat)>/dw at FP32 weights against the FP64 oracle
    dout = rng.normal(size=(n, 3)).astype(np.float32)
    dd = torch.from_numpy(dout.reshape(-1)).to(dev)
    wd = torch.from_numpy(w32).to(dev)
    grad = torch.zeros(oracle.NPARAM, dtype=torch.float64, device=dev)
    assert amg.lib().amg_mlp_backward(n, C.c_void_p(wd.data_ptr()), C.c_void_p(fd.data_ptr()),
                                      C.c_void_p(dd.data_ptr()), C.c_void_p(grad.data_ptr()), None) == 0
    torch.cuda.synchronize()
    gref, _ = oracle.mlp_backward(w32.astype(np.float64), feat, dout.astype(np.float64))
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)
    # element by element: every weight gradient is a sum over rows of products of
    # FP32 activations and back-propagated signals, so each component may differ
    # by a few FP32 roundings of the sum of its terms' magnitudes
    S = gradient_term_magnitudes(w32.astype(np.float64), feat.astype(np.float64), dout.astype(np.float64))
    assert (np.abs(g - gref) <= 2e-5 * S + 1e-12).all(), (np.abs(g - gref) / (S + 1e-30)).max()


@pytest.mark.parametrize("rows,scale", [(1, 0.3), (17, 0.3), (1000, 0.3), (4099, 0.6)])
def test_mlp_forward_tensor_cores_ragged(env, rows, scale):
    """Inference runs on the tensor cores 16 rows per warp (FP16 weights, each FP32
    activation as two FP16 parts, FP32 accumulation): row counts that are not a
    multiple of 16, and weights large enough to saturate tanh, against the
    oracle's FP32 evaluation element by element."""
    torch, amg, oracle = env
    rng = np.random.default_rng(rows)
    w16 = (rng.normal(size=oracle.NPARAM) * scale).astype(np.float16)
    feat = oracle.features(P.fem2d(70, 6))[:rows].copy()
    dev = torch.device("cuda")
    fd = torch.from_numpy(feat).to(dev)
    out = torch.full((rows * 3,), np.nan, dtype=torch.float32, device=dev)
    w16d = torch.from_numpy(w16.view(np.uint16).astype(np.int16)).to(dev)
    assert amg.lib().amg_mlp_forward(rows, C.c_void_p(w16d.data_ptr()), C.c_void_p(fd.data_ptr()),
                                     C.c_void_p(out.data_ptr()), None) == 0
    torch.cuda.synchronize()
    ref = oracle.mlp_forward(w16.view(np.uint16), feat)
    got = out.cpu().numpy().reshape(rows, 3)
    assert np.isfinite(got).all()
    assert np.allclose(got, ref, rtol=1e-5, atol=1e-5), np.abs(got - ref).max()


def test_twogrid_loss_and_gradient(env):
    torch, amg, oracle = env
    A = P.fem2d(24, 5)
    g = two_level(amg, A)
    o = oracle.Hierarchy(A, alpha=0.25, seed=1, coarse_max=16, max_levels=2, omega_mode=1, omega=2.0 / 3.0)
    assert g.nlevels == o.nlevels == 2
    rng = np.random.default_rng(2)
    coef = np.column_stack([rng.uniform(0.4, 0.8, A.n), rng.uniform(-0.2, 0.2, A.n), rng.uniform(-0.1, 0.1, A.n)])
    cd = torch.from_numpy(coef.reshape(-1).copy()).cuda()
    dc = torch.zeros_like(cd)
    loss = C.c_double()
    assert amg.lib().amg_twogrid_loss(g.h, C.c_void_p(cd.data_ptr()), 3, 7, C.byref(loss),
                                      C.c_void_p(dc.data_ptr()), None) == 0
    torch.cuda.synchronize()
    lref, gref = o.twogrid_loss(coef, nvec=3, seed=7)
    assert loss.value == pytest.approx(lref, rel=1e-10)
    assert np.allclose(dc.cpu().numpy().reshape(-1, 3), gref, rtol=1e-8, atol=1e-12 * np.abs(gref).max())


def test_training_reduces_twogrid_factor_and_iterations(env):
    """Train on small FEM problems; on a held-out, larger problem the learned
    smoother must beat damped Jacobi (omega = 2/3) in the two-grid factor and
    in flexible-CG iterations to 1e-8."""
    torch, amg, oracle = env
    train = [two_level(amg, P.fem2d(m, 100 + s)) for m, s in ((32, 0), (40, 1), (48, 2))]
    w = np.zeros(oracle.NPARAM, np.float32)
    rng = np.random.default_rng(3)
    w[: 64 * 16 + 64 + 64 * 64 + 64] = (rng.normal(size=64 * 16 + 64 + 64 * 64 + 64) * 0.2).astype(np.float32)
    steps = 60
    hist = np.zeros(steps)
    arr = (C.c_void_p * len(train))(*[t.h for t in train])
    assert amg.lib().amg_train_smoother(arr, len(train), steps, 3e-3, 2, 11, w.ctypes.data, hist.ctypes.data,
                                        None) == 0
    assert hist[-5:].mean() < hist[:3].mean()
    w16 = w.astype(np.float16).view(np.uint16)
    A = P.fem2d(96, 7)
    b = P.rhs_uniform(A.n, 7)
    # held-out two-grid factor: learned vs Jacobi
    h2 = two_level(amg, A)
    f = np.zeros((A.n, 16), np.float32)
    amg.lib().amg_features(h2.h, 0, f.ctypes.data, None)
    o = oracle.mlp_forward(w16, f).astype(np.float64)
    om = 2.0 / 3.0
    c_l = om * (np.column_stack([np.ones(A.n), np.zeros(A.n), np.zeros(A.n)]) + o)
    c_j = np.column_stack([np.full(A.n, om), np.zeros(A.n), np.zeros(A.n)])
    oh = oracle.Hierarchy(A, alpha=0.25, seed=1, coarse_max=16, max_levels=2, omega_mode=1, omega=om)
    lj, _ = oh.twogrid_loss(c_j, nvec=4, seed=99, grad=False)
    ll, _ = oh.twogrid_loss(c_l, nvec=4, seed=99, grad=False)
    assert ll < lj
    # full hierarchy: iterations with and without the trained network
    hj = amg.Hierarchy(A, alpha=0.25, seed=1, omega_mode=1, omega=om)
    hl = amg.Hierarchy(A, alpha=0.25, seed=1, omega_mode=1, omega=om, smoother=1)
    assert amg.lib().amg_apply_learned_smoother(hl.h, w16.ctypes.data, None) == 0
    _, ij = hj.solve(b, tol=1e-8)
    _, il = hl.solve(b, tol=1e-8)
    assert ij["final_relres"] <= 1e-8 and il["final_relres"] <= 1e-8
    print(f"two-grid factor Jacobi {lj:.4f} learned {ll:.4f}; FCG iterations Jacobi {ij['iters']} "
          f"learned {il['iters']}")
    assert il["iters"] < ij["iters"]
