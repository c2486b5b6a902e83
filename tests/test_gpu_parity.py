"""GPU path against the FP64 CPU oracle, through the C ABI.

Integer results (aggregates, coarse sparsity) and the FP64 hierarchy values must
be bit-identical; FP64 solutions within 1e-10 relative (iterates compared after
the same number of outer iterations, so that the stopping test cannot pick
different iterations); reduced-precision preconditioners must still reach the
FP64 residual tolerance.
"""
import numpy as np
import pytest

from paper_1403_1649_gb300 import problems as P

pytestmark = pytest.mark.gpu

CASES = {
    # 2D 5-point Poisson 64x64 (the small workload; oracle runs in milliseconds)
    "poisson2d_64": lambda: (P.poisson2d(64), 0.25, 0),
    # 37^2 = 1369 rows: ragged last slice, several SELL slices
    "poisson2d_37": lambda: (P.poisson2d(37), 0.25, 5),
    "varcoef2d_50": lambda: (P.varcoef2d(50, 7), 0.25, 7),
    "aniso2d_40": lambda: (P.aniso2d(40, 0.05), 0.25, 9),
    "poisson3d_20": lambda: (P.poisson3d(20), 0.5, 1),
    "varcoef3d_24": lambda: (P.varcoef3d(24, 2), 0.5, 2),
    "varcoef3d_16": lambda: (P.varcoef3d(16, 2, block=4), 0.5, 2),
    "fem2d_48": lambda: (P.fem2d(48, 3), 0.25, 3),
}

_cache = {}


def case(name):
    if name not in _cache:
        _cache[name] = CASES[name]()
    return _cache[name]


@pytest.fixture(scope="session")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1649_gb300 import amg, build
    build.build()
    amg.lib()
    return amg


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def pair(gpu, orc, name, **kw):
    A, alpha, seed = case(name)
    g = gpu.Hierarchy(A, alpha=alpha, seed=seed, **kw)
    okw = {k: v for k, v in kw.items() if k in ("coarse_max", "max_levels", "kcycle_levels", "kcycle_t",
                                                 "omega_mode", "omega", "outer", "restart")}
    o = orc.Hierarchy(A, alpha=alpha, seed=seed, **okw)
    return A, g, o


@pytest.mark.parametrize("name", list(CASES))
def test_hierarchy_bit_exact(gpu, orc, name):
    A, g, o = pair(gpu, orc, name)
    assert g.nlevels == o.nlevels
    for k in range(o.nlevels):
        gl, ol = g.level(k), o.level(k)
        assert gl["n"] == ol.n and gl["nnz"] == ol.nnz, k
        assert np.array_equal(gl["rowptr"], ol.rowptr), k
        assert np.array_equal(gl["col"], ol.col), k
        assert np.array_equal(gl["val"], ol.val), k  # keyed sum in the same order: identical values
        assert np.array_equal(gl["B"], ol.B), k
        if k < o.nlevels - 1:
            assert np.array_equal(gl["agg"], ol.agg), k
            assert np.array_equal(gl["P"], ol.P), k
            assert gl["mis_rounds"] == ol.mis_rounds, k
            assert gl["omega"] == pytest.approx(ol.omega, rel=1e-12), k


@pytest.mark.parametrize("name", list(CASES))
def test_preconditioner_parity(gpu, orc, name):
    A, g, o = pair(gpu, orc, name)
    b = P.rhs_uniform(A.n, 11)
    zg, zo = g.precond(b), o.precond(b)
    assert np.linalg.norm(zg - zo) <= 1e-11 * np.linalg.norm(zo)


@pytest.mark.parametrize("name,cmax", [("poisson2d_64", 600), ("varcoef3d_24", 600), ("fem2d_48", 400),
                                       ("poisson3d_20", 600)])
def test_large_coarsest_level(gpu, orc, name, cmax):
    """A coarsest level of more than 64 rows (the paper keeps about 600 on the
    GPU, Sec. 3): its inverse comes from the blocked Gauss-Jordan sweeps spread
    over the whole GPU, one launch per 16 pivots.  Same hierarchy as the oracle (whose
    coarsest solve is a Cholesky factorisation), preconditioner to 1e-11 and six
    outer iterations to 1e-10."""
    A, g, o = pair(gpu, orc, name, coarse_max=cmax, max_iter=6)
    nl = g.level(g.nlevels - 1)["n"]
    assert 64 < nl <= cmax and o.nlevels == g.nlevels and o.level(o.nlevels - 1).n == nl
    b = P.rhs_uniform(A.n, 13)
    zg, zo = g.precond(b), o.precond(b)
    assert np.linalg.norm(zg - zo) <= 1e-11 * np.linalg.norm(zo)
    xg, ig = g.solve(b, tol=0.0, allow=(gpu.AMG_OK, gpu.AMG_ERR_NOT_CONVERGED))
    xo, io = o.solve(b, tol=0.0, max_iter=6)
    assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("name", list(CASES))
def test_solve_iterates_parity(gpu, orc, name):
    A, g, o = pair(gpu, orc, name, max_iter=6)
    b = P.rhs_uniform(A.n, 12)
    xg, ig = g.solve(b, tol=0.0, allow=(gpu.AMG_OK, gpu.AMG_ERR_NOT_CONVERGED))
    xo, io = o.solve(b, tol=0.0, max_iter=6)
    assert ig["iters"] == io["iters"] == 6
    assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo)
    assert np.allclose(ig["hist"], io["hist"], rtol=1e-9, atol=0)


@pytest.mark.parametrize("name", list(CASES))
def test_solve_converges_like_oracle(gpu, orc, name):
    A, g, o = pair(gpu, orc, name)
    b = P.rhs_uniform(A.n, 13)
    xg, ig = g.solve(b, tol=1e-8)
    xo, io = o.solve(b, tol=1e-8, max_iter=500)
    assert ig["status"] == gpu.AMG_OK and ig["final_relres"] <= 1e-8
    assert abs(ig["iters"] - io["iters"]) <= 1
    r = b - A.matvec(xg)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    if ig["iters"] == io["iters"]:
        assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("name", ["poisson3d_20", "varcoef3d_24", "fem2d_48", "aniso2d_40"])
@pytest.mark.parametrize("outer", [0, 1])
def test_cycle_trace_matches_oracle(gpu, orc, name, outer):
    """The cycle as run: per level the visits, the Alg. 5 coarse parts and the
    second inner steps they took (||r~|| > t ||r||), counted on the device during
    an FP64 solve to 1e-8, equal the oracle's counts for the same solve."""
    A, g, o = pair(gpu, orc, name, outer=outer, restart=30)
    b = P.rhs_uniform(A.n, 27)
    xg, ig = g.solve(b, tol=1e-8)
    xo, io = o.solve(b, tol=1e-8, max_iter=500)
    assert ig["iters"] == io["iters"]
    tg, to = gpu.amg_cycle_trace(g.h), o.cycle_trace()
    for key in ("visits", "kcalls", "second"):
        assert np.array_equal(tg[key], to[key]), (key, tg[key], to[key])
    assert tg["visits"][0] == ig["iters"] and tg["second"].sum() > 0
    g.precond(b)
    o.precond(b)
    tg, to = gpu.amg_cycle_trace(g.h), o.cycle_trace()
    assert all(np.array_equal(tg[k], to[k]) for k in tg) and tg["visits"][0] == 1


@pytest.mark.parametrize("name", ["poisson2d_37", "varcoef3d_24", "fem2d_48"])
def test_spmv_every_level(gpu, orc, name):
    import torch
    A, g, o = pair(gpu, orc, name)
    for k in range(g.nlevels):
        L = g.level(k)
        Ak = P.CSR(L["n"], L["rowptr"], L["col"], L["val"])
        x = P.rhs_uniform(Ak.n, 20 + k)
        xd = torch.from_numpy(x).cuda()
        yd = torch.zeros_like(xd)
        gpu.amg_spmv(g.h, k, xd, yd)
        torch.cuda.synchronize()
        ref = Ak.matvec(x)
        assert np.abs(yd.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


def reduced_spmv_bound(A, x, u):
    """Per-row bound on |y - A x| for the reduced-precision SELL product: values
    rounded to a unit roundoff u with the rounding errors moved onto a
    compensated diagonal (so the product differs from A x by
    sum_j (a_ij - fl(a_ij)) (x_j - x_i)), FP32 accumulation of the row and an
    FP32 diagonal."""
    u32 = 2.0 ** -24
    n = A.n
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    off = A.col != rows
    absterm = np.abs(A.val) * np.abs(x[A.col])
    acc = np.bincount(rows, weights=absterm, minlength=n)
    comp = np.bincount(rows[off], weights=(np.abs(A.val) * (np.abs(x[A.col]) + np.abs(x[rows])))[off], minlength=n)
    width = np.diff(A.rowptr).astype(np.float64)
    return (width + 4) * u32 * acc + u * comp + 1e-300


@pytest.mark.parametrize("prec,grid", [(1, 128), (2, 128)])
def test_reduced_precision_level0_spmv_full_size(gpu, prec, grid):
    """The benchmarked level-0 product, at full size (128^3, 2,097,152 rows): the
    FP32 (and BF16) SELL kernel with its split diagonal against the FP64 CSR
    product of the same FP32 input vector, element by element, within the
    rounding bound of each row."""
    import torch
    A = P.poisson3d(grid)
    g = gpu.Hierarchy(A, alpha=0.5, seed=1, precision=prec)
    x = (P.rhs_uniform(A.n, 22)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    gpu.amg_spmv(g.h, 0, xd, yd)
    torch.cuda.synchronize()
    x64 = x.astype(np.float64)
    ref = A.matvec(x64)
    u = 2.0 ** -24 if prec == 1 else 2.0 ** -8
    err = np.abs(yd.cpu().numpy().astype(np.float64) - ref)
    bound = reduced_spmv_bound(A, x64, u)
    assert (err <= bound).all(), (err / bound).max()


def irregular_spd(n=1013, iso=40, seed=11):
    """A symmetric, diagonally dominant matrix whose rows have 0 to ~20
    off-diagonal entries, so that SELL slices get odd and even widths, rows
    shorter than their slice's longest, a ragged last slice, and (the last
    `iso` rows have no neighbours) a slice without off-diagonal entries."""
    m = n - iso
    deg = (P.uniform01(seed, 0, m) * 10).astype(np.int64)
    src = np.repeat(np.arange(m), deg)
    dst = (P.uniform01(seed, 1, src.size) * m).astype(np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    w = -(0.5 + P.uniform01(seed, 2, src.size))
    a = {}
    for i, j, v in zip(src.tolist(), dst.tolist(), w.tolist()):
        key = (min(i, j), max(i, j))
        a[key] = a.get(key, 0.0) + v
    rows = [[] for _ in range(n)]
    for (i, j), v in a.items():
        rows[i].append((j, v))
        rows[j].append((i, v))
    rp, ci, va = [0], [], []
    for i in range(n):
        d = 1.0 + sum(abs(v) for _, v in rows[i])
        ent = sorted(rows[i] + [(i, d)])
        ci += [j for j, _ in ent]
        va += [v for _, v in ent]
        rp.append(len(ci))
    return P.CSR(n, np.array(rp, np.int32), np.array(ci, np.int32), np.array(va, np.float64))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_spmv_irregular_rows(gpu, prec):
    """Level-0 product on rows of irregular length in every precision: FP32
    values take the {column, value} pair layout with even slice widths and the
    predicated step (only 6-wide slices take the unpredicated one), BF16 and
    FP64 the column and value arrays; an all-diagonal slice and the ragged last
    slice included.  The stored SELL passes the library's own structural check."""
    import torch
    A = irregular_spd()
    lens = np.diff(A.rowptr) - 1
    widths = np.array([lens[q:q + 32].max() for q in range(0, A.n, 32)])
    assert (widths % 2 == 1).any() and (widths % 2 == 0).any() and widths[-1] == 0 and A.n % 32
    g = gpu.Hierarchy(A, alpha=0.25, seed=3, precision=prec)
    assert gpu.lib().amg_validate_hierarchy(g.h) == 0, gpu.amg_last_error()
    vt = np.float64 if prec == 0 else np.float32
    x = P.rhs_uniform(A.n, 41).astype(vt)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    gpu.amg_spmv(g.h, 0, xd, yd)
    torch.cuda.synchronize()
    x64 = x.astype(np.float64)
    ref = A.matvec(x64)
    err = np.abs(yd.cpu().numpy().astype(np.float64) - ref)
    if prec == 0:
        assert err.max() <= 1e-14 * np.abs(ref).max()
    else:
        bound = reduced_spmv_bound(A, x64, 2.0 ** -24 if prec == 1 else 2.0 ** -8)
        assert (err <= bound).all(), (err / bound).max()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", ["varcoef3d_24", "fem2d_48"])
def test_reduced_precision_spmv_every_level_varcoef(gpu, orc, prec, name):
    """Reduced-precision products of every level of a variable-coefficient
    hierarchy (values not exact in FP32 / BF16, so the compensated diagonal is
    exercised), element by element within the rounding bound.  The FEM level 0
    has slices of 6 and 8 entries a row, which take the unpredicated steps."""
    import torch
    A, alpha, seed = case(name)
    g = gpu.Hierarchy(A, alpha=alpha, seed=seed, precision=prec)
    u = 2.0 ** -24 if prec == 1 else 2.0 ** -8
    for k in range(g.nlevels):
        L = g.level(k)
        Ak = P.CSR(L["n"], L["rowptr"], L["col"], L["val"])
        x = P.rhs_uniform(Ak.n, 30 + k).astype(np.float32)
        xd = torch.from_numpy(x).cuda()
        yd = torch.zeros_like(xd)
        gpu.amg_spmv(g.h, k, xd, yd)
        torch.cuda.synchronize()
        x64 = x.astype(np.float64)
        err = np.abs(yd.cpu().numpy().astype(np.float64) - Ak.matvec(x64))
        bound = reduced_spmv_bound(Ak, x64, u)
        assert (err <= bound).all(), (k, (err / bound).max())


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_precision_reaches_fp64_tolerance(gpu, orc, prec):
    A, g, o = pair(gpu, orc, "varcoef3d_16", precision=prec)
    b = P.rhs_uniform(A.n, 14)
    xg, ig = g.solve(b, tol=1e-8)
    assert ig["status"] == gpu.AMG_OK and ig["final_relres"] <= 1e-8
    xo, io = o.solve(b, tol=1e-12, max_iter=500)
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    ev = np.linalg.eigvalsh(A.to_dense())
    kappa = ev[-1] / ev[0]
    assert err <= kappa * 1e-8
    print(f"precision {prec}: {ig['iters']} iterations (fp64 oracle {io['iters']} to 1e-12), "
          f"rel. error vs FP64 oracle {err:.2e}")


@pytest.mark.parametrize("name", ["varcoef3d_16", "varcoef2d_50"])
def test_fgmres_iterates_parity_across_restart(gpu, orc, name):
    A, g, o = pair(gpu, orc, name, outer=1, restart=5, max_iter=8)
    b = P.rhs_uniform(A.n, 15)
    xg, ig = g.solve(b, tol=0.0, allow=(gpu.AMG_OK, gpu.AMG_ERR_NOT_CONVERGED))
    xo, io = o.solve(b, tol=0.0, max_iter=8)
    assert ig["iters"] == io["iters"] == 8
    assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo)
    assert np.allclose(ig["hist"], io["hist"], rtol=1e-8, atol=0)


def test_fgmres_converges(gpu, orc):
    A, g, o = pair(gpu, orc, "varcoef3d_24", outer=1, restart=30)
    b = P.rhs_uniform(A.n, 16)
    xg, ig = g.solve(b, tol=1e-8)
    xo, io = o.solve(b, tol=1e-8, max_iter=500)
    assert ig["status"] == gpu.AMG_OK and ig["final_relres"] <= 1e-8
    assert abs(ig["iters"] - io["iters"]) <= 1
    hist = ig["hist"]
    assert all(b_ <= a_ * (1 + 1e-9) for a_, b_ in zip(hist[:30], hist[1:30]))  # monotone within a cycle


@pytest.mark.parametrize("name", ["fem2d_48", "varcoef3d_16"])
def test_polynomial_smoother_parity(gpu, orc, name):
    """Per-row polynomial smoother (pre: sum_q diag(c_q)(D^-1A)^q D^-1, post: its
    transpose) against the oracle with the same coefficients on every level."""
    A, g, o = pair(gpu, orc, name, smoother=1, max_iter=5)
    rng = np.random.default_rng(9)
    for k in range(g.nlevels - 1):
        n = g.level(k)["n"]
        coef = np.column_stack([rng.uniform(0.3, 0.7, n), rng.uniform(-0.2, 0.2, n), rng.uniform(-0.1, 0.1, n)])
        gpu.amg_set_poly(g.h, k, coef)
        o.set_poly(k, coef)
    b = P.rhs_uniform(A.n, 17)
    zg, zo = g.precond(b), o.precond(b)
    assert np.linalg.norm(zg - zo) <= 1e-11 * np.linalg.norm(zo)
    xg, ig = g.solve(b, tol=0.0, allow=(gpu.AMG_OK, gpu.AMG_ERR_NOT_CONVERGED))
    xo, io = o.solve(b, tol=0.0, max_iter=g.params.max_iter)
    assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)


def test_polynomial_smoother_reduces_to_jacobi(gpu, orc):
    A, g, _ = pair(gpu, orc, "varcoef2d_50", smoother=1)
    b = P.rhs_uniform(A.n, 18)
    z_j = g.precond(b)  # no coefficients set yet: damped Jacobi on every level
    for k in range(g.nlevels - 1):
        L = g.level(k)
        gpu.amg_set_poly(g.h, k, np.tile([L["omega"], 0.0, 0.0], (L["n"], 1)))
    assert np.allclose(g.precond(b), z_j, rtol=1e-12, atol=1e-14 * np.abs(z_j).max())
    # a cleared level runs damped Jacobi again: bit-identical to never having set it
    for k in range(g.nlevels - 1):
        gpu.amg_set_poly(g.h, k, np.tile([0.3, 0.1, 0.05], (g.level(k)["n"], 1)))
    assert not np.array_equal(g.precond(b), z_j)
    for k in range(g.nlevels - 1):
        gpu.amg_set_poly(g.h, k, None)
    assert np.array_equal(g.precond(b), z_j)


@pytest.mark.parametrize("tail", [1, 2])
@pytest.mark.parametrize("name,prec", [("varcoef3d_24", 0), ("poisson2d_64", 0), ("fem2d_48", 1)])
def test_cluster_tail_matches_kernel_per_step(gpu, name, prec, tail):
    """The coarse levels run as one launch (a cluster of 8 blocks, or a single
    block) or as one kernel per step: same preconditioner up to rounding, same
    iterations."""
    A, alpha, seed = case(name)
    b = P.rhs_uniform(A.n, 19)
    g1 = gpu.Hierarchy(A, alpha=alpha, seed=seed, precision=prec, tail=tail)
    g0 = gpu.Hierarchy(A, alpha=alpha, seed=seed, precision=prec, tail=0)
    z1, z0 = g1.precond(b), g0.precond(b)
    tol = 1e-12 if prec == 0 else 1e-5
    assert np.linalg.norm(z1 - z0) <= tol * np.linalg.norm(z0)
    x1, i1 = g1.solve(b, tol=1e-8)
    x0, i0 = g0.solve(b, tol=1e-8)
    assert abs(i1["iters"] - i0["iters"]) <= (0 if prec == 0 else 1)
    assert i1["final_relres"] <= 1e-8 and i1["kernel_launches"] < i0["kernel_launches"]


@pytest.mark.parametrize("prec", [0, 1])
def test_programmatic_dependent_launch_changes_nothing(gpu, prec):
    """Launching with programmatic dependent launch only changes scheduling:
    the solution is bit-identical."""
    A, alpha, seed = case("varcoef3d_24")
    b = P.rhs_uniform(A.n, 20)
    xa, ia = gpu.Hierarchy(A, alpha=alpha, seed=seed, precision=prec, pdl=1).solve(b, tol=1e-8)
    xb, ib = gpu.Hierarchy(A, alpha=alpha, seed=seed, precision=prec, pdl=0).solve(b, tol=1e-8)
    assert ia["iters"] == ib["iters"] and np.array_equal(xa, xb)


@pytest.mark.parametrize("prec", [0, 1])
def test_autotuned_spmv_grid_changes_only_rounding(gpu, orc, prec):
    """The autotuner picks each level's SpMV grid among multiples of the SM count
    (at most the partial-sum capacity); the hierarchy is the same, and the tuned
    solve reaches the tolerance in the same number of iterations (FP64: within
    1e-10 of the untuned solution)."""
    A, alpha, seed = case("varcoef3d_24")
    b = P.rhs_uniform(A.n, 21)
    gt = gpu.Hierarchy(A, alpha=alpha, seed=seed, precision=prec, autotune=1)
    g0 = gpu.Hierarchy(A, alpha=alpha, seed=seed, precision=prec)
    for lt, l0 in zip(gt.info(), g0.info()):
        assert lt["n"] == l0["n"] and lt["nnz"] == l0["nnz"] and lt["seg_tile"] == 0
        nsl = (lt["n"] + 31) // 32
        assert 1 <= lt["spmv_blocks"] <= min(1216, max(1, (nsl + 7) // 8))
        assert l0["spmv_blocks"] == min(608, max(1, (nsl + 7) // 8))
    xt, it = gt.solve(b, tol=1e-8)
    x0, i0 = g0.solve(b, tol=1e-8)
    assert abs(it["iters"] - i0["iters"]) <= (0 if prec == 0 else 1) and it["final_relres"] <= 1e-8
    if prec == 0:
        assert np.linalg.norm(xt - x0) <= 1e-10 * np.linalg.norm(x0)


def test_single_level_one_iteration(gpu):
    A = P.poisson2d(7)
    g = gpu.Hierarchy(A, coarse_max=64)
    assert g.nlevels == 1
    x, info = g.solve(P.rhs_uniform(A.n, 1), tol=1e-12)
    assert info["iters"] == 1 and info["final_relres"] <= 1e-12


def test_bad_inputs_rejected(gpu):
    A = P.poisson1d(50)
    bad = P.CSR(A.n, A.rowptr, A.col, A.val.copy())
    bad.val[0] = 0.0
    with pytest.raises(gpu.AMGError) as e:
        gpu.Hierarchy(bad)
    assert e.value.code == gpu.AMG_ERR_BAD_INPUT and "diagonal" in gpu.amg_last_error()
    uns = P.CSR(A.n, A.rowptr, A.col.copy(), A.val)
    uns.col[1], uns.col[2] = uns.col[2], uns.col[1]
    with pytest.raises(gpu.AMGError) as e:
        gpu.Hierarchy(uns)
    assert e.value.code == gpu.AMG_ERR_BAD_INPUT
    nanv = P.CSR(A.n, A.rowptr, A.col, A.val.copy())
    nanv.val[5] = np.nan
    with pytest.raises(gpu.AMGError):
        gpu.Hierarchy(nanv)
    g = gpu.Hierarchy(A)
    xh, yh = np.ones(A.n), np.zeros(A.n)
    with pytest.raises(gpu.AMGError) as e:  # amg_spmv takes device pointers only
        gpu.amg_spmv(g.h, 0, xh, yh)
    assert e.value.code == gpu.AMG_ERR_BAD_INPUT and "device" in gpu.amg_last_error()


def test_not_converged_and_zero_rhs(gpu):
    A = P.varcoef2d(40, 3)
    g = gpu.Hierarchy(A, max_iter=2)
    x, info = g.solve(P.rhs_uniform(A.n, 2), tol=1e-14, allow=(gpu.AMG_OK, gpu.AMG_ERR_NOT_CONVERGED))
    assert info["status"] == gpu.AMG_ERR_NOT_CONVERGED and info["iters"] == 2 and len(info["hist"]) == 3
    x, info = g.solve(np.zeros(A.n), tol=1e-8)
    assert info["status"] == gpu.AMG_OK and info["iters"] == 0 and not x.any()


def test_true_residual_check_and_refinement(gpu):
    """A tolerance near the FP64 floor: the recursively updated residual meets it
    before the true residual does, so the solve checks the true residual and
    restarts flexible CG from it (iterative refinement) until the true residual
    meets the tolerance or the iteration cap ends the solve."""
    A = P.poisson2d(37)
    b = P.rhs_uniform(A.n, 6)
    for prec in (0, 1):
        g = gpu.Hierarchy(A, alpha=0.25, seed=5, precision=prec, max_iter=60)
        x, info = g.solve(b, tol=1e-14, allow=(gpu.AMG_OK, gpu.AMG_ERR_NOT_CONVERGED))
        true_rel = np.linalg.norm(b - A.matvec(x)) / np.linalg.norm(b)
        assert len(info["hist"]) == info["iters"] + 1 <= 61
        assert abs(info["final_relres"] - true_rel) <= 5e-15 + 0.5 * true_rel
        if info["status"] == gpu.AMG_OK:
            assert info["final_relres"] <= 1e-14
        else:
            assert info["iters"] == 60 and true_rel < 1e-12
        print(f"precision {prec}: status {info['status']}, {info['iters']} iterations, true relres {true_rel:.2e}")


def test_device_and_host_buffers_agree(gpu):
    import torch
    A, alpha, seed = case("poisson3d_20")
    g = gpu.Hierarchy(A, alpha=alpha, seed=seed)
    b = P.rhs_uniform(A.n, 3)
    xh, _ = g.solve(b, tol=1e-8)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    gpu.amg_solve(g.h, bd, xd, 1e-8, g.params.max_iter)
    torch.cuda.synchronize()
    assert np.array_equal(xd.cpu().numpy(), xh)


def test_graph_and_stream_launches_agree(gpu):
    A, alpha, seed = case("varcoef2d_50")
    b = P.rhs_uniform(A.n, 4)
    xg, ig = gpu.Hierarchy(A, alpha=alpha, seed=seed, use_graph=1).solve(b, tol=1e-8)
    xs, is_ = gpu.Hierarchy(A, alpha=alpha, seed=seed, use_graph=0).solve(b, tol=1e-8)
    assert ig["iters"] == is_["iters"] and np.array_equal(xg, xs)
    assert ig["kernel_launches"] == is_["kernel_launches"] > 0


@pytest.mark.slow
def test_full_size_poisson3d_128(gpu, orc):
    """128^3 7-point Poisson at full size in the benchmark's configuration: the
    whole hierarchy bit-exact and six FP64 iterations within 1e-10."""
    A = P.poisson3d(128)
    g = gpu.Hierarchy(A, alpha=0.5, seed=1, max_iter=6)
    o = orc.Hierarchy(A, alpha=0.5, seed=1)
    assert g.nlevels == o.nlevels
    for k in range(o.nlevels):
        gl, ol = g.level(k), o.level(k)
        assert np.array_equal(gl["col"], ol.col) and np.array_equal(gl["val"], ol.val), k
        if k < o.nlevels - 1:
            assert np.array_equal(gl["agg"], ol.agg), k
    b = P.rhs_uniform(A.n, 1)
    xg, ig = g.solve(b, tol=0.0, allow=(gpu.AMG_OK, gpu.AMG_ERR_NOT_CONVERGED))
    xo, io = o.solve(b, tol=0.0, max_iter=6)
    assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo)
