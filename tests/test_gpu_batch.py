"""Batches of independent systems in one block-diagonal hierarchy (GPU).

A batch of one system reproduces the single-system hierarchy bit for bit and,
in FP64, its iterates; an FP64 batch of systems of different sizes has the
oracle's hierarchy of the same block-diagonal matrix, and every system follows
the oracle's solve of that system alone (on its part of the hierarchy) iterate
for iterate; every system reaches the FP64 tolerance on its own, and a
converged system stops changing."""
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
    return amg, oracle


def level_arrays(amg, h, k):
    return amg.amg_export_level(h, k)


def test_batch_hierarchy_index_arrays_valid(env):
    amg, _ = env
    for mats in ([P.varcoef2d(45, 5)], [P.varcoef2d(m, 40 + q) for q, m in enumerate([20, 33, 47, 12, 60, 8, 29])]):
        for prec, seed in ((0, 3), (1, 1)):
            h = amg.amg_setup_batch(mats, amg.amg_default_params(alpha=0.25, seed=seed, precision=prec))
            try:
                rc = amg.lib().amg_validate_hierarchy(h)
                assert rc == 0, amg.amg_last_error()
            finally:
                amg.amg_free(h)
    A = P.varcoef3d(16, 2, block=4)
    h = amg.amg_setup(A.rowptr, A.col, A.val, amg.amg_default_params(alpha=0.5))
    try:
        assert amg.lib().amg_validate_hierarchy(h) == 0, amg.amg_last_error()
    finally:
        amg.amg_free(h)


def test_batch_fp64_iterates_match_oracle_per_system(env):
    """An FP64 batch of seven systems of uneven size, one with a zero right-hand
    side, run for six outer iterations.  The batch hierarchy equals the oracle's
    hierarchy of the same block-diagonal matrix bit for bit (same depth), and
    every system's iterate and final FP64 residual equal those of the oracle
    solving that system alone on its own part of that hierarchy, to 1e-10 and
    1e-9: the per-system inner products, step lengths and Alg. 5 branches of the
    batch are those of independent solves."""
    amg, oracle = env
    sides = [20, 33, 47, 12, 60, 8, 29]
    mats = [P.varcoef2d(m, 40 + q) for q, m in enumerate(sides)]
    rhs = [P.rhs_uniform(A.n, 70 + q) for q, A in enumerate(mats)]
    rhs[2][:] = 0.0
    b = np.concatenate(rhs)
    h = amg.amg_setup_batch(mats, amg.amg_default_params(alpha=0.25, seed=1, precision=0, max_iter=6))
    try:
        nl = len(amg.amg_hierarchy_info(h))
        o = oracle.Hierarchy(P.block_diag(mats), alpha=0.25, seed=1, max_levels=nl)
        assert o.nlevels == nl
        for k in range(nl):
            gl, ol = amg.amg_export_level(h, k), o.level(k)
            assert np.array_equal(gl["col"], ol.col) and np.array_equal(gl["val"], ol.val), k
            if k < nl - 1:
                assert np.array_equal(gl["agg"], ol.agg) and np.array_equal(gl["P"], ol.P), k
                assert gl["omega"] == pytest.approx(ol.omega, rel=1e-12), k
        x = np.zeros_like(b)
        rc, it, rel = amg.amg_solve_batch(h, b, x, 0.0, len(mats), allow=(amg.AMG_OK, amg.AMG_ERR_NOT_CONVERGED))
        off = np.cumsum([0] + [A.n for A in mats])
        for q, A in enumerate(mats):
            xs = x[off[q]:off[q + 1]]
            if not rhs[q].any():
                assert it[q] == 0 and not xs.any()
                continue
            sub = o.subsystem(int(off[q]), int(off[q + 1]))
            xo, io = sub.solve(rhs[q], tol=0.0, max_iter=6)
            assert it[q] == io["iters"] == 6, q
            assert np.linalg.norm(xs - xo) <= 1e-10 * np.linalg.norm(xo), q
            assert rel[q] == pytest.approx(io["relres"], rel=1e-9), q
    finally:
        amg.amg_free(h)


def test_batch_of_one_fp64_iterates_equal_single_system(env):
    """In FP64 a batch of one follows the single-system solve iterate for
    iterate: six outer iterations agree to 1e-12 (the batch sums its inner
    products per system tile, the single system inside the SpMV kernels)."""
    amg, _ = env
    A = P.varcoef2d(45, 5)
    b = P.rhs_uniform(A.n, 5)
    p = amg.amg_default_params(alpha=0.25, seed=3, precision=0, max_iter=6)
    hb = amg.amg_setup_batch([A], p)
    hs = amg.amg_setup(A.rowptr, A.col, A.val, p)
    try:
        allow = (amg.AMG_OK, amg.AMG_ERR_NOT_CONVERGED)
        xb = np.zeros(A.n)
        rc, it, rel = amg.amg_solve_batch(hb, b, xb, 0.0, 1, allow=allow)
        xs = np.zeros(A.n)
        rc2, its, hist = amg.amg_solve(hs, b, xs, 0.0, 6, allow=allow)
        assert int(it[0]) == its == 6
        assert np.linalg.norm(xb - xs) <= 1e-12 * np.linalg.norm(xs)
        assert rel[0] == pytest.approx(amg.amg_last_solve_info(hs)["final_relres"], rel=1e-10)
    finally:
        amg.amg_free(hb)
        amg.amg_free(hs)


def test_batch_of_one_equals_single_system(env):
    amg, _ = env
    A = P.varcoef2d(45, 5)
    b = P.rhs_uniform(A.n, 5)
    p = amg.amg_default_params(alpha=0.25, seed=3)
    hb = amg.amg_setup_batch([A], p)
    hs = amg.amg_setup(A.rowptr, A.col, A.val, p)
    try:
        nb, ns = len(amg.amg_hierarchy_info(hb)), len(amg.amg_hierarchy_info(hs))
        assert nb == ns
        for k in range(ns):
            lb, ls = level_arrays(amg, hb, k), level_arrays(amg, hs, k)
            assert np.array_equal(lb["col"], ls["col"]) and np.array_equal(lb["val"], ls["val"])
            if k < ns - 1:
                assert np.array_equal(lb["agg"], ls["agg"])
        xb = np.zeros(A.n)
        rc, it, rel = amg.amg_solve_batch(hb, b, xb, 1e-8, 1)
        xs = np.zeros(A.n)
        rc2, its, _ = amg.amg_solve(hs, b, xs, 1e-8, p.max_iter)
        assert rc == rc2 == amg.AMG_OK and abs(int(it[0]) - its) <= 1 and rel[0] <= 1e-8
        assert np.linalg.norm(xb - xs) <= 1e-6 * np.linalg.norm(xs)
    finally:
        amg.amg_free(hb)
        amg.amg_free(hs)


@pytest.mark.parametrize("prec", [0, 1])
def test_uneven_batch_each_system_converges(env, prec):
    amg, oracle = env
    sides = [20, 33, 47, 12, 60, 8, 29]
    mats = [P.varcoef2d(m, 40 + q) for q, m in enumerate(sides)]
    rhs = [P.rhs_uniform(A.n, 60 + q) for q, A in enumerate(mats)]
    rhs[3][:] = 0.0  # a system with a zero right-hand side
    b = np.concatenate(rhs)
    x = np.zeros_like(b)
    h = amg.amg_setup_batch(mats, amg.amg_default_params(alpha=0.25, seed=1, precision=prec))
    try:
        rc, it, rel = amg.amg_solve_batch(h, b, x, 1e-8, len(mats))
        assert rc == amg.AMG_OK
        off = np.cumsum([0] + [A.n for A in mats])
        for q, A in enumerate(mats):
            xs = x[off[q]:off[q + 1]]
            r = rhs[q] - A.matvec(xs)
            nb = np.linalg.norm(rhs[q])
            if nb == 0:
                assert it[q] == 0 and not xs.any()
                continue
            assert np.linalg.norm(r) <= 1e-8 * nb * (1 + 1e-6) and rel[q] <= 1e-8
            xo, _ = oracle.Hierarchy(A, alpha=0.25, seed=1).solve(rhs[q], tol=1e-12, max_iter=1000)
            ev = np.linalg.eigvalsh(A.to_dense())
            assert np.linalg.norm(xs - xo) <= (ev[-1] / ev[0]) * 1e-8 * np.linalg.norm(xo)
        print(f"precision {prec}: per-system iterations {it.tolist()}")
    finally:
        amg.amg_free(h)


def test_batch_status_codes_and_termination(env):
    """A batch whose systems all start converged stops at once with AMG_OK; a
    system that runs out of iterations reports AMG_ERR_NOT_CONVERGED after
    exactly max_iter iterations while the other reaches tol; a second solve on
    the same hierarchy repeats the first one bit for bit."""
    amg, _ = env
    mats = [P.varcoef2d(45, 5), P.poisson2d(20)]
    n = sum(A.n for A in mats)
    b = np.concatenate([P.rhs_uniform(A.n, 7 + q) for q, A in enumerate(mats)])
    h = amg.amg_setup_batch(mats, amg.amg_default_params(alpha=0.25, seed=3))
    try:
        x = np.zeros(n)
        rc, it, rel = amg.amg_solve_batch(h, np.zeros(n), x, 1e-8, 2)
        assert rc == amg.AMG_OK and (it == 0).all() and not x.any()
        rc, full, rel = amg.amg_solve_batch(h, b, np.zeros(n), 1e-8, 2)
        assert rc == amg.AMG_OK and (rel <= 1e-8).all() and full[1] < full[0]
    finally:
        amg.amg_free(h)
    cap = int(full[1] + full[0]) // 2
    h = amg.amg_setup_batch(mats, amg.amg_default_params(alpha=0.25, seed=3, max_iter=cap))
    try:
        allow = (amg.AMG_OK, amg.AMG_ERR_NOT_CONVERGED)
        x1 = np.zeros(n)
        rc, it, rel = amg.amg_solve_batch(h, b, x1, 1e-8, 2, allow=allow)
        assert rc == amg.AMG_ERR_NOT_CONVERGED and it[0] == cap and rel[0] > 1e-8
        assert it[1] == full[1] and rel[1] <= 1e-8
        x2 = np.zeros(n)
        rc2, it2, rel2 = amg.amg_solve_batch(h, b, x2, 1e-8, 2, allow=allow)
        assert rc2 == rc and np.array_equal(it2, it) and np.array_equal(x2, x1)
    finally:
        amg.amg_free(h)


def test_batch_autotuned_shapes(env):
    """With autotune the batch keeps its per-system results: the chosen row
    tiles are among the candidates, every system converges, and the iteration
    counts match the untuned batch."""
    amg, _ = env
    sides = [20, 33, 47, 12, 60, 8, 29]
    mats = [P.varcoef2d(m, 40 + q) for q, m in enumerate(sides)]
    b = np.concatenate([P.rhs_uniform(A.n, 60 + q) for q, A in enumerate(mats)])
    res = {}
    for tune in (0, 1):
        h = amg.amg_setup_batch(mats, amg.amg_default_params(alpha=0.25, seed=1, precision=1, autotune=tune))
        try:
            info = amg.amg_hierarchy_info(h)
            for k, lv in enumerate(info):
                assert lv["spmv_blocks"] >= 1
                assert lv["seg_tile"] in ((1024, 2048, 4096, 8192) if tune and k < len(info) - 1 else (2048,))
            x = np.zeros_like(b)
            rc, it, rel = amg.amg_solve_batch(h, b, x, 1e-8, len(mats))
            assert rc == amg.AMG_OK and (rel <= 1e-8).all()
            res[tune] = it
        finally:
            amg.amg_free(h)
    assert (np.abs(res[1] - res[0]) <= 1).all()


def test_batch_with_learned_smoother(env):
    amg, _ = env
    mats = [P.fem2d(m, 80 + q) for q, m in enumerate([24, 40, 16])]
    b = np.concatenate([P.rhs_uniform(A.n, 90 + q) for q, A in enumerate(mats)])
    x = np.zeros_like(b)
    h = amg.amg_setup_batch(mats, amg.amg_default_params(alpha=0.25, seed=1, precision=1, smoother=1,
                                                         omega_mode=1, omega=2.0 / 3.0))
    try:
        w16 = (np.random.default_rng(0).normal(size=5443) * 0.02).astype(np.float16).view(np.uint16)
        assert amg.lib().amg_apply_learned_smoother(h, w16.ctypes.data, None) == 0
        rc, it, rel = amg.amg_solve_batch(h, b, x, 1e-8, len(mats))
        assert rc == amg.AMG_OK and (rel <= 1e-8).all()
    finally:
        amg.amg_free(h)
