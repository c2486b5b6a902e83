"""Values-only re-setup (Sec. 3.1: the hierarchy's pattern depends only on the
aggregates and the pattern of A_0, so the Galerkin products can be repeated
from stored summation plans).

New values 4 A with the diagonal scaled by 1.5 keep the strength graph, the MIS
priorities and hence the aggregates (strength compares off-diagonal ratios;
scaling by 4 is exact), so a fresh setup on the new values must find the same
hierarchy: the re-setup has to match it bit for bit, level by level, and so
must the oracle's hierarchy of the new matrix."""
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


def new_values(A):
    v = 4.0 * A.val
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    v[A.col == rows] *= 1.5
    return v


def levels(amg, h):
    return [amg.amg_export_level(h, k) for k in range(len(amg.amg_hierarchy_info(h)))]


def assert_same(la, lb):
    assert len(la) == len(lb)
    for a, b in zip(la, lb):
        for key in ("rowptr", "col", "val", "B"):
            assert np.array_equal(a[key], b[key]), key
        assert (a["agg"] is None) == (b["agg"] is None)
        if a["agg"] is not None:
            assert np.array_equal(a["agg"], b["agg"]) and np.array_equal(a["P"], b["P"])
        assert a["omega"] == b["omega"]


CASES = {
    "varcoef3d_16": (lambda: P.varcoef3d(16, 2, block=4), 0.5, 0),
    "poisson2d_37": (lambda: P.poisson2d(37), 0.25, 1),
    "fem2d_48": (lambda: P.fem2d(48, 5), 0.25, 2),
}


@pytest.mark.parametrize("name", list(CASES))
def test_resetup_equals_full_setup_and_oracle(env, name):
    amg, oracle = env
    make, alpha, prec = CASES[name]
    A = make()
    A2 = P.CSR(A.n, A.rowptr, A.col, new_values(A))
    p = amg.amg_default_params(alpha=alpha, seed=5, precision=prec)
    h = amg.amg_setup(A.rowptr, A.col, A.val, p)
    hf = amg.amg_setup(A2.rowptr, A2.col, A2.val, p)
    try:
        amg.amg_resetup_values(h, A2.val)
        lr, lf = levels(amg, h), levels(amg, hf)
        assert_same(lr, lf)
        o = oracle.Hierarchy(A2, alpha=alpha, seed=5)
        for k, lv in enumerate(lr):
            ol = o.level(k)
            assert np.array_equal(lv["col"], ol.col) and np.array_equal(lv["val"], ol.val), k
        b = P.rhs_uniform(A.n, 23)
        xr, xf = np.zeros(A.n), np.zeros(A.n)
        _, ir, _ = amg.amg_solve(h, b, xr, 1e-8)
        _, i_f, _ = amg.amg_solve(hf, b, xf, 1e-8)
        assert ir == i_f and np.array_equal(xr, xf)
    finally:
        amg.amg_free(h)
        amg.amg_free(hf)


def test_resetup_with_the_same_values_changes_nothing_and_is_fast(env):
    amg, _ = env
    A = P.poisson3d(40)
    p = amg.amg_default_params(alpha=0.5, seed=1, precision=1)
    h = amg.amg_setup(A.rowptr, A.col, A.val, p)
    try:
        before = levels(amg, h)
        setup_ms = amg.amg_last_solve_info(h)["setup_ms"]
        b = P.rhs_uniform(A.n, 3)
        x0 = np.zeros(A.n)
        _, i0, _ = amg.amg_solve(h, b, x0, 1e-8)  # captures the solve graph
        amg.amg_resetup_values(h, A.val)
        resetup_ms = amg.amg_last_solve_info(h)["setup_ms"]
        assert_same(levels(amg, h), before)
        x1 = np.zeros(A.n)
        _, i1, _ = amg.amg_solve(h, b, x1, 1e-8)  # the captured graph still holds
        assert i1 == i0 and np.array_equal(x1, x0)
        print(f"setup {setup_ms:.2f} ms, values-only re-setup {resetup_ms:.2f} ms")
        assert resetup_ms < setup_ms
    finally:
        amg.amg_free(h)


def test_resetup_of_a_batch(env):
    amg, _ = env
    mats = [P.varcoef2d(m, 70 + q) for q, m in enumerate([25, 41, 18])]
    new = [P.CSR(A.n, A.rowptr, A.col, new_values(A)) for A in mats]
    p = amg.amg_default_params(alpha=0.25, seed=2, precision=1)
    h = amg.amg_setup_batch(mats, p)
    hf = amg.amg_setup_batch(new, p)
    try:
        amg.amg_resetup_values(h, np.concatenate([A.val for A in new]))
        assert_same(levels(amg, h), levels(amg, hf))
        b = np.concatenate([P.rhs_uniform(A.n, 80 + q) for q, A in enumerate(mats)])
        xr, xf = np.zeros_like(b), np.zeros_like(b)
        _, ir, _ = amg.amg_solve_batch(h, b, xr, 1e-8, len(mats))
        _, i_f, _ = amg.amg_solve_batch(hf, b, xf, 1e-8, len(mats))
        assert np.array_equal(ir, i_f) and np.array_equal(xr, xf)
    finally:
        amg.amg_free(h)
        amg.amg_free(hf)


def test_resetup_rejects_bad_values(env):
    amg, _ = env
    A = P.poisson2d(20)
    h = amg.amg_setup(A.rowptr, A.col, A.val, amg.amg_default_params())
    try:
        bad = A.val.copy()
        bad[3] = np.nan
        with pytest.raises(amg.AMGError) as e:
            amg.amg_resetup_values(h, bad)
        assert e.value.code == amg.AMG_ERR_BAD_INPUT
    finally:
        amg.amg_free(h)
