"""Aggressive coarsening with MIS(k) roots (Sec. 2.1.2: MIS(2) is the default,
k > 2 coarsens more aggressively at the cost of interpolation quality): k max
rounds per PMIS iteration and aggregation passes out to distance k.  The GPU
hierarchy must equal the oracle's bit for bit, integer and FP64 values alike,
and the preconditioner must agree within 1e-10."""
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


CASES = {
    "poisson2d_61": (lambda: P.poisson2d(61), 0.25, 4),
    "varcoef3d_20": (lambda: P.varcoef3d(20, 3, block=4), 0.5, 6),
    "fem2d_40": (lambda: P.fem2d(40, 2), 0.25, 8),
}


@pytest.mark.parametrize("k", [1, 3, 4])
@pytest.mark.parametrize("name", list(CASES))
def test_mis_k_hierarchy_bit_exact(env, name, k):
    amg, oracle = env
    make, alpha, seed = CASES[name]
    A = make()
    g = amg.Hierarchy(A, alpha=alpha, seed=seed, mis_k=k, precision=0)
    o = oracle.Hierarchy(A, alpha=alpha, seed=seed, mis_k=k)
    assert g.nlevels == o.nlevels >= 2
    for q in range(o.nlevels):
        gl, ol = g.level(q), o.level(q)
        assert np.array_equal(gl["rowptr"], ol.rowptr) and np.array_equal(gl["col"], ol.col), q
        assert np.array_equal(gl["val"], ol.val), q
        if q < o.nlevels - 1:
            assert np.array_equal(gl["agg"], ol.agg) and np.array_equal(gl["P"], ol.P), q
            assert gl["mis_rounds"] == ol.mis_rounds, q
            assert gl["omega"] == pytest.approx(ol.omega, rel=1e-12), q
    b = P.rhs_uniform(A.n, 11)
    zg, zo = g.precond(b), o.precond(b)
    assert np.linalg.norm(zg - zo) <= 1e-10 * np.linalg.norm(zo)


def test_mis3_coarsens_faster_and_every_precision_converges(env):
    amg, _ = env
    A = P.poisson3d(32)
    b = P.rhs_uniform(A.n, 12)
    n1 = {}
    for k in (2, 3):
        for prec in (0, 1, 2):
            h = amg.Hierarchy(A, alpha=0.5, seed=1, mis_k=k, precision=prec)
            n1[k] = h.level(1)["n"]
            x, info = h.solve(b, tol=1e-8)
            assert info["status"] == amg.AMG_OK
            assert np.linalg.norm(b - A.matvec(x)) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
            print(f"MIS({k}) precision {prec}: level-1 rows {n1[k]}, {info['iters']} iterations")
    assert n1[3] < n1[2] / 1.5


def test_mis_k_batch_of_one_equals_single_system(env):
    amg, _ = env
    A = P.varcoef2d(45, 5)
    p = amg.amg_default_params(alpha=0.25, seed=3, mis_k=3)
    hb = amg.amg_setup_batch([A], p)
    hs = amg.amg_setup(A.rowptr, A.col, A.val, p)
    try:
        nb, ns = len(amg.amg_hierarchy_info(hb)), len(amg.amg_hierarchy_info(hs))
        assert nb == ns
        for q in range(ns - 1):
            assert np.array_equal(amg.amg_export_level(hb, q)["agg"], amg.amg_export_level(hs, q)["agg"])
    finally:
        amg.amg_free(hb)
        amg.amg_free(hs)


@pytest.mark.parametrize("k", [0, 9])
def test_mis_k_out_of_range_is_rejected(env, k):
    amg, _ = env
    A = P.poisson2d(16)
    with pytest.raises(amg.AMGError) as e:
        amg.Hierarchy(A, mis_k=k)
    assert e.value.code == amg.AMG_ERR_BAD_INPUT
