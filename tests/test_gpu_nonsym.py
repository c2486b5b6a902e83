"""Nonsymmetric systems: upwind convection-diffusion solved by FGMRES with the
GMRES variant of Alg. 5 (Sec. 2.2: only GMRES applies to nonsymmetric matrices).
The hierarchy is bit-exact against the oracle; omega comes from the eigenvalues
of the Arnoldi Hessenberg matrix and the coarsest level is inverted through a
pivoted LU, both within 1e-10 of the oracle's."""
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


def pair(amg, oracle, A, **kw):
    g = amg.Hierarchy(A, alpha=0.25, seed=3, symmetric=0, outer=1, **kw)
    okw = {k: v for k, v in kw.items() if k in ("restart", "coarse_max")}
    o = oracle.Hierarchy(A, alpha=0.25, seed=3, symmetric=0, outer=1, **okw)
    return g, o


@pytest.mark.parametrize("m,pe", [(40, 2.0), (37, 10.0)])
def test_nonsymmetric_hierarchy_and_preconditioner(env, m, pe):
    amg, oracle = env
    A = P.convdiff2d(m, 5, pe=pe)
    g, o = pair(amg, oracle, A)
    assert g.nlevels == o.nlevels >= 3
    for k in range(o.nlevels):
        gl, ol = g.level(k), o.level(k)
        assert np.array_equal(gl["col"], ol.col) and np.array_equal(gl["val"], ol.val), k
        if k < o.nlevels - 1:
            assert np.array_equal(gl["agg"], ol.agg) and np.array_equal(gl["P"], ol.P), k
            assert gl["omega"] == pytest.approx(ol.omega, rel=1e-12), k
    D = A.to_dense()
    assert np.abs(D - D.T).max() > 0.5  # really nonsymmetric
    b = P.rhs_uniform(A.n, 31)
    zg, zo = g.precond(b), o.precond(b)
    assert np.linalg.norm(zg - zo) <= 1e-10 * np.linalg.norm(zo)


def test_nonsymmetric_fgmres_iterates_and_convergence(env):
    amg, oracle = env
    A = P.convdiff2d(40, 6, pe=4.0)
    g, o = pair(amg, oracle, A, restart=5, max_iter=8)
    b = P.rhs_uniform(A.n, 32)
    xg, ig = g.solve(b, tol=0.0, allow=(amg.AMG_OK, amg.AMG_ERR_NOT_CONVERGED))
    xo, io = o.solve(b, tol=0.0, max_iter=8)
    assert ig["iters"] == io["iters"] == 8
    assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo)
    assert np.allclose(ig["hist"], io["hist"], rtol=1e-8, atol=0)
    g2 = amg.Hierarchy(A, alpha=0.25, seed=3, symmetric=0, outer=1, restart=30)
    x, info = g2.solve(b, tol=1e-8)
    assert info["status"] == amg.AMG_OK and info["final_relres"] <= 1e-8
    assert np.linalg.norm(b - A.matvec(x)) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)


@pytest.mark.parametrize("prec", [1, 2])
def test_nonsymmetric_mixed_precision_reaches_fp64_tolerance(env, prec):
    amg, oracle = env
    A = P.convdiff2d(64, 7, pe=3.0)
    b = P.rhs_uniform(A.n, 33)
    g = amg.Hierarchy(A, alpha=0.25, seed=3, symmetric=0, outer=1, restart=30, precision=prec)
    x, info = g.solve(b, tol=1e-8)
    assert info["status"] == amg.AMG_OK
    assert np.linalg.norm(b - A.matvec(x)) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    xo, io = oracle.Hierarchy(A, alpha=0.25, seed=3, symmetric=0, outer=1).solve(b, tol=1e-12, max_iter=500)
    err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    # ||x - xo|| <= ||A^-1||_2 (||b - A x|| + ||b - A xo||), with
    # ||A^-1||_2 <= sqrt(||A^-1||_1 ||A^-1||_inf) from the dense inverse
    Ai = np.linalg.inv(A.to_dense())
    ninv = np.sqrt(np.abs(Ai).sum(0).max() * np.abs(Ai).sum(1).max())
    res = np.linalg.norm(b - A.matvec(x)) + np.linalg.norm(b - A.matvec(xo))
    assert np.linalg.norm(x - xo) <= ninv * res * (1 + 1e-6)
    assert err <= 1e-6
    print(f"precision {prec}: {info['iters']} FGMRES iterations, rel. error vs FP64 oracle {err:.2e} "
          f"(bound {ninv * res / np.linalg.norm(xo):.2e})")


def test_nonsymmetric_needs_fgmres_and_a_single_system(env):
    amg, _ = env
    A = P.convdiff2d(20, 1)
    with pytest.raises(amg.AMGError) as e:
        amg.Hierarchy(A, symmetric=0, outer=0)
    assert e.value.code == amg.AMG_ERR_BAD_INPUT and "FGMRES" in amg.amg_last_error()
    with pytest.raises(amg.AMGError) as e:
        amg.amg_setup_batch([A, A], amg.amg_default_params(symmetric=0))
    assert e.value.code == amg.AMG_ERR_UNSUPPORTED
