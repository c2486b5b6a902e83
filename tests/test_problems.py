"""The seeded synthetic inputs: sizes and structure of the benchmark workloads
(2D/3D Poisson, jump-coefficient finite volumes, jittered P1 finite elements,
the batch of variable-coefficient systems, upwind convection-diffusion), their
CSR invariants and their reproducibility.  No method arithmetic is involved."""
import numpy as np
import pytest

from paper_1403_1649_gb300 import problems as P


def csr_ok(A):
    """int32 CSR, ascending columns, diagonal present, finite values"""
    assert A.rowptr.dtype == np.int32 and A.col.dtype == np.int32 and A.val.dtype == np.float64
    assert A.rowptr[0] == 0 and len(A.rowptr) == A.n + 1 and np.all(np.diff(A.rowptr) >= 1)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    same_row = rows[1:] == rows[:-1]
    assert np.all(A.col[1:][same_row] > A.col[:-1][same_row])
    assert np.all((A.col >= 0) & (A.col < A.n))
    diag = A.col == rows
    assert np.bincount(rows[diag], minlength=A.n).min() == 1
    assert np.isfinite(A.val).all()
    return rows, diag


def symmetric(A, rows):
    key = rows.astype(np.int64) * A.n + A.col
    tkey = A.col.astype(np.int64) * A.n + rows
    o, t = np.argsort(key), np.argsort(tkey)
    return np.array_equal(key[o], tkey[t]) and np.allclose(A.val[o], A.val[t], rtol=1e-14, atol=0)


@pytest.mark.parametrize("m,n,nnz", [(64, 4096, 20224), (37, 1369, 1369 * 5 - 4 * 37)])
def test_poisson2d_sizes_and_stencil(m, n, nnz):
    A = P.poisson2d(m)
    rows, diag = csr_ok(A)
    assert (A.n, A.nnz) == (n, nnz)
    assert np.all(A.val[diag] == 4.0) and np.all(A.val[~diag] == -1.0) and symmetric(A, rows)


def test_poisson3d_128_sizes():
    A = P.poisson3d(128)
    assert (A.n, A.nnz) == (2_097_152, 14_581_760)
    rows, diag = csr_ok(A)
    assert np.all(A.val[diag] == 6.0) and np.all(A.val[~diag] == -1.0)


def test_varcoef3d_160_sizes_and_coefficients():
    A = P.varcoef3d(160, 2)
    assert (A.n, A.nnz) == (4_096_000, 28_518_400)
    rows, diag = csr_ok(A)
    off = A.val[~diag]
    assert np.all(off < 0)
    # harmonic means of log-uniform [1e-3, 1e3] coefficients, x100 on half the z faces
    assert -off.max() >= 1e-3 * 0.99 and -off.min() <= 1e3 * 100 * 1.01
    # row sums: zero inside, positive next to the Dirichlet boundary
    rs = np.add.reduceat(A.val, A.rowptr[:-1])
    assert rs.min() > -1e-9 * np.abs(A.val[diag]).max() and (rs > 1e-12 * A.val[diag]).sum() > 0
    assert symmetric(A, rows)


def test_fem2d_1024_sizes_and_spd_structure():
    A = P.fem2d(1024, 3)
    assert A.n == 1_048_576 and 7.2e6 < A.nnz < 7.4e6
    rows, diag = csr_ok(A)
    assert np.all(A.val[diag] > 0) and symmetric(A, rows)


def test_batch_sizes_and_systems():
    sides = P.batch_sizes(512, 4)
    assert len(sides) == 512 and sides.min() >= 32 and sides.max() <= 512
    assert len(np.unique(sides)) > 200  # uneven sizes
    total = int((sides.astype(np.int64) ** 2).sum())
    assert 4.0e7 < total < 5.6e7
    A = P.varcoef2d(int(sides[0]), 4)
    rows, diag = csr_ok(A)
    assert A.n == int(sides[0]) ** 2 and symmetric(A, rows)


@pytest.mark.parametrize("pe", [2.0, 10.0])
def test_convdiff2d_nonsymmetric_m_matrix(pe):
    A = P.convdiff2d(33, 5, pe=pe)
    rows, diag = csr_ok(A)
    assert np.all(A.val[~diag] < 0) and not symmetric(A, rows)
    rs = np.add.reduceat(A.val, A.rowptr[:-1])
    assert rs.min() >= -1e-12  # weakly diagonally dominant rows, strictly at the boundary
    D = A.to_dense()
    assert np.abs(D - D.T).max() > 0.5


def test_inputs_are_reproducible_and_seeded():
    a, b = P.rhs_uniform(1000, 7), P.rhs_uniform(1000, 7)
    assert np.array_equal(a, b) and a.min() >= -1.0 and a.max() < 1.0
    assert not np.array_equal(a, P.rhs_uniform(1000, 8))
    # element-wise: a longer draw starts with the shorter one
    assert np.array_equal(P.rhs_uniform(10, 7), a[:10])
    A1, A2 = P.varcoef2d(20, 3), P.varcoef2d(20, 3)
    assert np.array_equal(A1.val, A2.val) and not np.array_equal(A1.val, P.varcoef2d(20, 4).val)
