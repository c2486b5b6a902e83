"""Seeded synthetic linear systems shaped like the paper's elliptic PDE workloads.

This module is input generation only: it assembles sparse matrices and right-hand
sides from PDE discretisations and holds none of the multigrid method's arithmetic
(no strength test, no MIS, no aggregation, no Galerkin product, no smoothing, no
Krylov iteration).  Both the CPU oracle tests and the GPU path draw their inputs
from here, so the two sides always see byte-identical CSR arrays.

Every random draw comes from splitmix64 (Steele, Lea and Flood 2014; the mixer
constants are the published ones) evaluated on a counter
``(seed << 40) ^ (stream << 56) ^ index`` so that each array is reproducible
element by element, independently of array sizes.

The paper's own matrices (SPE10 pressure systems, Sec. 4, Table 2; the "RS and
pressure matrices" of Fig. 4) are not available; these generators stand in for
them:

* ``poisson2d(64)``        2D 5-point Laplacian, 64x64 interior grid, Dirichlet.
* ``poisson3d(128)``       3D 7-point Laplacian, 128^3.
* ``varcoef3d(160)``       cell-centred finite volumes for -div(k grad u) on 160^3,
                            k log-uniform in [1e-3, 1e3] constant on 8^3 blocks,
                            z-face coefficients x100 on the half x < 80.
* ``fem2d(1024)``          P1 finite elements on a jittered 1024^2 node grid with a
                            random diagonal per cell.
* ``batch_sizes`` / ``varcoef2d``  512 2D variable-coefficient 5-point systems.

All matrices are returned in CSR with int32 indices, ascending column order inside
each row and the diagonal present.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)

# stream ids: one per kind of random draw
STREAM_RHS = 1
STREAM_COEF = 2
STREAM_JITTER_X = 3
STREAM_JITTER_Y = 4
STREAM_DIAG = 5
STREAM_SIZE = 6


@dataclass
class CSR:
    """A square sparse matrix in compressed sparse row form (int32 indices, f64 values)."""

    n: int
    rowptr: np.ndarray  # int32, n+1
    col: np.ndarray  # int32, nnz, ascending inside each row
    val: np.ndarray  # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        np.add.at(d, (rows, self.col), self.val)
        return d

    def matvec(self, x: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        y = np.zeros(self.n)
        np.add.at(y, rows, self.val * x[self.col])
        return y


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied to uint64 counters (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def counter(seed: int, stream: int, n: int) -> np.ndarray:
    idx = np.arange(n, dtype=np.uint64)
    return (np.uint64(seed) << np.uint64(40)) ^ (np.uint64(stream) << np.uint64(56)) ^ idx


def uniform01(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1): the top 53 bits of splitmix64 times 2^-53 (exact)."""
    z = splitmix64(counter(seed, stream, n))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """Right-hand side with entries uniform in [-1, 1)."""
    return 2.0 * uniform01(seed, STREAM_RHS, n) - 1.0


# ----------------------------------------------------------------------------
# structured grids: cell-centred / node-centred stencils, Dirichlet eliminated
# ----------------------------------------------------------------------------

def _stencil_csr(shape: tuple[int, ...], face: list[np.ndarray], bface: list[tuple[np.ndarray, np.ndarray]]) -> CSR:
    """Assemble a (2d+1)-point symmetric stencil on a lexicographic grid (x fastest).

    ``face[a]`` holds the coupling coefficient t > 0 between cell p and its +1
    neighbour along axis ``a`` (array of the grid shape with the last index along
    ``a`` dropped); ``bface[a]`` = (low, high) boundary-face coefficients added to
    the diagonal of the first/last cell along axis a.  Off-diagonal = -t; diagonal =
    sum of all face coefficients of the cell.
    """
    d = len(shape)
    # numpy arrays are indexed [z, y, x] so that x is fastest in C order
    np_shape = tuple(reversed(shape))
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.int64).reshape(np_shape)
    diag = np.zeros(np_shape)
    offs = []  # list of (offset, coefficient array over np_shape or None mask)
    for a in range(d):
        ax = d - 1 - a  # numpy axis for grid axis a
        t = face[a]
        lo, hi = bface[a]
        # contributions to the diagonal
        sl_lo = [slice(None)] * d
        sl_hi = [slice(None)] * d
        sl_lo[ax] = slice(0, shape[a] - 1)
        sl_hi[ax] = slice(1, shape[a])
        diag[tuple(sl_lo)] += t
        diag[tuple(sl_hi)] += t
        first = [slice(None)] * d
        last = [slice(None)] * d
        first[ax] = slice(0, 1)
        last[ax] = slice(shape[a] - 1, shape[a])
        diag[tuple(first)] += lo
        diag[tuple(last)] += hi
        stride = int(np.prod(shape[:a]))
        # coefficient of neighbour at +stride for each cell (0 where absent)
        cplus = np.zeros(np_shape)
        cplus[tuple(sl_lo)] = -t
        vplus = np.zeros(np_shape, dtype=bool)
        vplus[tuple(sl_lo)] = True
        cminus = np.zeros(np_shape)
        cminus[tuple(sl_hi)] = -t
        vminus = np.zeros(np_shape, dtype=bool)
        vminus[tuple(sl_hi)] = True
        offs.append((-stride, cminus, vminus))
        offs.append((stride, cplus, vplus))
    offs.append((0, diag, np.ones(np_shape, dtype=bool)))
    offs.sort(key=lambda o: o[0])  # ascending column order
    k = len(offs)
    cols = np.empty((n, k), dtype=np.int64)
    vals = np.empty((n, k))
    mask = np.empty((n, k), dtype=bool)
    flat = idx.reshape(-1)
    for c, (off, coef, valid) in enumerate(offs):
        cols[:, c] = flat + off
        vals[:, c] = coef.reshape(-1)
        mask[:, c] = valid.reshape(-1)
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, rowptr.astype(np.int32), cols[mask].astype(np.int32), vals[mask].astype(np.float64))


def _const_faces(shape):
    d = len(shape)
    np_shape = tuple(reversed(shape))
    face, bface = [], []
    for a in range(d):
        ax = d - 1 - a
        s = list(np_shape)
        s[ax] = shape[a] - 1
        face.append(np.ones(s))
        b = list(np_shape)
        b[ax] = 1
        bface.append((np.ones(b), np.ones(b)))
    return face, bface


def poisson1d(m: int) -> CSR:
    """[-1 2 -1] on m interior nodes, Dirichlet eliminated."""
    face, bface = _const_faces((m,))
    return _stencil_csr((m,), face, bface)


def poisson2d(m: int) -> CSR:
    """5-point [-1 4 -1] Laplacian on an m x m interior grid (n = m^2)."""
    face, bface = _const_faces((m, m))
    return _stencil_csr((m, m), face, bface)


def poisson3d(m: int) -> CSR:
    """7-point Laplacian (diagonal 6) on an m^3 interior grid."""
    face, bface = _const_faces((m, m, m))
    return _stencil_csr((m, m, m), face, bface)


def aniso2d(m: int, eps: float) -> CSR:
    """Anisotropic 2D 5-point operator -u_xx - eps u_yy (x strongly coupled for eps < 1)."""
    face, bface = _const_faces((m, m))
    face[1] = face[1] * eps
    bface[1] = (bface[1][0] * eps, bface[1][1] * eps)
    return _stencil_csr((m, m), face, bface)


def _harmonic(kp: np.ndarray, kq: np.ndarray) -> np.ndarray:
    return 2.0 * kp * kq / (kp + kq)


def varcoef3d(m: int = 160, seed: int = 2, block: int = 8, lo: float = -3.0, hi: float = 3.0,
              zaniso: float = 100.0) -> CSR:
    """Finite-volume -div(k grad u) on an m^3 cell grid, Dirichlet on all faces.

    k is log-uniform in [10^lo, 10^hi], constant on aligned block^3 blocks; face
    coefficients are harmonic means of the two cells (2 k_p for boundary faces);
    z-face coefficients are multiplied by ``zaniso`` where the cell's x < m/2.
    """
    nb = (m + block - 1) // block
    u = uniform01(seed, STREAM_COEF, nb ** 3).reshape(nb, nb, nb)  # [bz, by, bx]
    kb = 10.0 ** (lo + (hi - lo) * u)
    r = np.arange(m) // block
    k = kb[np.ix_(r, r, r)]  # [z, y, x]
    xs = np.arange(m)
    zfac = np.where(xs < m // 2, zaniso, 1.0)  # along x
    face = [
        _harmonic(k[:, :, :-1], k[:, :, 1:]),  # x faces
        _harmonic(k[:, :-1, :], k[:, 1:, :]),  # y faces
        _harmonic(k[:-1, :, :], k[1:, :, :]) * zfac[None, None, :],  # z faces
    ]
    bface = [
        (2.0 * k[:, :, :1], 2.0 * k[:, :, -1:]),
        (2.0 * k[:, :1, :], 2.0 * k[:, -1:, :]),
        (2.0 * k[:1, :, :] * zfac[None, None, :], 2.0 * k[-1:, :, :] * zfac[None, None, :]),
    ]
    return _stencil_csr((m, m, m), face, bface)


def convdiff2d(m: int, seed: int, pe: float = 2.0) -> CSR:
    """Upwind finite differences for -Laplace(u) + b . grad(u) on an m^2 interior
    grid, Dirichlet eliminated, scaled by h^2: b = pe (cos t, sin t), t uniform
    on [0, 2 pi) from the seed, pe the cell Peclet number.  Neighbour entries are
    -1 - max(+-b_x, 0) (west / east) and -1 - max(+-b_y, 0) (south / north), the
    diagonal 4 + |b_x| + |b_y|: a nonsymmetric M-matrix."""
    t = 2.0 * np.pi * float(uniform01(seed, STREAM_COEF, 1)[0])
    bx, by = pe * np.cos(t), pe * np.sin(t)
    w, e = -1.0 - max(bx, 0.0), -1.0 - max(-bx, 0.0)
    so, no = -1.0 - max(by, 0.0), -1.0 - max(-by, 0.0)
    d = 4.0 + abs(bx) + abs(by)
    n = m * m
    idx = np.arange(n)
    x, y = idx % m, idx // m
    cols, vals = [], []
    for dc, v, ok in ((-m, so, y > 0), (-1, w, x > 0), (0, d, np.ones(n, bool)), (1, e, x < m - 1),
                      (m, no, y < m - 1)):
        cols.append(np.where(ok, idx + dc, -1))
        vals.append(np.where(ok, v, 0.0))
    C = np.stack(cols, 1)
    V = np.stack(vals, 1)
    keep = C >= 0
    rowptr = np.concatenate([[0], np.cumsum(keep.sum(1))]).astype(np.int32)
    return CSR(n, rowptr, C[keep].astype(np.int32), V[keep].astype(np.float64))


def varcoef2d(m: int, seed: int, lo: float = -2.0, hi: float = 2.0) -> CSR:
    """Finite-volume 5-point -div(k grad u) on an m^2 cell grid, k log-uniform per cell."""
    u = uniform01(seed, STREAM_COEF, m * m).reshape(m, m)  # [y, x]
    k = 10.0 ** (lo + (hi - lo) * u)
    face = [_harmonic(k[:, :-1], k[:, 1:]), _harmonic(k[:-1, :], k[1:, :])]
    bface = [(2.0 * k[:, :1], 2.0 * k[:, -1:]), (2.0 * k[:1, :], 2.0 * k[-1:, :])]
    return _stencil_csr((m, m), face, bface)


def batch_sizes(count: int = 512, seed: int = 4, lo: int = 32, hi: int = 512) -> np.ndarray:
    """Grid sides m_s uniform on {lo..hi} for the batched workload (system s uses seed+s)."""
    z = splitmix64(counter(seed, STREAM_SIZE, count))
    return (lo + (z % np.uint64(hi - lo + 1)).astype(np.int64)).astype(np.int64)


def fem2d(m: int = 1024, seed: int = 3, jitter: float = 0.3) -> CSR:
    """P1 finite-element Laplacian on an (m+2)^2 node grid with a Dirichlet ring.

    Interior nodes are moved by U[-jitter*h, jitter*h] per coordinate; every cell
    is split into two triangles along a diagonal chosen by a seeded coin.  All mesh
    edges stay structural entries even where the assembled value is ~0 or positive.
    Element matrices use |area| so the assembled matrix stays symmetric positive
    definite even if a jittered triangle flips orientation.
    """
    N = m + 2
    h = 1.0 / (m + 1)
    I, J = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")  # J rows (y), I cols (x)
    X = I * h
    Y = J * h
    interior = (I > 0) & (I < N - 1) & (J > 0) & (J < N - 1)
    jx = (2.0 * uniform01(seed, STREAM_JITTER_X, N * N) - 1.0).reshape(N, N) * jitter * h
    jy = (2.0 * uniform01(seed, STREAM_JITTER_Y, N * N) - 1.0).reshape(N, N) * jitter * h
    X = np.where(interior, X + jx, X).reshape(-1)
    Y = np.where(interior, Y + jy, Y).reshape(-1)
    node = np.arange(N * N).reshape(N, N)  # node[J, I]
    gid = np.full(N * N, -1, dtype=np.int64)
    gid[interior.reshape(-1)] = (I[interior] - 1) + m * (J[interior] - 1)
    a = node[:-1, :-1].reshape(-1)  # (I, J)
    b = node[:-1, 1:].reshape(-1)  # (I+1, J)
    c = node[1:, :-1].reshape(-1)  # (I, J+1)
    d = node[1:, 1:].reshape(-1)  # (I+1, J+1)
    coin = (splitmix64(counter(seed, STREAM_DIAG, (N - 1) * (N - 1))) >> np.uint64(63)).astype(bool)
    # coin 0: diagonal a-d ; coin 1: diagonal b-c
    t1 = np.where(coin[:, None], np.stack([a, b, c], 1), np.stack([a, b, d], 1))
    t2 = np.where(coin[:, None], np.stack([b, d, c], 1), np.stack([a, d, c], 1))
    tri = np.concatenate([t1, t2], 0)
    px, py = X[tri], Y[tri]
    # gradients of barycentric coordinates times 2*area
    bx = np.stack([py[:, 1] - py[:, 2], py[:, 2] - py[:, 0], py[:, 0] - py[:, 1]], 1)
    by = np.stack([px[:, 2] - px[:, 1], px[:, 0] - px[:, 2], px[:, 1] - px[:, 0]], 1)
    det = (px[:, 1] - px[:, 0]) * (py[:, 2] - py[:, 0]) - (px[:, 2] - px[:, 0]) * (py[:, 1] - py[:, 0])
    area2 = np.abs(det)
    Ke = (bx[:, :, None] * bx[:, None, :] + by[:, :, None] * by[:, None, :]) / (2.0 * area2)[:, None, None]
    g = gid[tri]
    rows = np.repeat(g, 3, axis=1).reshape(-1)
    cols = np.tile(g, (1, 3)).reshape(-1)
    vals = Ke.reshape(-1)
    keep = (rows >= 0) & (cols >= 0)
    rows, cols, vals = rows[keep], cols[keep], vals[keep]
    n = m * m
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    starts = np.flatnonzero(np.r_[True, key[1:] != key[:-1]])
    uval = np.add.reduceat(vals, starts)
    ukey = key[starts]
    urow = ukey // n
    ucol = ukey % n
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(urow, minlength=n), out=rowptr[1:])
    return CSR(n, rowptr.astype(np.int32), ucol.astype(np.int32), uval)


def from_dense(a: np.ndarray) -> CSR:
    """CSR of the structural nonzeros of a dense matrix (diagonal always kept)."""
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[0]
    mask = (a != 0) | np.eye(n, dtype=bool)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(mask.sum(1), out=rowptr[1:])
    r, c = np.nonzero(mask)
    return CSR(n, rowptr.astype(np.int32), c.astype(np.int32), a[r, c].copy())


def block_diag(mats: list[CSR]) -> CSR:
    """Block-diagonal concatenation of square CSR matrices."""
    n = sum(A.n for A in mats)
    rowptr = [np.zeros(1, dtype=np.int64)]
    cols, vals = [], []
    off_r, off_nz = 0, 0
    for A in mats:
        rowptr.append(A.rowptr[1:].astype(np.int64) + off_nz)
        cols.append(A.col.astype(np.int64) + off_r)
        vals.append(A.val)
        off_r += A.n
        off_nz += A.nnz
    return CSR(n, np.concatenate(rowptr).astype(np.int32), np.concatenate(cols).astype(np.int32),
               np.concatenate(vals))


WORKLOADS = {
    "poisson2d_64": lambda: (poisson2d(64), 0.25, rhs_uniform(64 * 64, 0)),
    "poisson3d_128": lambda: (poisson3d(128), 0.5, rhs_uniform(128 ** 3, 1)),
    "varcoef3d_160": lambda: (varcoef3d(160, 2), 0.5, rhs_uniform(160 ** 3, 2)),
    "fem2d_1024": lambda: (fem2d(1024, 3), 0.25, rhs_uniform(1024 * 1024, 3)),
}
