"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a value the
paper prints (the Sec. 3.1 worked example, Table 1's level-0 size), a closed form
(the spectrum of the 1D/2D Laplacian), a different algorithm with a provably
identical result (greedy MIS on the square graph), a library routine on a special
case (numpy dense products, eigvalsh, solve), or an invariant that a plausible
mistake would break.
"""
import os
from collections import deque

import numpy as np
import pytest

from paper_1403_1649_gb300 import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def csr_from_rows(rows: dict, n: int, vals: dict):
    rp = [0]
    ci, va = [], []
    for i in range(n):
        for j in sorted(rows[i]):
            ci.append(j)
            va.append(vals[(i, j)])
        rp.append(len(ci))
    return P.CSR(n, np.array(rp, np.int32), np.array(ci, np.int32), np.array(va, np.float64))


def adjacency(Sptr, Scol):
    n = len(Sptr) - 1
    return [set(Scol[Sptr[i]:Sptr[i + 1]].tolist()) for i in range(n)]


def bfs_dist(adj, src, cap=3):
    dist = {src: 0}
    dq = deque([src])
    while dq:
        u = dq.popleft()
        if dist[u] >= cap:
            continue
        for v in adj[u]:
            if v not in dist:
                dist[v] = dist[u] + 1
                dq.append(v)
    return dist


def random_sym_graph(n, deg, seed):
    rng = np.random.default_rng(seed)
    adj = [set() for _ in range(n)]
    for _ in range(n * deg // 2):
        a, b = rng.integers(0, n, 2)
        if a != b:
            adj[a].add(int(b))
            adj[b].add(int(a))
    Sptr = np.zeros(n + 1, np.int32)
    cols = []
    for i in range(n):
        cols.extend(sorted(adj[i]))
        Sptr[i + 1] = len(cols)
    return Sptr, np.array(cols, np.int32), adj


# ----------------------------------------------------------------- strength
def test_strength_1d_poisson_all_offdiag_strong(oracle_mod):
    A = P.poisson1d(7)
    Cm = oracle_mod.strength(A, 0.25)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    assert np.array_equal(Cm.astype(bool), rows != A.col)


def test_strength_anisotropic_keeps_only_strong_direction(oracle_mod):
    # -u_xx - 0.1 u_yy: |a_y| = 0.1 < 0.25 * |a_x| = 0.25, so only x-neighbours are strong
    m = 6
    A = P.aniso2d(m, 0.1)
    Cm = oracle_mod.strength(A, 0.25)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    dx = np.abs(A.col - rows)
    assert np.array_equal(Cm.astype(bool), dx == 1)
    # with alpha = 0.05 the y-connections (0.1 > 0.05) become strong too
    Cm2 = oracle_mod.strength(A, 0.05)
    assert np.array_equal(Cm2.astype(bool), rows != A.col)


def test_strength_signs_and_strict_threshold(oracle_mod):
    # row 0: positive diagonal; -A_01 = -1 < 0 (not strong), -A_02 = 2 strong,
    #        -A_03 = 0.5 = 0.25*2 exactly -> not strong (strict inequality)
    # row 1: negative diagonal, s = -1: -s*A_10 = 1 (strong, the max),
    #        -s*A_12 = -3 (opposite sign: never strong)
    # row 2: only same-sign off-diagonals -> no strong connection at all
    # row 3: 1x diagonal only
    rows = {0: [0, 1, 2, 3], 1: [0, 1, 2], 2: [1, 2, 3], 3: [3]}
    vals = {(0, 0): 4.0, (0, 1): 1.0, (0, 2): -2.0, (0, 3): -0.5,
            (1, 0): 1.0, (1, 1): -5.0, (1, 2): -3.0,
            (2, 1): 1.0, (2, 2): 3.0, (2, 3): 1.0,
            (3, 3): 1.0}
    A = csr_from_rows(rows, 4, vals)
    Cm = oracle_mod.strength(A, 0.25)
    expect = [0, 0, 1, 0,   1, 0, 0,   0, 0, 0,   0]
    assert Cm.tolist() == expect


def test_col_count_and_sym_graph(oracle_mod):
    # asymmetric strength pattern: C_01 = 1, C_10 = 0, C_21 = 1, C_12 = 1
    rows = {0: [0, 1], 1: [0, 1, 2], 2: [1, 2]}
    vals = {(0, 0): 2.0, (0, 1): -1.0, (1, 0): -0.1, (1, 1): 2.0, (1, 2): -1.0, (2, 1): -1.0, (2, 2): 2.0}
    A = csr_from_rows(rows, 3, vals)
    Cm = oracle_mod.strength(A, 0.25)
    assert Cm.tolist() == [0, 1, 0, 0, 1, 1, 0]
    assert oracle_mod.col_count(A, Cm).tolist() == [0, 2, 1]
    Sptr, Scol = oracle_mod.sym_graph(A, Cm)
    assert adjacency(Sptr, Scol) == [{1}, {0, 2}, {1}]


# ----------------------------------------------------------------- PMIS(2)
def greedy_mis2(adj, count, h):
    """Sequential greedy MIS on the square graph, nodes in descending (count, h, i)."""
    n = len(adj)
    order = sorted(range(n), key=lambda i: (int(count[i]), int(h[i]), i), reverse=True)
    blocked = np.zeros(n, bool)
    s = -np.ones(n, np.int8)
    for i in order:
        if blocked[i]:
            continue
        s[i] = 1
        for j, dd in bfs_dist(adj, i, 2).items():
            blocked[j] = True
    return s


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_pmis2_equals_greedy_mis_on_square_graph(oracle_mod, seed):
    n = 300
    Sptr, Scol, adj = random_sym_graph(n, 4, seed)
    rng = np.random.default_rng(100 + seed)
    count = rng.integers(0, 5, n).astype(np.int32)
    h = oracle_mod.mis_hash(seed, 0, n)
    s, rounds = oracle_mod.pmis2(Sptr, Scol, count, h)
    assert rounds >= 1
    assert np.array_equal(s, greedy_mis2(adj, count, h))


def test_pmis2_ties_broken_by_index(oracle_mod):
    # all priorities equal: the largest index wins every distance-2 ball (path graph)
    n = 10
    adj = [set() for _ in range(n)]
    for i in range(n - 1):
        adj[i].add(i + 1)
        adj[i + 1].add(i)
    Sptr = np.zeros(n + 1, np.int32)
    cols = []
    for i in range(n):
        cols.extend(sorted(adj[i]))
        Sptr[i + 1] = len(cols)
    s, _ = oracle_mod.pmis2(Sptr, np.array(cols, np.int32), np.zeros(n, np.int32), np.zeros(n, np.uint32))
    assert np.flatnonzero(s == 1).tolist() == [0, 3, 6, 9]


def test_pmis2_isolated_nodes_are_roots(oracle_mod):
    n = 5
    Sptr = np.zeros(n + 1, np.int32)
    s, _ = oracle_mod.pmis2(Sptr, np.zeros(0, np.int32), np.zeros(n, np.int32), np.arange(n, dtype=np.uint32))
    assert (s == 1).all()


def mis_invariants(adj, s):
    roots = np.flatnonzero(s == 1)
    rootset = set(roots.tolist())
    for r in roots:
        d = bfs_dist(adj, int(r), 2)
        assert not (set(d) - {int(r)}) & rootset, "two roots within distance 2"
    for i in np.flatnonzero(s != 1):
        d = bfs_dist(adj, int(i), 2)
        assert set(d) & rootset, "non-root farther than 2 from every root"


@pytest.mark.parametrize("seed", [5, 6])
def test_mis_and_aggregate_invariants_random(oracle_mod, seed):
    n = 400
    Sptr, Scol, adj = random_sym_graph(n, 5, seed)
    count = np.array([len(a) for a in adj], np.int32)
    h = oracle_mod.mis_hash(seed, 1, n)
    s, _ = oracle_mod.pmis2(Sptr, Scol, count, h)
    mis_invariants(adj, s)
    agg, nc = oracle_mod.aggregate(Sptr, Scol, count, h, s)
    check_aggregates(adj, s, agg, nc, count, h)


def check_aggregates(adj, s, agg, nc, count, h):
    roots = np.flatnonzero(s == 1)
    assert nc == len(roots)
    # roots numbered in ascending fine index, one root per aggregate
    assert agg[roots].tolist() == list(range(nc))
    assert (agg >= 0).all() and (agg < nc).all()
    root_of = {int(agg[r]): int(r) for r in roots}
    key = lambda r: (int(count[r]), int(h[r]), r)
    rootset = set(roots.tolist())
    for i in np.flatnonzero(s != 1):
        i = int(i)
        r = root_of[int(agg[i])]
        d = bfs_dist(adj, i, 2)
        assert r in d, "member farther than 2 from its root"
        near1 = [j for j in adj[i] if j in rootset]
        if near1:  # nearest root first; among those the largest priority
            assert d[r] == 1 and r == max(near1, key=key)
        else:
            cands = [max([q for q in adj[j] if q in rootset], key=key)
                     for j in adj[i] if any(q in rootset for q in adj[j])]
            assert d[r] == 2 and r == max(cands, key=key)


def test_aggregates_on_grid(oracle_mod):
    A = P.poisson2d(12)
    Cm = oracle_mod.strength(A, 0.25)
    count = oracle_mod.col_count(A, Cm)
    Sptr, Scol = oracle_mod.sym_graph(A, Cm)
    h = oracle_mod.mis_hash(0, 0, A.n)
    s, _ = oracle_mod.pmis2(Sptr, Scol, count, h)
    adj = adjacency(Sptr, Scol)
    mis_invariants(adj, s)
    agg, nc = oracle_mod.aggregate(Sptr, Scol, count, h, s)
    check_aggregates(adj, s, agg, nc, count, h)
    # in 2D a distance-2 ball has at most 13 nodes, and MIS(2) gives a ratio well above 2
    sizes = np.bincount(agg)
    assert sizes.max() <= 13 and A.n / nc > 3


# ----------------------------------------------------------------- MIS(k), k != 2
def greedy_mis_k(adj, count, h, k):
    """Sequential greedy MIS on the k-th power of the graph (nodes within distance
    k are adjacent), nodes in descending (count, h, i)."""
    n = len(adj)
    order = sorted(range(n), key=lambda i: (int(count[i]), int(h[i]), i), reverse=True)
    blocked = np.zeros(n, bool)
    s = -np.ones(n, np.int8)
    for i in order:
        if blocked[i]:
            continue
        s[i] = 1
        for j in bfs_dist(adj, i, k):
            blocked[j] = True
    return s


@pytest.mark.parametrize("k,seed", [(1, 0), (3, 1), (3, 2), (4, 3)])
def test_pmis_k_equals_greedy_mis_on_graph_power(oracle_mod, k, seed):
    n = 300
    Sptr, Scol, adj = random_sym_graph(n, 4, seed)
    rng = np.random.default_rng(200 + seed)
    count = rng.integers(0, 5, n).astype(np.int32)
    h = oracle_mod.mis_hash(seed, 0, n)
    s, rounds = oracle_mod.pmis(Sptr, Scol, count, h, k)
    assert rounds >= 1
    assert np.array_equal(s, greedy_mis_k(adj, count, h, k))


def root_distance(adj, roots):
    """multi-source breadth-first distance to the nearest root"""
    d = {int(r): 0 for r in roots}
    frontier = list(d)
    while frontier:
        nxt = []
        for u in frontier:
            for v in adj[u]:
                if v not in d:
                    d[v] = d[u] + 1
                    nxt.append(v)
        frontier = nxt
    return d


def check_aggregates_k(adj, s, agg, nc, count, h, k):
    """every node joins a nearest root (distance <= k); among the roots reached
    through neighbours one step nearer, the largest priority (pass d of the
    aggregation takes the nodes at distance d)"""
    roots = np.flatnonzero(s == 1)
    assert nc == len(roots) and agg[roots].tolist() == list(range(nc))
    assert (agg >= 0).all() and (agg < nc).all()
    root_of = {int(agg[r]): int(r) for r in roots}
    key = lambda r: (int(count[r]), int(h[r]), r)
    rootset = set(roots.tolist())
    dist = root_distance(adj, roots)
    assert len(dist) == len(adj) and max(dist.values()) <= k
    for i in np.flatnonzero(s != 1):
        i = int(i)
        r = root_of[int(agg[i])]
        if dist[i] == 1:
            expect = max((j for j in adj[i] if j in rootset), key=key)
        else:
            expect = max((root_of[int(agg[j])] for j in adj[i] if dist[j] == dist[i] - 1), key=key)
        assert r == expect
        assert bfs_dist(adj, i, k).get(r) == dist[i], "member not joined to a nearest root"


@pytest.mark.parametrize("k,seed", [(1, 7), (2, 8), (3, 9), (4, 10)])
def test_aggregate_k_nearest_root_rule(oracle_mod, k, seed):
    n = 400
    Sptr, Scol, adj = random_sym_graph(n, 3, seed)
    count = np.array([len(a) for a in adj], np.int32)
    h = oracle_mod.mis_hash(seed, 1, n)
    s, _ = oracle_mod.pmis(Sptr, Scol, count, h, k)
    agg, nc = oracle_mod.aggregate(Sptr, Scol, count, h, s, k)
    check_aggregates_k(adj, s, agg, nc, count, h, k)


def test_mis3_coarsens_more_and_still_converges(oracle_mod):
    A = P.poisson2d(40)
    b = P.rhs_uniform(A.n, 4)
    n1 = {}
    for k in (2, 3):
        H = oracle_mod.Hierarchy(A, alpha=0.25, seed=1, mis_k=k)
        n1[k] = H.level(1).n
        x, info = H.solve(b, tol=1e-8, max_iter=200)
        assert info["status"] == 0 and np.linalg.norm(b - A.matvec(x)) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    assert n1[3] < n1[2] / 1.5


# ----------------------------------------------------------------- interpolation
def test_interp_orthonormal_and_reproduces_B(oracle_mod):
    rng = np.random.default_rng(0)
    n, nc = 50, 9
    agg = np.concatenate([np.arange(nc), rng.integers(0, nc, n - nc)]).astype(np.int32)
    B = rng.uniform(0.5, 2.0, n)
    Pw, Bc = oracle_mod.interp(agg, nc, B)
    Pd = np.zeros((n, nc))
    Pd[np.arange(n), agg] = Pw
    assert np.allclose(Pd.T @ Pd, np.eye(nc), atol=4e-16 * 8)  # P^T P = I
    assert np.allclose(Pd @ Bc, B, rtol=4e-16 * 4, atol=0)  # B_k = P_k B_{k+1}
    # B_{k+1}(I) is the 2-norm of B over aggregate I
    for I in range(nc):
        assert Bc[I] == pytest.approx(np.linalg.norm(B[agg == I]), rel=1e-15)


# ----------------------------------------------------------------- Galerkin
def load_example():
    agg = None
    rows = {}
    coarse = {}
    for line in open(os.path.join(GOLDEN, "galerkin_example.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("agg"):
            agg = [int(t) - 1 for t in line.split()[1:]]
        elif line.startswith("row"):
            head, tail = line.split(":")
            rows[int(head.split()[1]) - 1] = [int(t) - 1 for t in tail.split()]
        elif line.startswith("coarse"):
            head, tail = line.split(":")
            _, I, J = head.split()
            coarse[(int(I) - 1, int(J) - 1)] = [tuple(int(u) - 1 for u in t.split(",")) for t in tail.split()]
    return agg, rows, coarse


def test_galerkin_worked_example_exact_order(oracle_mod):
    agg, rows, coarse = load_example()
    n = 8
    assert sum(len(r) for r in rows.values()) == 28
    rng = np.random.default_rng(7)
    # magnitudes spread over 16 decades: any change of grouping or summation order
    # changes the rounded sums
    vals = {(i, j): float(rng.choice([-1, 1]) * 10.0 ** rng.uniform(-8, 8)) for i in rows for j in rows[i]}
    A = csr_from_rows(rows, n, vals)
    Ac = oracle_mod.galerkin(A, np.array(agg, np.int32), 3, None)
    got = {}
    for I in range(3):
        for p in range(Ac.rowptr[I], Ac.rowptr[I + 1]):
            got[(I, int(Ac.col[p]))] = Ac.val[p]
    assert set(got) == set(coarse) and Ac.nnz == 7
    for key, terms in coarse.items():
        s = vals[terms[0]]
        for t in terms[1:]:
            s = s + vals[t]  # left to right, the order of the sorted list
        assert got[key] == s, key


def test_galerkin_equals_dense_triple_product(oracle_mod):
    for A, alpha in [(P.poisson2d(9), 0.25), (P.varcoef2d(10, 11), 0.25), (P.poisson3d(5), 0.5)]:
        Cm = oracle_mod.strength(A, alpha)
        count = oracle_mod.col_count(A, Cm)
        Sptr, Scol = oracle_mod.sym_graph(A, Cm)
        h = oracle_mod.mis_hash(3, 0, A.n)
        s, _ = oracle_mod.pmis2(Sptr, Scol, count, h)
        agg, nc = oracle_mod.aggregate(Sptr, Scol, count, h, s)
        B = np.random.default_rng(1).uniform(0.5, 1.5, A.n)
        Pw, Bc = oracle_mod.interp(agg, nc, B)
        Pd = np.zeros((A.n, nc))
        Pd[np.arange(A.n), agg] = Pw
        dense = Pd.T @ A.to_dense() @ Pd
        Ac = oracle_mod.galerkin(A, agg, nc, Pw)
        got = Ac.to_dense()
        scale = np.abs(dense).max()
        assert np.abs(got - dense).max() <= 1e-14 * scale
        # the coarse pattern is exactly symmetric; mirrored values are summed in
        # different orders, so they agree to rounding only
        assert np.array_equal(got != 0, got.T != 0)
        assert np.abs(got - got.T).max() <= 1e-15 * scale
        # coarse columns ascending within each row
        for I in range(nc):
            c = Ac.col[Ac.rowptr[I]:Ac.rowptr[I + 1]]
            assert (np.diff(c) > 0).all()


# ----------------------------------------------------------------- omega
@pytest.mark.parametrize("kind,m", [("1d", 60), ("2d", 12), ("2d", 30)])
def test_rho_estimate_against_laplacian_spectrum(oracle_mod, kind, m):
    A = P.poisson1d(m) if kind == "1d" else P.poisson2d(m)
    rho_exact = 1.0 + np.cos(np.pi / (m + 1))  # rho(D^-1 A) of the Dirichlet Laplacian
    rho, H = oracle_mod.rho_estimate(A, seed=0, level=0, m=5)
    assert rho <= rho_exact * (1 + 1e-12)
    assert rho >= 0.9 * rho_exact
    # the oracle's eigen-solver against LAPACK on the same symmetric part
    T = 0.5 * (H + H.T)
    assert rho == pytest.approx(np.abs(np.linalg.eigvalsh(T)).max(), rel=1e-13)
    # Arnoldi on a symmetric operator: H is tridiagonal up to rounding
    assert np.abs(np.triu(H, 2)).max() <= 1e-12


def test_sym_eig_against_lapack(oracle_mod):
    rng = np.random.default_rng(3)
    for m in (1, 2, 5, 8):
        a = rng.normal(size=(m, m))
        a = a + a.T
        assert np.allclose(oracle_mod.sym_eig(a), np.linalg.eigvalsh(a), atol=1e-12)


def test_cholesky_solve(oracle_mod):
    rng = np.random.default_rng(4)
    m = 40
    a = rng.normal(size=(m, m))
    a = a @ a.T + m * np.eye(m)
    L = oracle_mod.cholesky(a)
    assert np.allclose(L @ L.T, a, rtol=1e-13, atol=1e-12)
    b = rng.normal(size=m)
    assert np.allclose(oracle_mod.chol_solve(L, b), np.linalg.solve(a, b), rtol=1e-12)
    assert oracle_mod.cholesky(-a) is None


# ----------------------------------------------------------------- the whole method
def test_table1_level0_size():
    vals = dict(l.split() for l in open(os.path.join(GOLDEN, "table1_level0.txt")) if l[0] != "#")
    A = P.poisson2d(int(vals["m"]))
    assert A.n == int(vals["n"]) and A.nnz == int(vals["nnz"])


@pytest.mark.parametrize("kind", ["1d", "2d", "3d"])
def test_manufactured_solution(oracle_mod, kind):
    A, alpha = {"1d": (P.poisson1d(300), 0.25), "2d": (P.poisson2d(40), 0.25), "3d": (P.poisson3d(14), 0.5)}[kind]
    xs = np.sin(np.arange(A.n) * 0.37) + 0.1
    b = A.matvec(xs)
    H = oracle_mod.Hierarchy(A, alpha=alpha, coarse_max=16)
    assert H.nlevels >= 2
    tol = 1e-10
    x, info = H.solve(b, tol=tol, max_iter=300)
    assert info["status"] == 0 and info["relres"] <= tol
    kappa = np.linalg.cond(A.to_dense())
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * tol


def test_one_level_converges_in_one_iteration(oracle_mod):
    A = P.poisson2d(7)  # n = 49 <= coarse_max
    H = oracle_mod.Hierarchy(A, coarse_max=64)
    assert H.nlevels == 1
    x, info = H.solve(P.rhs_uniform(A.n, 0), tol=1e-12)
    assert info["iters"] == 1 and info["relres"] <= 1e-12


def test_fcg_error_decreases_in_A_norm(oracle_mod):
    A = P.varcoef2d(24, 9)
    Ad = A.to_dense()
    b = P.rhs_uniform(A.n, 5)
    xs = np.linalg.solve(Ad, b)
    H = oracle_mod.Hierarchy(A, coarse_max=20)
    errs = []
    for k in range(1, 12):
        x, info = H.solve(b, tol=0.0, max_iter=k)
        e = x - xs
        errs.append(np.sqrt(e @ Ad @ e))
    assert all(b_ <= a_ * (1 + 1e-12) for a_, b_ in zip(errs, errs[1:]))
    assert errs[-1] < 0.1 * errs[0]


def test_kcycle_inner_step_is_2x2_galerkin_solve(oracle_mod):
    A = P.poisson2d(40)
    H = oracle_mod.Hierarchy(A, coarse_max=16, kcycle_t=0.0)  # always take the second inner step
    assert H.nlevels >= 3
    L1 = H.level(1)
    A1 = P.CSR(L1.n, L1.rowptr, L1.col, L1.val).to_dense()
    r = P.rhs_uniform(L1.n, 8)
    x, c, d = H.krylov2_probe(1, r)
    G = np.array([[c @ A1 @ c, c @ A1 @ d], [d @ A1 @ c, d @ A1 @ d]])
    ab = np.linalg.solve(G, np.array([c @ r, d @ r]))
    assert np.allclose(x, ab[0] * c + ab[1] * d, rtol=1e-9, atol=1e-12 * np.abs(x).max())
    # with t large the first step is accepted: x = (c^T r / c^T A c) c
    H2 = oracle_mod.Hierarchy(A, coarse_max=16, kcycle_t=10.0)
    x2, c2, d2 = H2.krylov2_probe(1, r)
    assert np.allclose(x2, (c2 @ r) / (c2 @ A1 @ c2) * c2, rtol=1e-12)
    assert not d2.any()


def dense_hierarchy(H):
    levs = [H.level(k) for k in range(H.nlevels)]
    A = [P.CSR(L.n, L.rowptr, L.col, L.val).to_dense() for L in levs]
    Pm = []
    for k in range(len(levs) - 1):
        Pd = np.zeros((levs[k].n, levs[k + 1].n))
        Pd[np.arange(levs[k].n), levs[k].agg] = levs[k].P
        Pm.append(Pd)
    return levs, A, Pm


def test_two_grid_cycle_matches_textbook(oracle_mod):
    A = P.poisson2d(16)
    H = oracle_mod.Hierarchy(A, coarse_max=64)
    assert H.nlevels == 2
    levs, Ad, Pm = dense_hierarchy(H)
    w = levs[0].omega / np.diag(Ad[0])
    b = P.rhs_uniform(A.n, 2)
    x = w * b
    x = x + Pm[0] @ np.linalg.solve(Ad[1], Pm[0].T @ (b - Ad[0] @ x))
    x = x + w * (b - Ad[0] @ x)
    assert np.allclose(H.precond(b), x, rtol=1e-11, atol=1e-13)
    # Galerkin coarse operator equals P^T A P
    assert np.allclose(Ad[1], Pm[0].T @ Ad[0] @ Pm[0], rtol=1e-13, atol=1e-14)


def test_vcycle_symmetric_and_matches_recursion(oracle_mod):
    A = P.poisson2d(30)
    H = oracle_mod.Hierarchy(A, coarse_max=16, kcycle_levels=0)
    assert H.nlevels >= 3
    levs, Ad, Pm = dense_hierarchy(H)

    def vcyc(k, b):
        if k == len(Ad) - 1:
            return np.linalg.solve(Ad[k], b)
        w = levs[k].omega / np.diag(Ad[k])
        x = w * b
        xc = vcyc(k + 1, Pm[k].T @ (b - Ad[k] @ x))
        x = x + Pm[k] @ xc
        return x + w * (b - Ad[k] @ x)

    b = P.rhs_uniform(A.n, 3)
    assert np.allclose(H.precond(b), vcyc(0, b), rtol=1e-11, atol=1e-13)
    u, v = P.rhs_uniform(A.n, 4), P.rhs_uniform(A.n, 5)
    assert u @ H.precond(v) == pytest.approx(v @ H.precond(u), rel=1e-12)


def test_polynomial_smoother_reduces_to_jacobi(oracle_mod):
    A = P.poisson2d(20)
    b = P.rhs_uniform(A.n, 6)
    H = oracle_mod.Hierarchy(A, coarse_max=16)
    ref = H.precond(b)
    for k in range(H.nlevels - 1):
        L = H.level(k)
        H.set_poly(k, np.tile([L.omega, 0.0, 0.0], (L.n, 1)))
    assert np.allclose(H.precond(b), ref, rtol=1e-13, atol=1e-15)


def test_polynomial_smoother_vcycle_symmetric(oracle_mod):
    A = P.varcoef2d(20, 3)
    H = oracle_mod.Hierarchy(A, coarse_max=16, kcycle_levels=0)
    rng = np.random.default_rng(2)
    for k in range(H.nlevels - 1):
        H.set_poly(k, rng.uniform(0.1, 0.6, (H.level(k).n, 3)))
    u, v = P.rhs_uniform(A.n, 4), P.rhs_uniform(A.n, 5)
    assert u @ H.precond(v) == pytest.approx(v @ H.precond(u), rel=1e-11)


def test_fgmres_manufactured_and_monotone(oracle_mod):
    A = P.varcoef2d(30, 4)
    xs = np.cos(np.arange(A.n) * 0.11)
    b = A.matvec(xs)
    H = oracle_mod.Hierarchy(A, coarse_max=16, outer=1, restart=5)
    x, info = H.solve(b, tol=1e-10, max_iter=200)
    assert info["status"] == 0 and info["relres"] <= 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= np.linalg.cond(A.to_dense()) * 1e-10
    hist = info["hist"]
    assert all(b_ <= a_ * (1 + 1e-12) for a_, b_ in zip(hist, hist[1:]))


def test_setup_rejects_bad_csr(oracle_mod):
    A = P.poisson1d(5)
    bad = P.CSR(A.n, A.rowptr, A.col, A.val.copy())
    bad.val[0] = 0.0  # zero diagonal
    with pytest.raises(RuntimeError):
        oracle_mod.Hierarchy(bad)
    unsorted = P.CSR(A.n, A.rowptr, A.col.copy(), A.val)
    unsorted.col[1], unsorted.col[2] = unsorted.col[2], unsorted.col[1]
    with pytest.raises(RuntimeError):
        oracle_mod.Hierarchy(unsorted)


def test_splitmix64_published_vector(oracle_mod):
    # splitmix64 output sequence from state 0 (Vigna's reference implementation
    # advances the state by the golden gamma before mixing): first value
    assert oracle_mod.splitmix64(0) == 0xE220A8397B1DCDAF
    assert int(P.splitmix64(np.array([0], np.uint64))[0]) == 0xE220A8397B1DCDAF


# ----------------------------------------------------------------- learned smoother pieces
def test_features_of_1d_poisson_rows(oracle_mod):
    f = oracle_mod.features(P.poisson1d(5), level=1)
    interior = [1, 0.25, 0.5, 0.5, 0, 0, 0, 0, 0, 0, 0, 0, 0.25, 0.5, 0.5, 1.0]
    boundary = [1, 0.125, 0.5, 0, 0, 0, 0, 0, 0, 0, 0, 0.5, 0.25, 0.5, 0.5, 0.5]
    assert f[2].tolist() == interior and f[0].tolist() == boundary


def test_features_hand_computed_rows(oracle_mod):
    """Row 0: positive diagonal, ten off-diagonals of distinct magnitude in no
    particular order, three of them positive (so the top-8 list must drop the two
    smallest and keep the rest sorted, and the same-sign fraction and min / max of
    t_j see both signs).  Row 1: negative diagonal, so "same sign" means negative
    and the row sum is divided by a negative a_ii.  Every expected value below is
    worked out by hand and exact in binary."""
    a = np.zeros((12, 12))
    a[0, 0] = 8.0
    a[0, 1:11] = [-1.0, 0.5, -0.25, -2.0, 0.125, -0.75, -1.5, 0.375, -0.0625, -3.0]
    a[1, 1] = -2.0
    a[1, 0], a[1, 2], a[1, 3] = 0.5, -0.5, 1.0
    for i in range(2, 12):
        a[i, i] = 1.0
    f = oracle_mod.features(P.from_dense(a), level=2)
    row0 = [1.0, 10 / 8, 0.375, 0.25, 0.1875, 0.125, 0.09375, 0.0625, 0.046875, 0.03125,
            3 / 10, 0.4375 / 8, 0.5, -0.0625, 0.375, 1.1953125]
    row1 = [1.0, 3 / 8, 0.5, 0.25, 0.25, 0, 0, 0, 0, 0, 1 / 3, 0.5, 0.5, -0.5, 0.25, 1.0]
    assert f[0].tolist() == np.float32(row0).tolist()
    assert f[1].tolist() == np.float32(row1).tolist()
    # a row without off-diagonal entries
    assert f[5].tolist() == np.float32([1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0.5, 0, 0, 0]).tolist()


def test_half_decoding_exact(oracle_mod):
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    ref = bits.view(np.float16).astype(np.float32)
    ok = ~np.isnan(ref)
    # identity layer weights pick one half value per output: W3 row q = e_v, all else 0
    w = np.zeros(oracle_mod.NPARAM, np.uint16)
    b3 = oracle_mod.NPARAM - 3
    feat = np.zeros((1, 16), np.float32)
    got = []
    for chunk in np.array_split(bits[ok], 64):
        for h in chunk[:8]:
            w[b3] = h
            got.append((oracle_mod.mlp_forward(w, feat)[0, 0], np.uint16(h).view(np.float16).astype(np.float32)))
    assert all(a == b for a, b in got)


def test_mlp_forward_matches_numpy(oracle_mod):
    rng = np.random.default_rng(0)
    w = (rng.normal(size=oracle_mod.NPARAM) * 0.3).astype(np.float16)
    feat = oracle_mod.features(P.varcoef2d(12, 1))
    out = oracle_mod.mlp_forward(w.view(np.uint16), feat)
    wf = w.astype(np.float64)
    o = 0
    W1 = wf[o:o + 1024].reshape(64, 16); o += 1024
    b1 = wf[o:o + 64]; o += 64
    W2 = wf[o:o + 4096].reshape(64, 64); o += 4096
    b2 = wf[o:o + 64]; o += 64
    W3 = wf[o:o + 192].reshape(3, 64); o += 192
    b3 = wf[o:o + 3]
    h1 = np.tanh(feat.astype(np.float64) @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    ref = h2 @ W3.T + b3
    assert np.allclose(out, ref, rtol=1e-4, atol=1e-5)


def test_mlp_backward_against_finite_differences(oracle_mod):
    rng = np.random.default_rng(1)
    w = rng.normal(size=oracle_mod.NPARAM) * 0.3
    feat = oracle_mod.features(P.varcoef2d(6, 2))
    dout = rng.normal(size=(feat.shape[0], 3))
    grad, out = oracle_mod.mlp_backward(w, feat, dout)
    L = lambda ww: float((oracle_mod.mlp_backward(ww, feat, dout)[1] * dout).sum())
    for k in rng.choice(oracle_mod.NPARAM, 40, replace=False):
        e = np.zeros_like(w)
        e[k] = 1e-6
        fd = (L(w + e) - L(w - e)) / 2e-6
        assert fd == pytest.approx(grad[k], rel=1e-5, abs=1e-8), k


def test_twogrid_loss_against_dense_and_fd(oracle_mod):
    A = P.fem2d(14, 5)
    H = oracle_mod.Hierarchy(A, coarse_max=16, max_levels=2)
    assert H.nlevels == 2
    levs, Ad, Pm = dense_hierarchy(H)
    A0 = Ad[0]
    T = np.eye(A.n) - Pm[0] @ np.linalg.solve(Ad[1], Pm[0].T @ A0)
    Dinv = 1.0 / np.diag(A0)
    rng = np.random.default_rng(3)
    coef = np.column_stack([rng.uniform(0.3, 0.8, A.n), rng.uniform(-0.2, 0.2, A.n), rng.uniform(-0.1, 0.1, A.n)])
    Lval, grad = H.twogrid_loss(coef, nvec=3, seed=7)
    # dense restatement of the two-grid error propagation on the same error vectors:
    # e0 from the counter generator reproduced through the zero smoother and T
    L0, _ = H.twogrid_loss(np.zeros_like(coef), nvec=3, seed=7)
    G = (np.diag(coef[:, 0]) + np.diag(coef[:, 1]) @ np.diag(Dinv) @ A0
         + np.diag(coef[:, 2]) @ (np.diag(Dinv) @ A0) @ (np.diag(Dinv) @ A0)) @ np.diag(Dinv)
    E = T @ (np.eye(A.n) - G @ A0)
    # the worst-case factor bounds every measured ratio
    # the exact value: the same error vectors e0 (uniform in [-1, 1) from the
    # counter splitmix64(seed ^ (v + 1) << 44 ^ i), top 53 bits), propagated densely
    def e0(v):
        z = P.splitmix64(np.uint64(7) ^ (np.uint64(v + 1) << np.uint64(44)) ^ np.arange(A.n, dtype=np.uint64))
        return 2.0 * ((z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53) - 1.0
    ratio = lambda M, e: float((M @ e) @ A0 @ (M @ e) / (e @ A0 @ e))
    assert Lval == pytest.approx(np.mean([ratio(E, e0(v)) for v in range(3)]), rel=1e-12)
    assert L0 == pytest.approx(np.mean([ratio(T, e0(v)) for v in range(3)]), rel=1e-12)
    # and the worst-case factor bounds it
    w, V = np.linalg.eigh(A0)
    S = V @ np.diag(np.sqrt(w)) @ V.T
    Si = V @ np.diag(1 / np.sqrt(w)) @ V.T
    rho_E = np.linalg.norm(S @ E @ Si, 2) ** 2
    assert 0 < Lval <= rho_E * (1 + 1e-10)
    for k in rng.choice(coef.size, 12, replace=False):
        c = coef.copy().reshape(-1)
        c[k] += 1e-6
        lp, _ = H.twogrid_loss(c.reshape(-1, 3), 3, 7, grad=False)
        c[k] -= 2e-6
        lm, _ = H.twogrid_loss(c.reshape(-1, 3), 3, 7, grad=False)
        assert (lp - lm) / 2e-6 == pytest.approx(grad.reshape(-1)[k], rel=1e-4, abs=1e-9)
    # damped Jacobi reduces the error better than no smoothing at all
    om = levs[0].omega
    LJ, _ = H.twogrid_loss(np.column_stack([np.full(A.n, om), np.zeros(A.n), np.zeros(A.n)]), 3, 7, False)
    assert LJ < L0


# ------------------------------------------------------------ nonsymmetric systems
def test_hess_rho_against_lapack(oracle_mod):
    """The shifted complex QR's largest modulus equals LAPACK's, also for
    Hessenberg matrices with complex conjugate eigenvalue pairs."""
    rng = np.random.default_rng(7)
    for m in (1, 2, 3, 5, 8):
        for _ in range(6):
            H = np.triu(rng.normal(size=(m, m)), -1)
            ev = np.linalg.eigvals(H)
            assert oracle_mod.hess_rho(H) == pytest.approx(np.abs(ev).max(), rel=1e-12)
    R = np.array([[0.0, -2.0], [2.0, 0.0]])  # a pure rotation: eigenvalues +-2i
    assert oracle_mod.hess_rho(R) == pytest.approx(2.0, rel=1e-14)


def test_lu_solve_against_lapack(oracle_mod):
    rng = np.random.default_rng(8)
    for n in (1, 4, 17, 40):
        A = rng.normal(size=(n, n))
        b = rng.normal(size=n)
        LU, piv = oracle_mod.lu(A)
        assert np.allclose(oracle_mod.lu_solve(LU, piv, b), np.linalg.solve(A, b), rtol=1e-11, atol=1e-11)
    assert oracle_mod.lu(np.zeros((3, 3))) is None


def test_rho_estimate_nonsymmetric_full_krylov_space(oracle_mod):
    """With m = n Arnoldi steps the Hessenberg matrix is similar to
    |D|^-1/2 A |D|^-1/2: rho equals its spectral radius."""
    A = P.convdiff2d(2, 3, pe=3.0)  # 4 x 4, nonsymmetric
    D = A.to_dense()
    dh = 1.0 / np.sqrt(np.abs(np.diag(D)))
    M = dh[:, None] * D * dh[None, :]
    rho, _ = oracle_mod.rho_estimate(A, seed=1, level=0, m=A.n, symmetric=False)
    assert rho == pytest.approx(np.abs(np.linalg.eigvals(M)).max(), rel=1e-12)
    rho_sym, _ = oracle_mod.rho_estimate(A, seed=1, level=0, m=A.n, symmetric=True)
    assert rho_sym != pytest.approx(rho, rel=1e-6)  # the symmetric part's estimate differs


def test_fgmres_nonsymmetric_manufactured(oracle_mod):
    A = P.convdiff2d(30, 5, pe=2.0)
    xs = np.sin(np.arange(A.n) * 0.07)
    b = A.matvec(xs)
    H = oracle_mod.Hierarchy(A, coarse_max=16, outer=1, restart=10, symmetric=0)
    x, info = H.solve(b, tol=1e-10, max_iter=300)
    assert info["status"] == 0 and info["relres"] <= 1e-10
    assert np.linalg.norm(b - A.matvec(x)) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= np.linalg.cond(A.to_dense()) * 1e-10


# ----------------------------------------------------------- batches of systems
def test_subsystem_of_joint_hierarchy_is_its_own_hierarchy(oracle_mod):
    """Independent systems set up together as one block-diagonal matrix: the
    first system starts at row 0, so its MIS priorities are those of its own
    setup, and with a fixed omega and the same depth its part of the joint
    hierarchy is the hierarchy of its own setup and solves bit for bit the same.
    A row range that cuts a connected system is rejected."""
    A0, A1 = P.varcoef2d(30, 5), P.poisson2d(23)
    kw = dict(alpha=0.25, seed=3, omega_mode=1, omega=0.6)
    own = oracle_mod.Hierarchy(A0, **kw)
    joint = oracle_mod.Hierarchy(P.block_diag([A0, A1]), max_levels=own.nlevels, **kw)
    sub = joint.subsystem(0, A0.n)
    assert sub.nlevels == own.nlevels == joint.nlevels
    for k in range(own.nlevels):
        a, b = own.level(k), sub.level(k)
        assert a.n == b.n and np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.col, b.col)
        assert np.array_equal(a.val, b.val) and np.array_equal(a.B, b.B)
        if k < own.nlevels - 1:
            assert np.array_equal(a.agg, b.agg) and np.array_equal(a.P, b.P)
    rhs = P.rhs_uniform(A0.n, 4)
    xa, ia = own.solve(rhs, tol=0.0, max_iter=5)
    xb, ib = sub.solve(rhs, tol=0.0, max_iter=5)
    assert np.array_equal(xa, xb) and np.array_equal(ia["hist"], ib["hist"])
    # the second system's part has the second block's rows on every level
    sub1 = joint.subsystem(A0.n, A0.n + A1.n)
    assert sum(sub1.level(k).n for k in range(sub1.nlevels)) + sum(
        sub.level(k).n for k in range(sub.nlevels)) == sum(joint.level(k).n for k in range(joint.nlevels))
    with pytest.raises(ValueError):
        joint.subsystem(0, A0.n // 2)


def test_openmp_timing_build_matches_parity_build(oracle_mod):
    """The CPU-baseline timing build (solve stage and the heavy setup loops on all
    host cores) computes the same hierarchy bit for bit and the same solve up to
    the order of its chunked inner products."""
    A = P.varcoef3d(24, 2)
    b = P.rhs_uniform(A.n, 5)
    hs = oracle_mod.Hierarchy(A, alpha=0.5, seed=2)
    ho = oracle_mod.Hierarchy(A, omp=True, alpha=0.5, seed=2)
    assert ho.nlevels == hs.nlevels
    for k in range(hs.nlevels):
        a, c = hs.level(k), ho.level(k)
        assert np.array_equal(a.col, c.col) and np.array_equal(a.val, c.val) and a.omega == c.omega
        if k < hs.nlevels - 1:
            assert np.array_equal(a.agg, c.agg) and np.array_equal(a.P, c.P)
    xs, i_s = hs.solve(b, tol=1e-8)
    xo, i_o = ho.solve(b, tol=1e-8)
    assert abs(i_s["iters"] - i_o["iters"]) <= 1 and i_o["relres"] <= 1e-8
    if i_s["iters"] == i_o["iters"]:
        assert np.linalg.norm(xs - xo) <= 1e-10 * np.linalg.norm(xs)
    assert oracle_mod.threads(omp=False) == 1 and oracle_mod.threads(omp=True) >= 1


def test_cycle_trace_follows_alg4_alg5(oracle_mod):
    """The oracle's cycle trace obeys the control flow of Alg. 4 / Alg. 5: the
    preconditioner applications equal the flexible-CG iterations; Alg. 5 at level
    m runs once per visit of level m-1 (for m-1 among the Krylov-accelerated
    levels) and visits level m once more for every second inner step taken;
    Alg. 4 visits the next level once; the coarsest is solved once per visit of
    the level above.  With t = 0 the second step always runs; with a threshold
    beyond any norm ratio the first step is always accepted."""
    A = P.poisson3d(20)
    b = P.rhs_uniform(A.n, 1)
    for kw in ({}, {"kcycle_levels": 1}, {"kcycle_levels": 0}, {"kcycle_t": 0.0}, {"kcycle_t": 1e300}):
        o = oracle_mod.Hierarchy(A, alpha=0.5, seed=1, **kw)
        x, info = o.solve(b, tol=1e-8)
        t = o.cycle_trace()
        L = o.nlevels
        kl = kw.get("kcycle_levels", 2)
        assert L >= 4 and t["visits"][0] == info["iters"]
        for m in range(1, L):
            k = m - 1
            if m < L - 1 and k < kl:
                assert t["kcalls"][m] == t["visits"][k]
                assert 0 <= t["second"][m] <= t["kcalls"][m]
                assert t["visits"][m] == t["visits"][k] + t["second"][m]
            else:
                assert t["kcalls"][m] == 0 and t["visits"][m] == t["visits"][k]
        if kw.get("kcycle_t") == 0.0:
            assert all(t["second"][m] == t["kcalls"][m] for m in range(1, L - 1))
        if kw.get("kcycle_t") == 1e300:
            assert t["second"].sum() == 0
