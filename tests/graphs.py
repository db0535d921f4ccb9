"""Seeded synthetic graphs in CSR form (input generator only; no method arithmetic)."""
import numpy as np


def to_csr(n, edges):
    """Symmetric CSR (row_ptr int64, col uint32, rows sorted) from undirected pairs."""
    adj = [set() for _ in range(n)]
    for a, b in edges:
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    rp = np.zeros(n + 1, np.int64)
    for i in range(n):
        rp[i + 1] = rp[i] + len(adj[i])
    col = np.array([j for i in range(n) for j in sorted(adj[i])], np.uint32)
    return rp, col


def erdos_renyi(n, p, seed):
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < p
    return to_csr(n, zip(iu[0][keep].tolist(), iu[1][keep].tolist()))


def geometric(n, radius, seed):
    """Random points in the unit square joined when closer than radius (SCO-like locality),
    numbered in row-major order of a coarse grid so that nearby indices are nearby points."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    order = np.lexsort((pts[:, 0], np.floor(pts[:, 1] * 16)))
    pts = pts[order]
    d = np.linalg.norm(pts[:, None, :] - pts[None, :, :], axis=2)
    iu = np.triu_indices(n, 1)
    keep = d[iu] < radius
    return to_csr(n, zip(iu[0][keep].tolist(), iu[1][keep].tolist()))


def clique(n):
    return to_csr(n, [(a, b) for a in range(n) for b in range(a + 1, n)])


def path(n):
    return to_csr(n, [(a, a + 1) for a in range(n - 1)])


def star(n):
    return to_csr(n, [(0, b) for b in range(1, n)])


def empty(n):
    return to_csr(n, [])


def lattice(Lx, Ly):
    e = []
    for y in range(Ly):
        for x in range(Lx):
            i = x + Lx * y
            if x + 1 < Lx:
                e.append((i, i + 1))
            if y + 1 < Ly:
                e.append((i, i + Lx))
    return to_csr(Lx * Ly, e)


def shuffled(n, rp, col, seed):
    """Same graph with vertices renumbered by a seeded permutation."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    edges = []
    for i in range(n):
        for j in col[rp[i]:rp[i + 1]]:
            if i < j:
                edges.append((perm[i], perm[int(j)]))
    return to_csr(n, edges)
