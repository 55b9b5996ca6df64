"""Seeded synthetic surface meshes and the RWG basis built on them.

Meshes stand in for the paper's workloads (Sec. 5: plates and closed bodies meshed
at about lambda/10).  Two families:

* icosphere: the regular icosahedron, each triangle split into four through its edge
  midpoints ``d`` times, every vertex projected onto the sphere of radius ``a``
  (20*4^d triangles, 30*4^d edges, all interior on the closed surface);
* plate: an n x n grid on [0,W]^2 in the z = 0 plane, every square cut along its
  (i,j)->(i+1,j+1) diagonal, interior vertices jittered in x and y by
  U(-j*h, j*h) drawn from ``numpy.random.default_rng(seed)`` (3n^2 - 2n interior
  edges).

RWG functions (Sec. 2, the basis of Eq. 7): one per interior edge, T+ is the lower
numbered adjacent triangle, the free vertex is the vertex of each triangle opposite
the edge.  Basis order: interior edges sorted by (smaller vertex id, larger vertex id).
"""
import numpy as np


def icosphere(d, a):
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(d):
        mid = {}

        def midpoint(i, j):
            key = (min(i, j), max(i, j))
            if key not in mid:
                p = verts[i] + verts[j]
                verts.append(p / np.linalg.norm(p))
                mid[key] = len(verts) - 1
            return mid[key]

        nf = []
        for (i, j, k) in faces:
            ij, jk, ki = midpoint(i, j), midpoint(j, k), midpoint(k, i)
            nf += [(i, ij, ki), (j, jk, ij), (k, ki, jk), (ij, jk, ki)]
        faces = nf
    V = np.array(verts) * a
    T = np.array(faces, dtype=np.int32)
    return V, T


def plate(n, width, jitter=0.1, seed=0):
    h = width / n
    xs = np.linspace(0.0, width, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    V = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        dx = rng.uniform(-jitter * h, jitter * h, size=(V.shape[0], 2))
        ij = np.stack(np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy"), -1).reshape(-1, 2)
        interior = (ij[:, 0] > 0) & (ij[:, 0] < n) & (ij[:, 1] > 0) & (ij[:, 1] < n)
        V[interior, :2] += dx[interior]
    T = []
    for j in range(n):
        for i in range(n):
            v00 = j * (n + 1) + i
            v10 = v00 + 1
            v01 = v00 + (n + 1)
            v11 = v01 + 1
            T.append((v00, v10, v11))
            T.append((v00, v11, v01))
    return V, np.array(T, dtype=np.int32)


class RWG:
    """RWG basis data: for basis n, ``tri[n] = (T+, T-)``, ``free[n] = (v+, v-)``
    (vertex ids opposite the edge), ``edge[n] = (va, vb)`` and ``length[n]``."""

    def __init__(self, V, T):
        edges = {}
        for t, (a, b, c) in enumerate(T):
            for (p, q, r) in ((a, b, c), (b, c, a), (c, a, b)):
                key = (min(p, q), max(p, q))
                edges.setdefault(key, []).append((t, r))
        keys = sorted(k for k, lst in edges.items() if len(lst) == 2)
        bad = [k for k, lst in edges.items() if len(lst) > 2]
        if bad:
            raise ValueError("non-manifold mesh edge")
        nb = len(keys)
        self.V = np.asarray(V, dtype=np.float64)
        self.T = np.asarray(T, dtype=np.int32)
        self.edge = np.array(keys, dtype=np.int32).reshape(nb, 2)
        self.tri = np.empty((nb, 2), dtype=np.int32)
        self.free = np.empty((nb, 2), dtype=np.int32)
        for n, k in enumerate(keys):
            (t0, r0), (t1, r1) = sorted(edges[k])
            self.tri[n] = (t0, t1)
            self.free[n] = (r0, r1)
        self.length = np.linalg.norm(self.V[self.edge[:, 1]] - self.V[self.edge[:, 0]], axis=1)
        self.n = nb

    def midpoints(self):
        return 0.5 * (self.V[self.edge[:, 0]] + self.V[self.edge[:, 1]])

    def tri_areas(self):
        P = self.V[self.T]
        return 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)

    def support_boxes(self):
        """Per basis: AABB (lo, hi) of the vertices of its two support triangles."""
        P = self.V[self.T[self.tri]]            # nb x 2 x 3 x 3
        P = P.reshape(self.n, 6, 3)
        return P.min(axis=1), P.max(axis=1)
