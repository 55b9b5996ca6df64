"""Octree cluster tree (Sec. 2; Sec. 4 uniform model) and the admissibility-based block
partition (Eq. 8, Fig. 1) of the H-matrix.

Cluster tree.  Points are the RWG edge midpoints.  The root is the axis-aligned cube
anchored at the minimum corner of the mesh vertices with side = the largest extent.
A cube is split at its centre, a point goes to the upper half of an axis when its
coordinate is >= the midpoint; child index = x bit 0, y bit 1, z bit 2 (Morton order);
empty children are dropped.  A node is a leaf when it holds at most ``leaf_size``
points (the paper stops when a box has fewer than the leaf size; the off-by-one is a
stated reading) or reaches depth ``max_depth``.  Leaves are numbered in depth-first
order; inside a leaf the points keep ascending original index.  Unknowns renumbered in
that order give the cluster order, and every node covers a contiguous index range.
``fixed_level`` instead splits every node to exactly that depth (for the Sec. 3 plate
example with oct-tree level 2 / 3).

Partition.  diam(t) is the diagonal of the bounding box of all vertices of the support
triangles of t's bases; dist(t, s) the distance between the two boxes (0 if they
overlap).  A pair is admissible (far) when min(diam t, diam s) <= eta * dist(t, s)
(Eq. 8).  Starting from (root, root): admissible -> far block; two leaves -> near
block; otherwise split whichever node is not a leaf (both if neither is).
"""
import numpy as np


class Node:
    __slots__ = ("lo", "hi", "children", "depth", "box_lo", "box_hi", "leaf_id", "idx")

    def __init__(self, depth):
        self.depth = depth
        self.children = []
        self.leaf_id = -1


def build_tree(points, leaf_size=64, max_depth=20, vertices=None, fixed_level=None):
    pts = np.asarray(points, dtype=np.float64)
    ref = pts if vertices is None else np.asarray(vertices, dtype=np.float64)
    lo = ref.min(axis=0)
    side = float((ref.max(axis=0) - lo).max())
    order = []
    leaves = []

    def rec(idx, corner, s, depth):
        node = Node(depth)
        node.lo = len(order)
        if fixed_level is not None:
            is_leaf = depth >= fixed_level
        else:
            is_leaf = len(idx) <= leaf_size or depth >= max_depth
        if is_leaf:
            node.idx = np.sort(idx)
            order.extend(node.idx.tolist())
            node.leaf_id = len(leaves)
            leaves.append(node)
        else:
            mid = corner + 0.5 * s
            p = pts[idx]
            code = ((p[:, 0] >= mid[0]).astype(np.int64)
                    | ((p[:, 1] >= mid[1]).astype(np.int64) << 1)
                    | ((p[:, 2] >= mid[2]).astype(np.int64) << 2))
            for ch in range(8):
                sel = idx[code == ch]
                if sel.size == 0:
                    continue
                off = np.array([(ch >> 0) & 1, (ch >> 1) & 1, (ch >> 2) & 1], dtype=np.float64) * 0.5 * s
                node.children.append(rec(sel, corner + off, 0.5 * s, depth + 1))
            if not node.children:
                raise RuntimeError("empty split")
        node.hi = len(order)
        return node

    root = rec(np.arange(len(pts)), lo, side, 0)
    perm = np.array(order, dtype=np.int32)
    return root, leaves, perm


def attach_boxes(root, perm, blo, bhi):
    """Per node: bounding box of the support-triangle vertices of its bases."""
    lo_c = blo[perm]
    hi_c = bhi[perm]

    def rec(node):
        node.box_lo = lo_c[node.lo:node.hi].min(axis=0)
        node.box_hi = hi_c[node.lo:node.hi].max(axis=0)
        for ch in node.children:
            rec(ch)

    rec(root)


def _diam(n):
    return float(np.linalg.norm(n.box_hi - n.box_lo))


def _dist(a, b):
    gap = np.maximum(0.0, np.maximum(a.box_lo - b.box_hi, b.box_lo - a.box_hi))
    return float(np.linalg.norm(gap))


def partition(root, eta=1.0):
    """Returns (near, far): near = list of (leaf_t, leaf_s) over ALL ordered leaf pairs;
    far = list of (node_t, node_s) over all ordered admissible pairs."""
    near, far = [], []
    stack = [(root, root)]
    while stack:
        t, s = stack.pop()
        if min(_diam(t), _diam(s)) <= eta * _dist(t, s):
            far.append((t, s))
        elif not t.children and not s.children:
            near.append((t.leaf_id, s.leaf_id))
        elif not t.children:
            for c in s.children:
                stack.append((t, c))
        elif not s.children:
            for c in t.children:
                stack.append((c, s))
        else:
            for a in t.children:
                for c in s.children:
                    stack.append((a, c))
    return near, far
