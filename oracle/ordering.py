"""Near-field block ordering (Sec. 3.3, Algorithm 1) with reverse Cuthill-McKee.

Algorithm 1: nodes = leaf clusters, edges = near-field leaf interactions, a bandwidth
reducing renumbering of the nodes, then the unknowns renumbered leaf by leaf in the new
node order.  The paper does not fix the start node, tie breaks or disconnected graphs;
the reading used here:

* components are taken in order of their lowest node index;
* in each component the start node is a George-Liu pseudo-peripheral node, searched
  from the component's minimum-degree node (lowest index on ties): build the rooted
  level structure, take the minimum-degree node (lowest index) of the last level, and
  move there while the depth grows;
* Cuthill-McKee visits breadth first, each node's unvisited neighbours appended in
  ascending (degree, index);
* the whole concatenated sequence is reversed.

Parity unpinned beyond: bijectivity, bandwidth not above the input order's, and
bandwidth close to scipy's reverse_cuthill_mckee (which uses another start rule).
"""
import numpy as np


def adjacency(n, pairs):
    adj = [set() for _ in range(n)]
    for t, s in pairs:
        if t != s:
            adj[t].add(s)
            adj[s].add(t)
    return [sorted(a) for a in adj]


def _levels(adj, root, allowed):
    depth = {root: 0}
    levels = [[root]]
    while True:
        nxt = []
        for u in levels[-1]:
            for v in adj[u]:
                if v in allowed and v not in depth:
                    depth[v] = len(levels)
                    nxt.append(v)
        if not nxt:
            return levels
        levels.append(nxt)


def pseudo_peripheral(adj, comp):
    allowed = set(comp)
    deg = {u: len(adj[u]) for u in comp}
    r = min(comp, key=lambda u: (deg[u], u))
    lv = _levels(adj, r, allowed)
    while True:
        x = min(lv[-1], key=lambda u: (deg[u], u))
        lx = _levels(adj, x, allowed)
        if len(lx) > len(lv):
            r, lv = x, lx
        else:
            return r


def rcm(n, pairs):
    """Returns order[p] = old node id placed at new position p."""
    adj = adjacency(n, pairs)
    deg = [len(a) for a in adj]
    seen = [False] * n
    seq = []
    for s in range(n):
        if seen[s]:
            continue
        comp = []                                # the component of s (plain BFS)
        stack = [s]
        seen_c = {s}
        while stack:
            u = stack.pop()
            comp.append(u)
            for v in adj[u]:
                if v not in seen_c:
                    seen_c.add(v)
                    stack.append(v)
        start = pseudo_peripheral(adj, comp)
        seen[start] = True
        q = [start]
        head = 0
        while head < len(q):
            u = q[head]
            head += 1
            nb = sorted((v for v in adj[u] if not seen[v]), key=lambda v: (deg[v], v))
            for v in nb:
                seen[v] = True
                q.append(v)
        seq.extend(q)
    return np.array(seq[::-1], dtype=np.int64)


def bandwidth(n, pairs, order=None):
    pos = np.arange(n) if order is None else np.argsort(order)
    b = 0
    for t, s in pairs:
        b = max(b, abs(int(pos[t]) - int(pos[s])))
    return b
