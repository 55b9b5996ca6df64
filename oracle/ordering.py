"""Near-field block ordering (Sec. 3.3, Algorithm 1) with reverse Cuthill-McKee or Sloan.

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

Sloan's profile and wavefront reducing ordering (the best of the orderings compared in
Sec. 3.3, Tables 3-4; the paper gives no details of it), as read here from Sloan's
published algorithm (S. W. Sloan, Int. J. Numer. Meth. Eng. 23, 1986):

* per component (components in order of their lowest node), a start node s and an end
  node e: s = the minimum-(degree, index) node; build the rooted level structure of s;
  take the last level's nodes in ascending (degree, index), keeping the first node of
  each degree; for each of them build its level structure: if it is deeper than s's and
  narrower than every one seen so far, it becomes s and the search restarts; otherwise,
  if it is narrower than every one seen so far, it becomes e;
* priorities P(i) = W1 dist(i, e) - W2 (deg(i) + 1) with W1 = 2, W2 = 1;
* statuses inactive / preactive / active / postactive; s starts preactive in the queue;
  repeatedly the queued node of highest priority (lowest index on ties) is numbered: if
  it was preactive, each neighbour gains W2 and an inactive neighbour becomes preactive
  and is queued; the node becomes postactive; each preactive neighbour j becomes active
  and gains W2, and each neighbour k of j that is not postactive gains W2 (an inactive k
  becomes preactive and is queued);
* the numbering is not reversed.

Pinned by: bijectivity, the end-to-end order of a path, a small graph numbered by hand,
and a profile not above RCM's on grid graphs (profile reduction is the method's aim).
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


def _bfs_dist(adj, root, allowed):
    dist = {root: 0}
    q = [root]
    head = 0
    while head < len(q):
        u = q[head]
        head += 1
        for v in adj[u]:
            if v in allowed and v not in dist:
                dist[v] = dist[u] + 1
                q.append(v)
    return dist


def sloan_endpoints(adj, comp):
    """(s, e) of one component, as described in the module docstring."""
    allowed = set(comp)
    deg = {u: len(adj[u]) for u in comp}
    s = min(comp, key=lambda u: (deg[u], u))
    while True:
        ls = _levels(adj, s, allowed)
        last = sorted(ls[-1], key=lambda u: (deg[u], u))
        cand, seen_deg = [], set()
        for u in last:                                # one node per degree
            if deg[u] not in seen_deg:
                seen_deg.add(deg[u])
                cand.append(u)
        wmin, e, restart = None, None, False
        for i in cand:
            li = _levels(adj, i, allowed)
            wi = max(len(L) for L in li)
            if len(li) > len(ls) and (wmin is None or wi < wmin):
                s, restart = i, True
                break
            if wmin is None or wi < wmin:
                e, wmin = i, wi
        if not restart:
            return s, e


def sloan(n, pairs, w1=2, w2=1):
    """Returns order[p] = old node id placed at new position p (Sloan's ordering)."""
    adj = adjacency(n, pairs)
    deg = [len(a) for a in adj]
    INACTIVE, PREACTIVE, ACTIVE, POSTACTIVE = 0, 1, 2, 3
    status = [INACTIVE] * n
    prio = [0] * n
    done = [False] * n
    seq = []
    for c0 in range(n):
        if done[c0]:
            continue
        comp = sorted(_bfs_dist(adj, c0, set(range(n))).keys())
        for u in comp:
            done[u] = True
        s, e = sloan_endpoints(adj, comp)
        dist = _bfs_dist(adj, e, set(comp))
        for u in comp:
            prio[u] = w1 * dist[u] - w2 * (deg[u] + 1)
        status[s] = PREACTIVE
        queue = [s]
        while queue:
            i = max(queue, key=lambda u: (prio[u], -u))
            queue.remove(i)
            if status[i] == PREACTIVE:
                for j in adj[i]:
                    prio[j] += w2
                    if status[j] == INACTIVE:
                        status[j] = PREACTIVE
                        queue.append(j)
            seq.append(i)
            status[i] = POSTACTIVE
            for j in adj[i]:
                if status[j] == PREACTIVE:
                    status[j] = ACTIVE
                    prio[j] += w2
                    for k in adj[j]:
                        if status[k] != POSTACTIVE:
                            prio[k] += w2
                            if status[k] == INACTIVE:
                                status[k] = PREACTIVE
                                queue.append(k)
    return np.array(seq, dtype=np.int64)


def profile(n, pairs, order=None):
    """Envelope size: sum over rows i of i - (lowest column j <= i with a_ij != 0), in the
    numbering given by order (pattern symmetric, diagonal nonzero)."""
    pos = np.arange(n) if order is None else np.argsort(order)
    first = np.arange(n)
    for t, s in pairs:
        a, b = int(pos[t]), int(pos[s])
        if a > b:
            a, b = b, a
        first[b] = min(first[b], a)
    return int(np.sum(np.arange(n) - first))
