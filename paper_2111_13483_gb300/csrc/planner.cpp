// Host planner of the hmsolve library: description checks, the near-field block order
// (Sec. 3.3, Algorithm 1 with reverse Cuthill-McKee), the symbolic fill of the scaling
// coefficients (Sec. 3.3, Figs. 3b-7b), storage layout and the far-field incidence lists.
// Integer work only; every floating-point step runs on the device.
#include <algorithm>
#include <array>
#include <map>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "hm_internal.h"

namespace hm {

static int fail(hm_ctx *h, const char *msg)
{
    h->err = msg;
    return HM_EINVAL;
}

int validate_and_copy(hm_ctx *h, const hm_desc *d)
{
    if (!d) return fail(h, "null description");
    if (d->n <= 0 || d->n_leaves <= 0 || d->n_leaves > d->n) return fail(h, "bad n / n_leaves");
    if (!d->perm || !d->leaf_ptr) return fail(h, "null perm / leaf_ptr");
    const int n = d->n, nl = d->n_leaves;
    h->n = n;
    h->nl = nl;
    h->perm.assign(d->perm, d->perm + n);
    h->leaf_ptr.assign(d->leaf_ptr, d->leaf_ptr + nl + 1);
    if (h->leaf_ptr[0] != 0 || h->leaf_ptr[nl] != n) return fail(h, "leaf_ptr must start at 0 and end at n");
    for (int l = 0; l < nl; ++l) {
        int sz = h->leaf_ptr[l + 1] - h->leaf_ptr[l];
        if (sz < 1 || sz > 64) return fail(h, "leaf sizes must be 1..64");
    }
    {
        std::vector<char> seen(n, 0);
        for (int i = 0; i < n; ++i) {
            int p = h->perm[i];
            if (p < 0 || p >= n || seen[p]) return fail(h, "perm is not a permutation");
            seen[p] = 1;
        }
    }
    if (d->n_near < nl || !d->near_t || !d->near_s || !d->near_off || !d->near_data)
        return fail(h, "near pairs missing");
    h->near_t.assign(d->near_t, d->near_t + d->n_near);
    h->near_s.assign(d->near_s, d->near_s + d->n_near);
    h->near_off.assign(d->near_off, d->near_off + d->n_near);
    h->near_len = d->near_len;
    std::vector<char> diag(nl, 0);
    int64_t covered = 0;
    {
        std::vector<std::pair<int, int>> pr;
        pr.reserve(d->n_near);
        for (int b = 0; b < d->n_near; ++b) {
            int t = h->near_t[b], s = h->near_s[b];
            if (t < 0 || s >= nl || t > s) return fail(h, "near pair out of range or t > s");
            int64_t m = h->leaf_ptr[t + 1] - h->leaf_ptr[t], c = h->leaf_ptr[s + 1] - h->leaf_ptr[s];
            if (h->near_off[b] < 0 || h->near_off[b] + m * c > d->near_len) return fail(h, "near block outside near_data");
            if (t == s) diag[t] = 1;
            covered += (t == s) ? m * c : 2 * m * c;
            pr.push_back({t, s});
        }
        std::sort(pr.begin(), pr.end());
        for (size_t i = 1; i < pr.size(); ++i)
            if (pr[i] == pr[i - 1]) return fail(h, "duplicate near pair");
    }
    for (int l = 0; l < nl; ++l)
        if (!diag[l]) return fail(h, "every leaf needs its diagonal near block");
    const int nf = d->n_far;
    if (nf < 0) return fail(h, "n_far < 0");
    if (nf > 0 && (!d->far_r0 || !d->far_r1 || !d->far_c0 || !d->far_c1 || !d->far_rank || !d->far_uoff ||
                   !d->far_voff || !d->far_U))
        return fail(h, "far arrays missing");
    h->far_r0.assign(d->far_r0, d->far_r0 + nf);
    h->far_r1.assign(d->far_r1, d->far_r1 + nf);
    h->far_c0.assign(d->far_c0, d->far_c0 + nf);
    h->far_c1.assign(d->far_c1, d->far_c1 + nf);
    h->far_rank.assign(d->far_rank, d->far_rank + nf);
    h->far_uoff.assign(d->far_uoff, d->far_uoff + nf);
    h->far_voff.assign(d->far_voff, d->far_voff + nf);
    h->farU_len = d->far_U_len;
    h->farV_len = d->far_V_len;
    std::vector<char> is_bound(n + 1, 0);
    for (int l = 0; l <= nl; ++l) is_bound[h->leaf_ptr[l]] = 1;
    for (int b = 0; b < nf; ++b) {
        int r0 = h->far_r0[b], r1 = h->far_r1[b], c0 = h->far_c0[b], c1 = h->far_c1[b], r = h->far_rank[b];
        if (r0 < 0 || r0 >= r1 || r1 > c0 || c0 >= c1 || c1 > n) return fail(h, "far block ranges invalid");
        if (!is_bound[r0] || !is_bound[r1] || !is_bound[c0] || !is_bound[c1])
            return fail(h, "far block ranges must be unions of whole leaves");
        int64_t m = r1 - r0, c = c1 - c0;
        if (r < -1 || r > std::min(m, c)) return fail(h, "far rank out of range");
        if (r < 0) {
            if (h->far_uoff[b] < 0 || h->far_uoff[b] + m * c > d->far_U_len) return fail(h, "dense far block outside far_U");
        } else {
            if (!d->far_V && r > 0) return fail(h, "far_V missing");
            if (h->far_uoff[b] < 0 || h->far_uoff[b] + m * r > d->far_U_len) return fail(h, "U factor outside far_U");
            if (h->far_voff[b] < 0 || h->far_voff[b] + c * r > d->far_V_len) return fail(h, "V factor outside far_V");
        }
        covered += 2 * m * c;
    }
    if (covered != (int64_t)n * n) return fail(h, "near and far blocks do not cover Z exactly once");
    return HM_OK;
}

// Reverse Cuthill-McKee on the near-field leaf graph (Algorithm 1, step 3): components in
// order of their lowest node; George-Liu pseudo-peripheral start searched from the
// component's minimum-(degree, index) node; neighbours enqueued by ascending (degree,
// index); the whole sequence reversed.
static std::vector<std::vector<int>> bfs_levels(const std::vector<std::vector<int>> &adj, int root,
                                                std::vector<int> &mark, int stamp)
{
    std::vector<std::vector<int>> lv{{root}};
    mark[root] = stamp;
    while (true) {
        std::vector<int> nxt;
        for (int u : lv.back())
            for (int v : adj[u])
                if (mark[v] != stamp) {
                    mark[v] = stamp;
                    nxt.push_back(v);
                }
        if (nxt.empty()) return lv;
        lv.push_back(std::move(nxt));
    }
}

std::vector<int> rcm_order(int nl, const std::vector<int> &t, const std::vector<int> &s)
{
    std::vector<std::vector<int>> adj(nl);
    for (size_t b = 0; b < t.size(); ++b)
        if (t[b] != s[b]) {
            adj[t[b]].push_back(s[b]);
            adj[s[b]].push_back(t[b]);
        }
    for (auto &a : adj) {
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
    }
    std::vector<int> deg(nl);
    for (int i = 0; i < nl; ++i) deg[i] = (int)adj[i].size();
    auto key_less = [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; };
    std::vector<char> seen(nl, 0);
    std::vector<int> mark(nl, -1), seq;
    seq.reserve(nl);
    int stamp = 0;
    for (int s0 = 0; s0 < nl; ++s0) {
        if (seen[s0]) continue;
        // component of s0
        auto comp_lv = bfs_levels(adj, s0, mark, stamp++);
        int r = -1;
        for (auto &L : comp_lv)
            for (int u : L)
                if (r < 0 || key_less(u, r)) r = u;
        auto lv = bfs_levels(adj, r, mark, stamp++);
        while (true) {
            int x = *std::min_element(lv.back().begin(), lv.back().end(), key_less);
            auto lx = bfs_levels(adj, x, mark, stamp++);
            if (lx.size() > lv.size()) {
                r = x;
                lv = std::move(lx);
            } else
                break;
        }
        size_t head = seq.size();
        seen[r] = 1;
        seq.push_back(r);
        while (head < seq.size()) {
            int u = seq[head++];
            std::vector<int> nb;
            for (int v : adj[u])
                if (!seen[v]) nb.push_back(v);
            std::sort(nb.begin(), nb.end(), key_less);
            for (int v : nb) {
                seen[v] = 1;
                seq.push_back(v);
            }
        }
    }
    std::reverse(seq.begin(), seq.end());
    return seq;
}

// Sloan's profile and wavefront reducing ordering (compared in Sec. 3.3, Tables 3-4), from
// Sloan's published algorithm: per component (in order of its lowest node) a start node s and
// an end node e from rooted level structures (s = the minimum-(degree, index) node; the last
// level's nodes in ascending (degree, index), one per degree, are tried: one deeper than s's
// structure and narrower than all tried so far becomes s and the search restarts, one only
// narrower becomes e); priorities 2 dist(i, e) - (deg(i) + 1); then nodes are numbered by
// highest priority (lowest index on ties) from a queue of preactive/active nodes, numbering a
// preactive node raising its neighbours by 1 and activating them, and every neighbour of a node
// that turns active gaining 1 (inactive ones queued as preactive).  Not reversed.
std::vector<int> sloan_order(int nl, const std::vector<int> &t, const std::vector<int> &s)
{
    std::vector<std::vector<int>> adj(nl);
    for (size_t b = 0; b < t.size(); ++b)
        if (t[b] != s[b]) {
            adj[t[b]].push_back(s[b]);
            adj[s[b]].push_back(t[b]);
        }
    for (auto &a : adj) {
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
    }
    std::vector<int> deg(nl);
    for (int i = 0; i < nl; ++i) deg[i] = (int)adj[i].size();
    auto key_less = [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; };
    auto width = [](const std::vector<std::vector<int>> &lv) {
        size_t w = 0;
        for (auto &L : lv) w = std::max(w, L.size());
        return (int)w;
    };
    enum { INACTIVE = 0, PREACTIVE, ACTIVE, POSTACTIVE };
    std::vector<int> status(nl, INACTIVE), mark(nl, -1), seq;
    std::vector<long> prio(nl, 0);
    std::vector<char> placed(nl, 0);
    seq.reserve(nl);
    int stamp = 0;
    for (int c0 = 0; c0 < nl; ++c0) {
        if (placed[c0]) continue;
        auto comp_lv = bfs_levels(adj, c0, mark, stamp++);
        int sn = -1;
        for (auto &L : comp_lv)
            for (int u : L) {
                placed[u] = 1;
                if (sn < 0 || key_less(u, sn)) sn = u;
            }
        // start and end nodes
        int en = sn;
        while (true) {
            auto ls = bfs_levels(adj, sn, mark, stamp++);
            std::vector<int> last = ls.back();
            std::sort(last.begin(), last.end(), key_less);
            std::vector<int> cand;
            for (int u : last)
                if (cand.empty() || deg[cand.back()] != deg[u]) cand.push_back(u);
            int wmin = -1;
            bool restart = false;
            for (int i : cand) {
                auto li = bfs_levels(adj, i, mark, stamp++);
                const int wi = width(li);
                if (li.size() > ls.size() && (wmin < 0 || wi < wmin)) {
                    sn = i;
                    restart = true;
                    break;
                }
                if (wmin < 0 || wi < wmin) {
                    en = i;
                    wmin = wi;
                }
            }
            if (!restart) break;
        }
        // priorities from the distance to the end node
        auto le = bfs_levels(adj, en, mark, stamp++);
        for (size_t d = 0; d < le.size(); ++d)
            for (int u : le[d]) prio[u] = 2L * (long)d - (long)(deg[u] + 1);
        std::vector<int> queue{sn};
        status[sn] = PREACTIVE;
        while (!queue.empty()) {
            size_t bi = 0;
            for (size_t q = 1; q < queue.size(); ++q) {
                const int u = queue[q], b = queue[bi];
                if (prio[u] > prio[b] || (prio[u] == prio[b] && u < b)) bi = q;
            }
            const int i = queue[bi];
            queue.erase(queue.begin() + bi);
            if (status[i] == PREACTIVE)
                for (int j : adj[i]) {
                    prio[j] += 1;
                    if (status[j] == INACTIVE) {
                        status[j] = PREACTIVE;
                        queue.push_back(j);
                    }
                }
            seq.push_back(i);
            status[i] = POSTACTIVE;
            for (int j : adj[i])
                if (status[j] == PREACTIVE) {
                    status[j] = ACTIVE;
                    prio[j] += 1;
                    for (int k : adj[j])
                        if (status[k] != POSTACTIVE) {
                            prio[k] += 1;
                            if (status[k] == INACTIVE) {
                                status[k] = PREACTIVE;
                                queue.push_back(k);
                            }
                        }
                }
        }
    }
    return seq;
}

// Symbolic elimination on bitsets (Sec. 3.3, the fill of Figs. 3b-7b): eliminating block
// k couples every pair of its later neighbours.  Pairs (i, j) in block numbering; returns
// S_k (sorted, > k) as CSR.  closure = false: S_k = the later near-field neighbours of k only
// (the elimination without fill of the null-field comparison).
void symbolic_fill(int nl, const std::vector<int> &pi, const std::vector<int> &pj, std::vector<int> &sptr,
                   std::vector<int> &sidx, bool closure)
{
    const int W = (nl + 63) / 64;
    std::vector<uint64_t> bits((size_t)nl * W, 0);
    for (size_t b = 0; b < pi.size(); ++b) {
        int i = pi[b], j = pj[b];
        if (i == j) continue;
        bits[(size_t)i * W + j / 64] |= 1ull << (j % 64);
        bits[(size_t)j * W + i / 64] |= 1ull << (i % 64);
    }
    sptr.assign(nl + 1, 0);
    sidx.clear();
    std::vector<uint64_t> mask(W);
    std::vector<int> later;
    for (int k = 0; k < nl; ++k) {
        const uint64_t *row = &bits[(size_t)k * W];
        std::fill(mask.begin(), mask.end(), 0);
        later.clear();
        for (int w = k / 64; w < W; ++w) {
            uint64_t x = row[w];
            if (w == k / 64) x &= (k % 64 == 63) ? 0 : (~0ull << (k % 64 + 1));
            mask[w] = x;
            while (x) {
                int bit = __builtin_ctzll(x);
                later.push_back(w * 64 + bit);
                x &= x - 1;
            }
        }
        if (closure)
            for (int a : later) {
                uint64_t *ra = &bits[(size_t)a * W];
                for (int w = k / 64; w < W; ++w) ra[w] |= mask[w];
            }
        sidx.insert(sidx.end(), later.begin(), later.end());
        sptr[k + 1] = (int)sidx.size();
    }
}

// Super-rows of the sweeps (see Plan::xptr): members are SWEEP_SR consecutive blocks in
// sweep order; their dependency lists are merged, the pairs inside the super-row kept apart.
static void plan_superrows(Plan &P)
{
    const int nb = P.nb, SR = SWEEP_SR, nsr = (nb + SR - 1) / SR;
    for (int dir = 0; dir < 2; ++dir) {
        std::vector<int> &xp = P.xptr[dir], &xd = P.xdep[dir], &xo = P.xoff[dir], &xi = P.xint[dir];
        xp.assign(nsr + 1, 0);
        xd.clear();
        xo.clear();
        xi.assign((size_t)nsr * SR * SR, -1);
        for (int r = 0; r < nsr; ++r) {
            int mem[SWEEP_SR], nm = 0;
            for (int s = 0; s < SR && r * SR + s < nb; ++s) mem[nm++] = dir == 0 ? r * SR + s : nb - 1 - (r * SR + s);
            std::map<int, std::vector<int>> deps;   // dependency block -> offset per member
            for (int s = 0; s < nm; ++s) {
                const int b = mem[s];
                const int lo = dir == 0 ? P.rptr[b] : P.sptr[b], hi = dir == 0 ? P.rptr[b + 1] : P.sptr[b + 1];
                for (int e = lo; e < hi; ++e) {
                    const int k = dir == 0 ? P.ridx[e] : P.sidx[e];
                    const int off = dir == 0 ? P.rcol[e] : P.srow[e];
                    int sk = -1;
                    for (int t = 0; t < nm; ++t)
                        if (mem[t] == k) sk = t;
                    if (sk >= 0) {
                        xi[((size_t)r * SR + sk) * SR + s] = off;
                        continue;
                    }
                    std::vector<int> &v = deps[k];
                    if (v.empty()) v.assign(SR, -1);
                    v[s] = off;
                }
            }
            std::vector<int> keys;
            for (auto &kv : deps) keys.push_back(kv.first);
            if (dir == 1) std::reverse(keys.begin(), keys.end());   // the backward sweep adds downwards
            for (int k : keys) {
                xd.push_back(k);
                for (int s = 0; s < SR; ++s) xo.push_back(deps[k][s]);
            }
            xp[r + 1] = (int)xd.size();
        }
    }
    // recent dependencies (chain-and-helpers sweeps), in walk order
    for (int dir = 0; dir < 2; ++dir) {
        P.rec[dir].assign((size_t)nb * SWEEP_T, -1);
        P.reccol[dir].assign((size_t)nb * SWEEP_T, 0);
        for (int b = 0; b < nb; ++b) {
            std::vector<std::pair<int, int>> rv;
            if (dir == 0) {
                for (int p = P.rptr[b + 1] - 1; p >= P.rptr[b] && P.ridx[p] >= b - SWEEP_T; --p)
                    rv.push_back({P.ridx[p], P.rcol[p]});
                std::reverse(rv.begin(), rv.end());   // ascending
            } else
                for (int p = P.sptr[b]; p < P.sptr[b + 1] && P.sidx[p] <= b + SWEEP_T; ++p)
                    rv.push_back({P.sidx[p], P.srow[p]});
            if (dir == 1) std::reverse(rv.begin(), rv.end());   // descending (the backward walk)
            for (size_t j = 0; j < rv.size(); ++j) {
                P.rec[dir][(size_t)b * SWEEP_T + j] = rv[j].first;
                P.reccol[dir][(size_t)b * SWEEP_T + j] = rv[j].second;
            }
        }
    }
}

void plan_order(hm_ctx *h)
{
    Plan &P = h->plan;
    const int nl = h->nl;
    P.nb = nl;
    P.n = h->n;
    if (h->opts.ordering == 1)
        P.order = rcm_order(nl, h->near_t, h->near_s);
    else if (h->opts.ordering == 2)
        P.order = sloan_order(nl, h->near_t, h->near_s);
    else {
        P.order.resize(nl);
        std::iota(P.order.begin(), P.order.end(), 0);
    }
    P.pos.assign(nl, 0);
    for (int p = 0; p < nl; ++p) P.pos[P.order[p]] = p;
    P.size.resize(nl);
    P.boff.assign(nl + 1, 0);
    for (int p = 0; p < nl; ++p) {
        int l = P.order[p];
        P.size[p] = h->leaf_ptr[l + 1] - h->leaf_ptr[l];
        P.boff[p + 1] = P.boff[p] + P.size[p];
    }
    P.new2cl.resize(h->n);
    P.new2orig.resize(h->n);
    P.cl2new.resize(h->n);
    for (int p = 0; p < nl; ++p) {
        int l = P.order[p];
        for (int i = 0; i < P.size[p]; ++i) {
            int cl = h->leaf_ptr[l] + i;
            P.new2cl[P.boff[p] + i] = cl;
            P.cl2new[cl] = P.boff[p] + i;
            P.new2orig[P.boff[p] + i] = h->perm[cl];
        }
    }
    std::vector<int> bi(h->near_t.size()), bj(h->near_t.size());
    P.bandwidth = 0;
    for (size_t b = 0; b < h->near_t.size(); ++b) {
        bi[b] = P.pos[h->near_t[b]];
        bj[b] = P.pos[h->near_s[b]];
        P.bandwidth = std::max(P.bandwidth, std::abs(bi[b] - bj[b]));
    }
    const bool no_fill = h->opts.preconditioner == 2;
    symbolic_fill(nl, bi, bj, P.sptr, P.sidx, !no_fill);
    // near pairs (i > j) as keys i * nl + j, sorted
    std::vector<int64_t> nkey;
    nkey.reserve(bi.size());
    for (size_t b = 0; b < bi.size(); ++b)
        if (bi[b] != bj[b]) nkey.push_back((int64_t)std::max(bi[b], bj[b]) * nl + std::min(bi[b], bj[b]));
    std::sort(nkey.begin(), nkey.end());
    {
        // entries of the coefficient pattern that are not near pairs: the fill-in blocks
        P.fill_e.clear();
        P.fill_k.clear();
        P.fill_ptr.assign(nl + 1, 0);
        for (int k = 0; k < nl; ++k) {
            for (int e = P.sptr[k]; e < P.sptr[k + 1]; ++e)
                if (!std::binary_search(nkey.begin(), nkey.end(), (int64_t)P.sidx[e] * nl + k)) {
                    P.fill_e.push_back(e);
                    P.fill_k.push_back(k);
                }
            P.fill_ptr[k + 1] = (int)P.fill_e.size();
        }
    }
    // layouts
    P.srow.resize(P.sidx.size());
    P.M.assign(nl, 0);
    P.coff.assign(nl + 1, 0);
    P.doff.assign(nl + 1, 0);
    P.max_S = 0;
    P.max_M = 0;
    P.n_updates = 0;
    double macs = 0;
    for (int k = 0; k < nl; ++k) {
        int acc = 0;
        for (int e = P.sptr[k]; e < P.sptr[k + 1]; ++e) {
            P.srow[e] = acc;
            acc += P.size[P.sidx[e]];
        }
        P.M[k] = acc;
        int64_t nk = P.size[k];
        P.coff[k + 1] = P.coff[k] + (int64_t)acc * nk;
        P.doff[k + 1] = P.doff[k] + nk * nk;
        int ns = P.sptr[k + 1] - P.sptr[k];
        P.max_S = std::max(P.max_S, ns);
        P.max_M = std::max(P.max_M, acc);
        P.n_updates += (int64_t)ns * (ns + 1) / 2;
        // complex MACs: explicit inverse n^3, panel n^2 M, updates sum_{i>=j} n_i n_k n_j
        macs += (double)nk * nk * nk + (double)nk * nk * acc;
        double run = 0;
        for (int e = P.sptr[k]; e < P.sptr[k + 1]; ++e) {
            run += P.size[P.sidx[e]];
            if (!no_fill) {
                macs += (double)P.size[P.sidx[e]] * nk * run;
                continue;
            }
            // without fill only the updates of near pairs (and of the diagonal blocks) are made
            const int i = P.sidx[e];
            for (int f = P.sptr[k]; f <= e; ++f) {
                const int j = P.sidx[f];
                if (i == j || std::binary_search(nkey.begin(), nkey.end(), (int64_t)i * nl + j))
                    macs += (double)P.size[i] * (double)P.size[k] * P.size[j];
            }
        }
    }
    P.setup_flops = 8.0 * macs;
    P.coef_entries = P.coff[nl];
    P.diag_entries = P.doff[nl];
    // forward-sweep gather lists: row j <- (k, column offset of block j in panel k)
    std::vector<int> cnt(nl + 1, 0);
    for (int k = 0; k < nl; ++k)
        for (int e = P.sptr[k]; e < P.sptr[k + 1]; ++e) cnt[P.sidx[e] + 1]++;
    P.rptr.assign(nl + 1, 0);
    for (int i = 0; i < nl; ++i) P.rptr[i + 1] = P.rptr[i] + cnt[i + 1];
    P.ridx.resize(P.rptr[nl]);
    P.rcol.resize(P.rptr[nl]);
    P.rent.resize(P.rptr[nl]);
    std::vector<int> fillp(P.rptr.begin(), P.rptr.end() - 1);
    for (int k = 0; k < nl; ++k)
        for (int e = P.sptr[k]; e < P.sptr[k + 1]; ++e) {
            int j = P.sidx[e];
            P.ridx[fillp[j]] = k;
            P.rcol[fillp[j]] = P.srow[e];
            P.rent[fillp[j]] = e;
            fillp[j]++;
        }
    P.pboff.resize(P.sidx.size() + 1);
    for (int k = 0; k < nl; ++k)
        for (int e = P.sptr[k]; e < P.sptr[k + 1]; ++e) P.pboff[e] = P.coff[k] + (int64_t)P.srow[e] * P.size[k];
    P.pboff[P.sidx.size()] = P.coef_entries;
    plan_superrows(P);
}

void plan_far(hm_ctx *h)
{
    FarPlan &F = h->fplan;
    const int nl = h->nl, nf = (int)h->far_rank.size();
    F.nf = nf;
    std::vector<int> leaf_of(h->n + 1, -1);
    for (int l = 0; l < nl; ++l) leaf_of[h->leaf_ptr[l]] = l;
    std::vector<std::vector<int>> lists(nl);
    F.toff.assign(nf + 1, 0);
    for (int b = 0; b < nf; ++b) {
        bool lr = h->far_rank[b] >= 0;
        for (int l = leaf_of[h->far_r0[b]]; l < nl && h->leaf_ptr[l] < h->far_r1[b]; ++l)
            lists[l].push_back((b << 2) | (lr ? 0 : 2));
        for (int l = leaf_of[h->far_c0[b]]; l < nl && h->leaf_ptr[l] < h->far_c1[b]; ++l)
            lists[l].push_back((b << 2) | (lr ? 1 : 3));
        F.toff[b + 1] = F.toff[b] + (lr ? h->far_rank[b] : 0);
    }
    F.tlen = F.toff[nf];
    F.item_blk.resize(F.tlen);
    for (int b = 0; b < nf; ++b)
        for (int64_t e = F.toff[b]; e < F.toff[b + 1]; ++e) F.item_blk[e] = b;
    F.lptr.assign(nl + 1, 0);
    for (int l = 0; l < nl; ++l) F.lptr[l + 1] = F.lptr[l] + (int)lists[l].size();
    F.lent.clear();
    F.lent.reserve(F.lptr[nl]);
    for (int l = 0; l < nl; ++l) F.lent.insert(F.lent.end(), lists[l].begin(), lists[l].end());
    std::vector<std::vector<int>> nl_lists(nl);
    for (size_t b = 0; b < h->near_t.size(); ++b) {
        nl_lists[h->near_t[b]].push_back((int)(b << 1));
        if (h->near_t[b] != h->near_s[b]) nl_lists[h->near_s[b]].push_back((int)((b << 1) | 1));
    }
    F.nptr.assign(nl + 1, 0);
    for (int l = 0; l < nl; ++l) F.nptr[l + 1] = F.nptr[l] + (int)nl_lists[l].size();
    F.nent.clear();
    for (int l = 0; l < nl; ++l) F.nent.insert(F.nent.end(), nl_lists[l].begin(), nl_lists[l].end());
    // phase-2 segments: every list entry of leaf l cut into contraction pieces of <= 32
    F.seg_ptr.assign(nl + 1, 0);
    F.segs.clear();
    for (int l = 0; l < nl; ++l) {
        const int a = h->leaf_ptr[l];
        for (int p = F.lptr[l]; p < F.lptr[l + 1]; ++p) {
            const int b = F.lent[p] >> 2, kind = F.lent[p] & 3;
            const int64_t m = h->far_r1[b] - h->far_r0[b], c = h->far_c1[b] - h->far_c0[b];
            FarSegD g{};
            int K;
            if (kind == 0) {
                g = {h->far_uoff[b] + (a - h->far_r0[b]), F.toff[b], 1, (int)m, 0, 0};
                K = h->far_rank[b];
            } else if (kind == 1) {
                g = {h->far_voff[b] + (a - h->far_c0[b]), F.toff[b], 1, (int)c, 0, 1 | (1 << 1)};
                K = h->far_rank[b];
            } else if (kind == 2) {
                g = {h->far_uoff[b] + (a - h->far_r0[b]), h->far_c0[b], 1, (int)m, 0, 2 << 1};
                K = (int)c;
            } else {
                g = {h->far_uoff[b] + (int64_t)(a - h->far_c0[b]) * m, h->far_r0[b], (int)m, 1, 0, 2 << 1};
                K = (int)m;
            }
            for (int k0 = 0; k0 < K; k0 += 32) {
                FarSegD q = g;
                q.foff += (int64_t)k0 * g.fk;
                q.yrow += k0;
                q.len = std::min(32, K - k0);
                F.segs.push_back(q);
            }
        }
        F.seg_ptr[l + 1] = (int)F.segs.size();
    }
    F.seg_kcum.assign(F.segs.size() + 1, 0);
    for (size_t q = 0; q < F.segs.size(); ++q) F.seg_kcum[q + 1] = F.seg_kcum[q] + F.segs[q].len;
    F.part_ptr.assign((size_t)nl * FAR_PARTS + 1, 0);
    for (int l = 0; l < nl; ++l) {
        const int b = F.seg_ptr[l], e = F.seg_ptr[l + 1];
        const int64_t K = F.seg_kcum[e] - F.seg_kcum[b];
        int q = b;
        for (int p = 0; p < FAR_PARTS; ++p) {
            F.part_ptr[(size_t)l * FAR_PARTS + p] = q;
            const int64_t target = K * (p + 1) / FAR_PARTS;
            while (q < e && F.seg_kcum[q] - F.seg_kcum[b] < target) ++q;
        }
    }
    F.part_ptr[(size_t)nl * FAR_PARTS] = (int)F.segs.size();
    // rank-vector tasks: group the factor columns by the range they contract over
    // (V_b over the column range for t_b, U_b over the row range for s_b), 64 per task,
    // larger tasks first
    std::map<std::pair<int, int>, std::vector<std::array<int64_t, 5>>> by_range;
    for (int b = 0; b < nf; ++b) {
        const int rk = h->far_rank[b];
        if (rk <= 0) continue;
        const int m = h->far_r1[b] - h->far_r0[b], c = h->far_c1[b] - h->far_c0[b];
        for (int l0 = 0; l0 < rk; l0 += 64) {
            const int64_t cols = std::min(64, rk - l0);
            by_range[{h->far_c0[b], h->far_c1[b]}].push_back({h->far_voff[b] + l0 * c, c, cols, F.toff[b] + l0, 1});
            by_range[{h->far_r0[b], h->far_r1[b]}].push_back({h->far_uoff[b] + l0 * m, m, cols, F.toff[b] + l0, 0});
        }
    }
    struct Task {
        int lo, hi;
        std::vector<std::array<int64_t, 5>> items;
    };
    std::vector<Task> tasks;
    for (auto &kv : by_range) {
        Task cur{kv.first.first, kv.first.second, {}};
        int R = 0;
        for (auto &it : kv.second) {
            if (R + it[2] > 64) {
                tasks.push_back(cur);
                cur.items.clear();
                R = 0;
            }
            cur.items.push_back(it);
            R += (int)it[2];
        }
        if (!cur.items.empty()) tasks.push_back(cur);
    }
    std::stable_sort(tasks.begin(), tasks.end(), [](const Task &x, const Task &y) {
        return (int64_t)(x.hi - x.lo) * (int64_t)x.items.size() > (int64_t)(y.hi - y.lo) * (int64_t)y.items.size();
    });
    F.p1_lo.clear(), F.p1_hi.clear(), F.p1_ld.clear(), F.p1_rank.clear(), F.p1_row.clear(), F.p1_isv.clear();
    F.p1_off.clear();
    F.p1_ptr.assign(1, 0);
    for (const Task &tk : tasks) {
        F.p1_lo.push_back(tk.lo);
        F.p1_hi.push_back(tk.hi);
        for (auto &it : tk.items) {
            F.p1_off.push_back(it[0]);
            F.p1_ld.push_back((int)it[1]);
            F.p1_rank.push_back((int)it[2]);
            F.p1_row.push_back((int)it[3]);
            F.p1_isv.push_back((int)it[4]);
        }
        F.p1_ptr.push_back((int)F.p1_off.size());
    }
    F.entries = 0;
    for (int b = 0; b < nf; ++b) {
        int64_t m = h->far_r1[b] - h->far_r0[b], c = h->far_c1[b] - h->far_c0[b];
        F.entries += h->far_rank[b] < 0 ? m * c : (int64_t)h->far_rank[b] * (m + c);
    }
}

}  // namespace hm

// ---- host-only planning entry points (no device work) -----------------------------------
extern "C" int hm_plan_order_method(int32_t method, int32_t n_leaves, int32_t n_pairs, const int32_t *t,
                                    const int32_t *s, int32_t *order)
{
    if (method < 0 || method > 2 || n_leaves <= 0 || n_pairs < 0 || !order || (n_pairs > 0 && (!t || !s)))
        return HM_EINVAL;
    for (int b = 0; b < n_pairs; ++b)
        if (t[b] < 0 || s[b] < 0 || t[b] >= n_leaves || s[b] >= n_leaves) return HM_EINVAL;
    std::vector<int> tv(t, t + n_pairs), sv(s, s + n_pairs), o;
    if (method == 1) o = hm::rcm_order(n_leaves, tv, sv);
    else if (method == 2) o = hm::sloan_order(n_leaves, tv, sv);
    else {
        o.resize(n_leaves);
        std::iota(o.begin(), o.end(), 0);
    }
    std::memcpy(order, o.data(), sizeof(int32_t) * n_leaves);
    return HM_OK;
}

extern "C" int hm_plan_order(int32_t n_leaves, int32_t n_pairs, const int32_t *t, const int32_t *s, int32_t *order)
{
    return hm_plan_order_method(1, n_leaves, n_pairs, t, s, order);
}

extern "C" int hm_plan_fill_closure(int32_t closure, int32_t n_blocks, int32_t n_pairs, const int32_t *i,
                                    const int32_t *j, int32_t *ptr, int32_t *idx, int64_t idx_cap)
{
    if ((closure != 0 && closure != 1) || n_blocks <= 0 || n_pairs < 0 || !ptr || (n_pairs > 0 && (!i || !j)))
        return HM_EINVAL;
    for (int b = 0; b < n_pairs; ++b)
        if (i[b] < 0 || j[b] < 0 || i[b] >= n_blocks || j[b] >= n_blocks) return HM_EINVAL;
    std::vector<int> iv(i, i + n_pairs), jv(j, j + n_pairs), sp, si;
    hm::symbolic_fill(n_blocks, iv, jv, sp, si, closure == 1);
    std::memcpy(ptr, sp.data(), sizeof(int32_t) * (n_blocks + 1));
    if (idx) {
        if ((int64_t)si.size() > idx_cap) return HM_EINVAL;
        std::memcpy(idx, si.data(), sizeof(int32_t) * si.size());
    }
    return HM_OK;
}

extern "C" int hm_plan_fill(int32_t n_blocks, int32_t n_pairs, const int32_t *i, const int32_t *j, int32_t *ptr,
                            int32_t *idx, int64_t idx_cap)
{
    return hm_plan_fill_closure(1, n_blocks, n_pairs, i, j, ptr, idx, idx_cap);
}

extern "C" int hm_plan_far(int32_t n, int32_t n_leaves, const int32_t *leaf_ptr, int32_t n_far, const int32_t *far_r0,
                           const int32_t *far_r1, const int32_t *far_c0, const int32_t *far_c1,
                           const int32_t *far_rank, const int64_t *far_uoff, const int64_t *far_voff, int32_t what,
                           int64_t *out, int64_t *count)
{
    if (n <= 0 || n_leaves <= 0 || !leaf_ptr || n_far < 0 || !count || what < 0 || what > 4) return HM_EINVAL;
    if (n_far > 0 && (!far_r0 || !far_r1 || !far_c0 || !far_c1 || !far_rank || !far_uoff || !far_voff))
        return HM_EINVAL;
    if (leaf_ptr[0] != 0 || leaf_ptr[n_leaves] != n) return HM_EINVAL;
    std::vector<char> is_bound(n + 1, 0);
    for (int l = 0; l < n_leaves; ++l) {
        const int sz = leaf_ptr[l + 1] - leaf_ptr[l];
        if (sz < 1 || sz > 64) return HM_EINVAL;
        is_bound[leaf_ptr[l]] = 1;
    }
    is_bound[n] = 1;
    for (int b = 0; b < n_far; ++b) {
        const int r0 = far_r0[b], r1 = far_r1[b], c0 = far_c0[b], c1 = far_c1[b], r = far_rank[b];
        if (r0 < 0 || r0 >= r1 || r1 > c0 || c0 >= c1 || c1 > n) return HM_EINVAL;
        if (!is_bound[r0] || !is_bound[r1] || !is_bound[c0] || !is_bound[c1]) return HM_EINVAL;
        if (r < -1 || r > std::min(r1 - r0, c1 - c0) || far_uoff[b] < 0 || far_voff[b] < 0) return HM_EINVAL;
    }
    hm_ctx h;   // host fields only: the planner does no device work
    h.n = n;
    h.nl = n_leaves;
    h.leaf_ptr.assign(leaf_ptr, leaf_ptr + n_leaves + 1);
    h.far_r0.assign(far_r0, far_r0 + n_far);
    h.far_r1.assign(far_r1, far_r1 + n_far);
    h.far_c0.assign(far_c0, far_c0 + n_far);
    h.far_c1.assign(far_c1, far_c1 + n_far);
    h.far_rank.assign(far_rank, far_rank + n_far);
    h.far_uoff.assign(far_uoff, far_uoff + n_far);
    h.far_voff.assign(far_voff, far_voff + n_far);
    hm::plan_far(&h);
    const hm::FarPlan &F = h.fplan;
    std::vector<int64_t> v;
    if (what == 0) v.assign(F.seg_ptr.begin(), F.seg_ptr.end());
    if (what == 1)
        for (const hm::FarSegD &g : F.segs) v.insert(v.end(), {g.foff, g.yrow, g.fi, g.fk, g.len, g.src});
    if (what == 2) v.assign(F.part_ptr.begin(), F.part_ptr.end());
    if (what == 3)
        for (size_t t = 0; t < F.p1_lo.size(); ++t) v.insert(v.end(), {F.p1_lo[t], F.p1_hi[t], F.p1_ptr[t], F.p1_ptr[t + 1]});
    if (what == 4)
        for (size_t e = 0; e < F.p1_off.size(); ++e)
            v.insert(v.end(), {F.p1_off[e], F.p1_ld[e], F.p1_rank[e], F.p1_row[e], F.p1_isv[e]});
    const int64_t cap = *count;
    *count = (int64_t)v.size();
    if (out) {
        if ((int64_t)v.size() > cap) return HM_EINVAL;
        std::memcpy(out, v.data(), sizeof(int64_t) * v.size());
    }
    return HM_OK;
}
