// Operator of the preconditioned system (Eq. 28) on the GPU, in complex FP64 or FP32:
//
//   A x~ = D^{-1} [ D x~ + L^{-1} Z_F L^{-T} x~ ],   c = D^{-1} L^{-1} b,   x = L^{-T} x~
//
// L^{-1} / L^{-T} are the products of the left / right scaling coefficients (Eqs. 20, 23,
// 24) applied as block-triangular sweeps over the coefficient panels W_k (L_jk = W_kj^T).
// Each sweep is one sync-free launch: a CTA takes the next block row from a ticket counter
// (so every block it waits on belongs to a CTA that is already running), stages the
// coefficient blocks of its dependencies in fixed chunks, waits on their ready flags (a
// bounded wait that reports HM_ETIMEOUT instead of hanging), and publishes its own block
// with a flag.  The most recently finished dependency is always alone in the last chunk,
// so the chain's critical path carries one small block product per step.  Chunking does not
// change the order of the arithmetic: every output subtracts its terms block by block in
// dependency order, so results are bitwise reproducible and independent of the batch width.
//
// Z_F is applied by far_product (far.cu) in cluster order.
// Vectors are column-major n x nrhs (ld n) in solve order.
#include <cmath>
#include <cstdio>
#include <vector>

#include "cluster.cuh"
#include "cplx.cuh"
#include "hm_internal.h"
#include "tc.cuh"
#include "tile.cuh"

namespace hm {

namespace {

// The handle's error word block: err[ERR_CODE] is set by a failing wait, err[ERR_HOLD] names a
// block row the sweeps leave out (a test hook: -1 = none; every wait on that row then runs
// out), err[ERR_BOUND..+1] holds the bound on any single wait in ns (2 s unless a test sets it).
__device__ __forceinline__ unsigned long long wait_bound(const int *err)
{
    return __ldcg((const unsigned long long *)(err + ERR_BOUND));
}
__device__ __forceinline__ bool held_back(const int *err, int blk) { return __ldcg(err + ERR_HOLD) == blk; }

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One thread waits until flags[k] == epoch; false (and ERR_TIMEOUT recorded) when the
// bound expires or another CTA already failed.
__device__ bool wait_ready(const int *flags, int k, int epoch, int *err)
{
    const volatile int *f = flags + k;
    if (*f == epoch) {
        __threadfence();
        return true;
    }
    const unsigned long long t0 = gtimer(), bound = wait_bound(err);
    while (*f != epoch) {
        if (*(volatile int *)err) return false;
        if (gtimer() - t0 > bound) {
            atomicCAS(err, 0, ERR_TIMEOUT);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();
    return true;
}


// Dependencies finishing last (the final TAIL entries of a list) are taken one per chunk,
// so that the chain's critical path never carries more than one block product.
constexpr int TAIL = 4;

// Next chunk [p, q) of a dependency list walked from p towards pend (step +1 or -1): blocks
// are added while their staged entries fit the budget; each of the last TAIL dependencies
// forms a chunk of its own.
// Low-rank blocks (see lowrank_t) also count their r * nrhs outputs, at most LR_OUT per chunk.
constexpr int LR_REG = 16;                 // outputs of lowrank_t per thread
constexpr int LR_OUT = LR_REG * 256;       // per chunk (256 threads)

__device__ __forceinline__ int dep_rank(const int *crk, const int *ent, int b)
{
    return crk ? crk[ent ? ent[b] : b] : -1;
}

template <int TR, int TC>
__device__ __forceinline__ int next_chunk(int p, int pend, int step, const int *dep, const int *size, int no,
                                          int nrhs, int budget, const int *crk, const int *ent)
{
    const int tail0 = pend - TAIL * step;   // first position of the tail
    if ((step > 0 && p >= tail0) || (step < 0 && p <= tail0)) return p + step;
    int q = p, used = 0, cnt = 0, lr = 0;
    while (q != tail0 && cnt < 16) {
        const int need = stage_need(no, size[dep[q]], nrhs, TR, TC), r = dep_rank(crk, ent, q);
        const int lo = r > 0 ? r * nrhs : 0;
        if (cnt > 0 && (used + need > budget || lr + lo > LR_OUT)) break;
        used += need;
        lr += lo;
        ++cnt;
        q += step;
    }
    return q;
}

template <class T> __device__ __forceinline__ void cp_async_el(T *dst, const T *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

// Complex-FP32 sweeps: a chunk's contraction length is at most 64, so its coefficient blocks
// fit one of two buffers of SW_WCAP entries (64 x stage_ldw(64)) and its vector blocks a
// 64 x stage_ldr(nrhs) area; the shared memory of a row is 2 SW_WCAP + 64 stage_ldr entries.
constexpr int SW_WCAP = 64 * 65;

__device__ __forceinline__ int next_chunk_ll(int p, int pend, int step, const int *dep, const int *size)
{
    const int tail0 = pend - TAIL * step;
    if ((step > 0 && p >= tail0) || (step < 0 && p <= tail0)) return p + step;
    int q = p, used = 0;
    while (q != tail0) {
        const int nc = size[dep[q]];
        if (used > 0 && used + nc > 64) break;
        used += nc;
        q += step;
    }
    return q;
}

// One block row of a sweep (Eqs. 23, 24): out = x_o - sum over the dependency list of
// M_b y_b, with M_b = W_ko^T (forward, W_ko at Wsrc, nc x no column-major) or W_oj
// (backward, no x nc column-major).  FP64: the CTA stages each chunk's coefficient blocks
// before waiting on the chunk's ready flags, then the vector blocks, then runs the tile
// products.  Complex FP32: the coefficient blocks of the next chunk are copied with cp.async
// while the current chunk waits and multiplies, and the vector blocks come from the tagged
// copy.  Tagged publication (complex FP32): next to y, every entry is also written as two
// 8-byte words (value half, launch epoch) -- each naturally aligned 8-byte store is observed
// whole -- so a consumer validates the data it reads instead of waiting on a flag behind a
// fence.
__device__ __forceinline__ uint4 ld_tag(const uint4 *p)
{
    uint4 v;
    asm volatile("ld.volatile.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Staging copy from the tagged array: SB words per thread are loaded together; while any of
// them still carries another epoch, those are loaded again together (one round trip per
// retry, bounded by the handle's wait bound, given up once *err is set).
template <int SB = 8, class Addr, class St>
__device__ __forceinline__ void stage_tagged(int count, unsigned epoch, int *err, Addr &&addr, St &&st)
{
    for (int e0 = threadIdx.x; e0 < count; e0 += SB * blockDim.x) {
        uint4 v[SB];
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < count) v[u] = ld_tag(addr(e));
        }
        bool timing = false;
        unsigned long long t0 = 0;
        for (;;) {
            unsigned stale = 0;
#pragma unroll
            for (int u = 0; u < SB; ++u) {
                const int e = e0 + u * blockDim.x;
                if (e < count && (v[u].y != epoch || v[u].w != epoch)) stale |= 1u << u;
            }
            if (!stale || *(volatile int *)err) break;   // all current, or a wait already expired
            if (!timing) {
                timing = true;
                t0 = gtimer();
            } else if (gtimer() - t0 > wait_bound(err)) {
                atomicCAS(err, 0, ERR_TIMEOUT);
                break;
            }
            __nanosleep(32);
#pragma unroll
            for (int u = 0; u < SB; ++u)
                if (stale & (1u << u)) v[u] = ld_tag(addr(e0 + u * blockDim.x));
        }
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < count) st(e, make_float2(__uint_as_float(v[u].x), __uint_as_float(v[u].z)));
        }
    }
}

// ---- cluster-chained complex-FP32 sweeps (schedule kinds 5 and 6) -------------------------
// The C CTAs of a thread-block cluster take C consecutive tickets, i.e. consecutive block rows
// of the sweep order (C / G rows of each of the G column groups).  A finished row stays in its
// CTA's shared memory (the result buffer of sweep_row) beside a ready word holding the launch
// epoch; a later row of the same cluster and group reads that dependency through distributed
// shared memory instead of waiting for its tagged words to reach L2.  Every CTA of the cluster
// waits at a cluster barrier before it exits, so those buffers stay readable.  The sums and
// their order are those of kind 1: the values read are the same FP32 numbers.
struct CLink {
    int t0, G, g, nb;   // the cluster's first ticket; groups, this CTA's group; blocks
    unsigned buf;       // shared-window address of the result buffer (same in every CTA)
    unsigned flag;      // shared-window address of the ready word
};

// Ys[e] <- entry e of the finished block of cluster CTA `rank` (count entries, its result
// buffer's layout), once its ready word carries this launch's epoch; a thread with no entry
// does not wait.  The wait is bounded like every other (ERR_TIMEOUT), and ends early once
// another wait has expired.
__device__ void cluster_stage(int count, unsigned epoch, int *err, unsigned rank, const CLink &lk, float2 *Ys)
{
    if ((int)threadIdx.x >= count) return;
    const unsigned fl = cluster_map(lk.flag, rank), bs = cluster_map(lk.buf, rank);
    if (ld_cluster_u32(fl) != epoch) {
        const unsigned long long t0 = gtimer();
        for (;;) {
            if (*(volatile int *)err) return;
            __nanosleep(20);
            if (ld_cluster_u32(fl) == epoch) break;
            if (gtimer() - t0 > wait_bound(err)) {
                atomicCAS(err, 0, ERR_TIMEOUT);
                return;
            }
        }
    }
    fence_cluster();   // acquire: the entries were written before the ready word (release)
    for (int e = threadIdx.x; e < count; e += blockDim.x) Ys[e] = ld_cluster_f2(bs + 8u * (unsigned)e);
}

// A compressed fill-in coefficient block (Sec. 3.4) is stored as P (n_k x r), Q (n_j x r),
// W_kj ~ P Q^T, and applied as two products: with G the factor on the dependency's side and H
// the one on the row's side (forward, block W_ko: G = P, H = Q; backward, W_oj: G = Q, H = P),
// t = G^T y_dep (r x nrhs), then out -= H t.  Staging: H in the block's coefficient slot as an
// r-long contraction (Ws[l * ldw + row]), G behind it (Ws[r * ldw + q + l * nc]), y_dep as for
// a dense block; r (ldw + nc) <= nc ldw holds for every compressed block, so it fits the slot.
// lowrank_t computes every t of a chunk into registers, then (after a barrier) writes each over
// its block's vector slot (t[l + c * r]), so the chunk's products run as for dense blocks.
// SPLIT (complex-FP32 sweeps): coefficient blocks packed in wbase (nc * ldw entries each),
// vector blocks in ybase (nc * nrhs each); otherwise (FP64) block after block in wbase, each
// its coefficients then its vector block (nc * ldw + nc * ldr entries).
template <class T, bool SPLIT>
__device__ void lowrank_t(int p, int q, int step, const int *lidx, const int *size, const int *crk, const int *ent,
                          T *wbase, T *ybase, int ldw, int ldr, int nrhs)
{
    T treg[LR_REG];
    int u = 0, ng = threadIdx.x, base = 0, ow = 0, oy = 0;
    for (int b = p; b != q; b += step) {
        const int nc = size[lidx[b]], r = dep_rank(crk, ent, b);
        if (r >= 0) {
            const T *G = wbase + ow + r * ldw, *Y = SPLIT ? ybase + oy : wbase + ow + nc * ldw;
            const int len = r * nrhs;
            for (; ng < base + len && u < LR_REG; ng += blockDim.x) {
                const int o = ng - base, l = o % r, c = o / r;
                T acc = czero(T());
                for (int qq = 0; qq < nc; ++qq) acc = cfma(G[qq + l * nc], Y[qq + c * nc], acc);
                treg[u++] = acc;
            }
            base += len;
        }
        ow += SPLIT ? nc * ldw : nc * (ldw + ldr);
        oy += nc * nrhs;
    }
    __syncthreads();   // every t read its vector block
    u = 0;
    ng = threadIdx.x;
    base = 0;
    ow = 0;
    oy = 0;
    for (int b = p; b != q; b += step) {
        const int nc = size[lidx[b]], r = dep_rank(crk, ent, b);
        if (r >= 0) {
            T *Y = SPLIT ? ybase + oy : wbase + ow + nc * ldw;
            const int len = r * nrhs;
            for (; ng < base + len && u < LR_REG; ng += blockDim.x) Y[ng - base] = treg[u++];
            base += len;
        }
        ow += SPLIT ? nc * ldw : nc * (ldw + ldr);
        oy += nc * nrhs;
    }
    __syncthreads();
}

// Where dependency b's coefficient block is staged from, and how: copy(dst, src) is the element
// copy (cp.async or a load and a store) of entry src into the staged entry dst.  Dense: the
// block M (rows of o, contraction over the dependency's rows) as Ws[qq * ldw + row]; low rank
// (lowrank_t): H as Ws[l * ldw + row] and G behind it.
template <class T, bool FWD, class Copy>
__device__ __forceinline__ void stage_block(int b, int no, int nc, const int *lent, const int64_t *cbo,
                                            const int *crk, const T *W, T *Ws, int ldw, Copy &&copy)
{
    const int e = lent ? lent[b] : b, r = crk[e];
    const T *base = W + cbo[e];
    if (r < 0) {
        if (FWD)   // W_ko: nc x no; M(row, qq) = W_ko(qq, row)
            for (int x = threadIdx.x; x < nc * no; x += blockDim.x) copy(Ws + (x % nc) * ldw + x / nc, base + x);
        else       // W_oj: no x nc; M(row, qq) = W_oj(row, qq)
            for (int x = threadIdx.x; x < nc * no; x += blockDim.x) copy(Ws + (x / no) * ldw + x % no, base + x);
        return;
    }
    // W_kj ~ P Q^T with P (n_k x r) then Q (n_j x r): forward (k = dep, j = o) G = P, H = Q;
    // backward (k = o, j = dep) H = P, G = Q
    const T *H = FWD ? base + (int64_t)nc * r : base, *G = FWD ? base : base + (int64_t)no * r;
    for (int x = threadIdx.x; x < no * r; x += blockDim.x) copy(Ws + (x / no) * ldw + x % no, H + x);
    for (int x = threadIdx.x; x < nc * r; x += blockDim.x) copy(Ws + r * ldw + x, G + x);
}

template <class T, int TR, int TC, int NT, bool FWD, bool LL = false, bool CLU = false>
__device__ __forceinline__ void sweep_row(int o_blk, int no, const int *size, const int *boff, const int *lptr,
                                          const int *lidx, const int *lent, const int64_t *cbo, const int *crk,
                                          const T *W, const T *x, T *y, int n, int nrhs, int budget, int *flags,
                                          int epoch, int *err, T *buf, int cut = 0, int *pub = nullptr,
                                          uint4 *tag = nullptr, CLink lk = CLink{})
{
    // CLU (with LL): dependencies finished by an earlier CTA of the same cluster are read from
    // its shared memory (cluster_stage), and the result's ready word is raised for the later ones
    // LL (complex FP32 only): dependencies are read from, and the result published to, the
    // tagged copy `tag` (same layout as y); no flags, no fence
    // cut > 0: leave the last `cut` dependencies of the walk out (they are added by the
    // chain CTA of a chain-and-helpers sweep) and publish the partial sum on `pub`
    // Dependency b of the walk is S-list entry lent[b] (forward) or b itself (backward), its
    // coefficients at W + cbo[e], dense or of rank crk[e] (stage_block, lowrank_t).
    if (!pub) pub = flags;
    const int o = boff[o_blk];
    const int nrt = (no + TR - 1) / TR, ntiles = nrt * ((nrhs + TC - 1) / TC);
    const int ldw = stage_ldw(no, TR);
    Tile<T, TR, TC, NT> acc;
    tile_load(acc, x + o, 1, n, no, nrhs, nrt, ntiles);
    // forward: list ascending over [lptr[o], lptr[o+1]); backward: descending
    const int step = FWD ? 1 : -1;
    const int pa = FWD ? lptr[o_blk] : lptr[o_blk + 1] - 1,
              pend = (FWD ? lptr[o_blk + 1] : lptr[o_blk] - 1) - cut * step;
    // contraction length of dependency b's product: its rows, or its rank when compressed
    auto kdim = [&](int b, int nc) {
        const int r = dep_rank(crk, lent, b);
        return r < 0 ? nc : r;
    };
    if constexpr (LL) {
        // the coefficient blocks of the next chunk are copied (cp.async, no registers held)
        // into the other buffer while the current chunk waits for its vector blocks and
        // multiplies, so the copies of static data stay off the wait-to-publish path
        T *const ys = buf + 2 * SW_WCAP;
        auto wbuf = [&](int w) { return buf + w * SW_WCAP; };
        auto stage_w = [&](int p, int q, T *dst) {
            int off = 0;
            for (int b = p; b != q; b += step) {
                const int nc = size[lidx[b]];
                stage_block<T, FWD>(b, no, nc, lent, cbo, crk, W, dst + off, ldw,
                                    [](T *d, const T *src) { cp_async_el(d, src); });
                off += nc * ldw;
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        };
        if (pa != pend) {
            int p = pa, q = next_chunk_ll(pa, pend, step, lidx, size);
            stage_w(p, q, wbuf(0));
            for (int cur = 0; p != pend; cur ^= 1) {
                int q2 = q;
                if (q != pend) {
                    q2 = next_chunk_ll(q, pend, step, lidx, size);
                    stage_w(q, q2, wbuf(cur ^ 1));
                }
                int yoff = 0;
                bool lr = false;
                for (int b = p; b != q; b += step) {
                    const int k = lidx[b], nc = size[k], ok = boff[k];
                    T *Ys = ys + yoff;
                    lr = lr || dep_rank(crk, lent, b) >= 0;
                    bool local = false;
                    if constexpr (CLU) {
                        const int tk = (FWD ? k : lk.nb - 1 - k) * lk.G + lk.g;   // the producer's ticket
                        if (tk >= lk.t0) {
                            cluster_stage((int)(nc * nrhs), (unsigned)epoch, err, (unsigned)(tk - lk.t0), lk, Ys);
                            local = true;
                        }
                    }
                    if (!local)
                        stage_tagged((int)(nc * nrhs), (unsigned)epoch, err,
                                     [&](int e) { return tag + ok + e % nc + (int64_t)(e / nc) * n; },
                                     [&](int e, float2 v) { Ys[e] = v; });
                    yoff += nc * nrhs;
                }
                if (q != pend) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
                else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                __syncthreads();
                T *wc = wbuf(cur);
                if (lr) lowrank_t<T, true>(p, q, step, lidx, size, crk, lent, wc, ys, ldw, 0, nrhs);
                int woff = 0;
                yoff = 0;
                for (int b = p; b != q; b += step) {
                    const int nc = size[lidx[b]], kd = kdim(b, nc);
                    tile_mac<true>(acc, wc + woff, ldw, ys + yoff, 1, kd, kd, nrt, ntiles);
                    woff += nc * ldw;
                    yoff += nc * nrhs;
                }
                __syncthreads();
                p = q;
                q = q2;
            }
        }
    }
    for (int p = pa; !LL && p != pend;) {
        const int q = next_chunk<TR, TC>(p, pend, step, lidx, size, no, nrhs, budget, crk, lent);
        const int ldr = stage_ldr(nrhs, TC);
        // stage the coefficient blocks (static data) before waiting
        int off = 0;
        bool lr = false;
        for (int b = p; b != q; b += step) {
            const int nc = size[lidx[b]];
            lr = lr || dep_rank(crk, lent, b) >= 0;
            stage_block<T, FWD>(b, no, nc, lent, cbo, crk, W, buf + off, ldw, [](T *d, const T *src) { *d = *src; });
            off += stage_need(no, nc, nrhs, TR, TC);
        }
        if (threadIdx.x == 0)
            for (int b = p; b != q; b += step) wait_ready(flags, lidx[b], epoch, err);
        __syncthreads();
        off = 0;
        for (int b = p; b != q; b += step) {
            const int k = lidx[b], nc = size[k], ok = boff[k];
            T *Ys = buf + off + nc * ldw;
            stage_copy(nc * nrhs, [&](int e) { return ldcg(y + ok + e % nc + (int64_t)(e / nc) * n); },
                       [&](int e, T v) { Ys[e] = v; });
            off += stage_need(no, nc, nrhs, TR, TC);
        }
        __syncthreads();
        if (lr) lowrank_t<T, false>(p, q, step, lidx, size, crk, lent, buf, buf, ldw, ldr, nrhs);
        off = 0;
        for (int b = p; b != q; b += step) {
            const int nc = size[lidx[b]], kd = kdim(b, nc);
            tile_mac<true>(acc, buf + off, ldw, buf + off + nc * ldw, 1, kd, kd, nrt, ntiles);
            off += stage_need(no, nc, nrhs, TR, TC);
        }
        __syncthreads();
        p = q;
    }
    if constexpr (LL) {
        // the block goes through shared memory (free after the last product) so that the
        // tagged words, which the consumers wait on, leave first and coalesced (a warp writes
        // 32 consecutive rows of a column); y follows
        tile_store(acc, buf, 1, no, no, nrhs, nrt, ntiles);   // buf[r * no + row]
        __syncthreads();
        if constexpr (CLU) {
            if (threadIdx.x == 0) {   // release: the barrier orders every thread's entries first
                fence_cluster();
                st_cluster_u32(lk.flag, (unsigned)epoch);
            }
        }
        for (int e = threadIdx.x; e < no * nrhs; e += blockDim.x) {
            const float2 v = buf[e];
            tag[o + e % no + (int64_t)(e / no) * n] =
                make_uint4(__float_as_uint(v.x), (unsigned)epoch, __float_as_uint(v.y), (unsigned)epoch);
        }
        for (int e = threadIdx.x; e < no * nrhs; e += blockDim.x) y[o + e % no + (int64_t)(e / no) * n] = buf[e];
        return;
    }
    tile_store(acc, y + o, 1, n, no, nrhs, nrt, ntiles);
    // publish: the barrier orders every thread's stores before thread 0's fence and flag
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        *(volatile int *)(pub + o_blk) = epoch;
    }
}

// ---- complex-FP32 sweeps on the tensor cores ----------------------------------------------
// One CTA per block row o and column group, as sweep_row, with the block products on the
// tensor-core micro-kernel of tc.cuh.  The row's dependency list is walked in chunks of at most
// tc::KC contraction entries: whole dependency blocks are packed while they fit, a block longer
// than a chunk is split, and each of the last TAIL dependencies (the ones the chain publishes
// last) starts a chunk of its own.  Per chunk: the coefficient rows of the next chunk are copied
// with cp.async into the other raw buffer; the chunk's vector entries are read from the tagged
// copy into registers (each word re-polled until it carries this sweep's epoch); then, once the
// previous chunk's MMAs have finished, the raw coefficients are split into the A' planes, the
// vector entries into the B' planes, and thread 0 issues the chunk's MMAs.  At the end
// out = x - D and the block is published as tagged words, then as plain values.  Every output
// adds its terms in walk order whatever the number of columns, so the result of a column does
// not depend on the others.
constexpr int TCW_LD = 64;                       // raw coefficient buffer: raw[kk * TCW_LD + row]
constexpr int TCW_BYTES = tc::KC * TCW_LD * 8;   // one raw buffer (16 KB)

struct TcChunk {                 // a chunk's per-entry sources, filled by thread 0
    int64_t wbase[tc::KC];       // coefficient of contraction entry kk, row r: W[wbase + r * wstr]
    int wstr[tc::KC];
    int yrow[tc::KC];            // vector entry kk of column c: tag[yrow + c * n]
    int kl;                      // entries in the chunk (0: none left)
};

struct TcWalk {
    int p, koff;   // next dependency position and the first row of it not yet taken
};

// Thread 0: the next chunk of o's dependency list (see the comment above).
template <bool FWD>
__device__ void tc_next_chunk(TcWalk &w, int pend, int o_blk, int no, const int *size, const int *boff,
                              const int *lidx, const int *lcol, const int64_t *coff, TcChunk &c)
{
    const int step = FWD ? 1 : -1, tail0 = pend - TAIL * step;
    int kl = 0;
    while (w.p != pend && kl < tc::KC) {
        const int k = lidx[w.p], nk = size[k];
        const bool tail = FWD ? w.p >= tail0 : w.p <= tail0;
        if (tail && kl > 0) break;                                       // tail blocks start a chunk
        const int take = min(nk - w.koff, tc::KC - kl);
        if (!tail && w.koff == 0 && take < nk && kl > 0) break;           // pack whole blocks only
        for (int i = 0; i < take; ++i) {
            const int q = w.koff + i;
            if (FWD) {   // M(row, q) = W_ko(q, row), W_ko: nk x no at coff[k] + lcol * nk
                c.wbase[kl + i] = coff[k] + (int64_t)lcol[w.p] * nk + q;
                c.wstr[kl + i] = nk;
            } else {     // M(row, q) = W_ok(row, q), W_ok: no x nk at coff[o] + lcol * no
                c.wbase[kl + i] = coff[o_blk] + (int64_t)lcol[w.p] * no + (int64_t)q * no;
                c.wstr[kl + i] = 1;
            }
            c.yrow[kl + i] = boff[k] + q;
        }
        kl += take;
        w.koff += take;
        if (w.koff == nk) {
            w.p += step;
            w.koff = 0;
        }
        if (tail) break;                                                  // ... and end it
    }
    c.kl = kl;
}

template <bool FWD>
__global__ void __launch_bounds__(256, 2) k_sweep_tc(int nb, const int *size, const int *boff, const int *lptr,
                                                  const int *lidx, const int *lcol, const int64_t *coff,
                                                  const float2 *W, const float2 *x, float2 *y, int n, int nrhs,
                                                  int G, int gw, int epoch, int *ticket, int *err, uint4 *tag)
{
    extern __shared__ unsigned char smraw[];
    __shared__ int s_t;
    __shared__ uint64_t s_mbar;
    __shared__ uint32_t s_tmem;
    __shared__ TcChunk s_ch[2];
    if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int bi = s_t / G, g = s_t % G;
    if (bi >= nb) return;
    const int o_blk = FWD ? bi : nb - 1 - bi;
    const int c0 = g * gw, nc = min(gw, nrhs - c0);
    if (nc <= 0 || held_back(err, o_blk)) return;
    x += (int64_t)c0 * n;
    y += (int64_t)c0 * n;
    tag += (int64_t)c0 * n;
    const int no = size[o_blk], o = boff[o_blk];
    const unsigned long long bound = wait_bound(err);
    unsigned char *region = tc::align1024(smraw);
    float2 *raw[2] = {(float2 *)(region + tc::REGION_BYTES), (float2 *)(region + tc::REGION_BYTES + TCW_BYTES)};
    // the thread's outputs e = tid + u * blockDim (row e % no, column e / no): x first, so its
    // load stays off the critical path
    constexpr int NE = 64 * 64 / 256;
    float2 xr[NE];
#pragma unroll
    for (int u = 0; u < NE; ++u) {
        const int e = threadIdx.x + u * blockDim.x;
        xr[u] = e < no * nc ? x[o + e % no + (int64_t)(e / no) * n] : make_float2(0.f, 0.f);
    }
    const int pa = FWD ? lptr[o_blk] : lptr[o_blk + 1] - 1, pend = FWD ? lptr[o_blk + 1] : lptr[o_blk] - 1;
    tc::Acc acc;
    acc.planes = region;
    acc.mbar = &s_mbar;
    acc.tslot = &s_tmem;
    const bool deps = pa != pend;
    if (deps) {
        TcWalk w{pa, 0};
        auto prefetch = [&](int buf) {   // raw coefficients of chunk s_ch[buf]
            const TcChunk &c = s_ch[buf];
            const int kl = c.kl;
            for (int e = threadIdx.x; e < kl * no; e += blockDim.x) {
                int kk, r;
                if (FWD) kk = e % kl, r = e / kl;
                else kk = e / no, r = e % no;
                cp_async_el(raw[buf] + kk * TCW_LD + r, W + c.wbase[kk] + (int64_t)r * c.wstr[kk]);
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        };
        if (threadIdx.x == 0) tc_next_chunk<FWD>(w, pend, o_blk, no, size, boff, lidx, lcol, coff, s_ch[0]);
        acc.open(no, nc);   // synchronises: s_ch[0] is visible
        prefetch(0);
        for (int cur = 0; s_ch[cur].kl > 0; cur ^= 1) {
            const TcChunk &c = s_ch[cur];
            const int kl = c.kl;
            // the next chunk: its sources (thread 0) and, after the barrier below, its copies
            if (threadIdx.x == 0) tc_next_chunk<FWD>(w, pend, o_blk, no, size, boff, lidx, lcol, coff, s_ch[cur ^ 1]);
            // this chunk's vector entries into registers, re-polled until current
            uint4 v[8];
            const int cnt = kl * nc;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = threadIdx.x + u * blockDim.x;
                if (e < cnt) v[u] = ld_tag(tag + c.yrow[e % kl] + (int64_t)(e / kl) * n);
            }
            {
                bool timing = false;
                unsigned long long t0 = 0;
                for (;;) {
                    unsigned stale = 0;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int e = threadIdx.x + u * blockDim.x;
                        if (e < cnt && (v[u].y != (unsigned)epoch || v[u].w != (unsigned)epoch)) stale |= 1u << u;
                    }
                    if (!stale || *(volatile int *)err) break;
                    if (!timing) {
                        timing = true;
                        t0 = gtimer();
                    } else if (gtimer() - t0 > bound) {
                        atomicCAS(err, 0, ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(32);
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (stale & (1u << u)) {
                            const int e = threadIdx.x + u * blockDim.x;
                            v[u] = ld_tag(tag + c.yrow[e % kl] + (int64_t)(e / kl) * n);
                        }
                }
            }
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            __syncthreads();                   // raw[cur] landed for every thread; s_ch[cur ^ 1] written
            if (s_ch[cur ^ 1].kl > 0) prefetch(cur ^ 1);
            acc.wait(err, bound);              // the previous chunk's MMAs no longer read the planes
            const float2 *rw = raw[cur];
            for (int e = threadIdx.x; e < acc.m8 * kl; e += blockDim.x) {
                const int r = e % acc.m8, kk = e / acc.m8;
                acc.put_a(r, kk, r < no ? rw[kk * TCW_LD + r] : make_float2(0.f, 0.f));
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = threadIdx.x + u * blockDim.x;
                if (e < cnt) acc.put_b(e / kl, e % kl, make_float2(__uint_as_float(v[u].x), __uint_as_float(v[u].z)));
            }
            acc.zero_pad(kl);
            acc.issue(kl);                     // barrier inside: this chunk's raw buffer is consumed
        }
        acc.wait(err, bound);
    }
    float *dsm = (float *)region;
    const bool any = deps && acc.drain(dsm);
    float2 *out = xr;   // out = x - D, in place
#pragma unroll
    for (int u = 0; u < NE; ++u) {
        const int e = threadIdx.x + u * blockDim.x;
        if (any && e < no * nc) {
            const float2 d = acc.entry(dsm, e % no, e / no);
            out[u].x -= d.x;
            out[u].y -= d.y;
        }
    }
    // tagged words first (the consumers wait on them), then the plain copy
#pragma unroll
    for (int u = 0; u < NE; ++u) {
        const int e = threadIdx.x + u * blockDim.x;
        if (e < no * nc)
            tag[o + e % no + (int64_t)(e / no) * n] =
                make_uint4(__float_as_uint(out[u].x), (unsigned)epoch, __float_as_uint(out[u].y), (unsigned)epoch);
    }
#pragma unroll
    for (int u = 0; u < NE; ++u) {
        const int e = threadIdx.x + u * blockDim.x;
        if (e < no * nc) y[o + e % no + (int64_t)(e / no) * n] = out[u];
    }
    if (deps) acc.close();
}

}  // namespace

// The columns are split into G groups of gw (the last may be narrower), each an independent
// chain with its own ready flags; ticket t takes block t / G (in sweep order) of group t % G.

// y = L^{-1} x : y_i = x_i - sum_{k < i, i in S_k} W_ki^T y_k   (Eq. 23)
template <class T, int TR, int TC, int NT>
__global__ void __launch_bounds__(256) k_sweep_fwd(int nb, const int *size, const int *boff, const int *rptr,
                                                   const int *ridx, const int *rent, const int64_t *cbo,
                                                   const int *crk, const T *W, const T *x, T *y, int n, int nrhs, int G, int gw,
                                                   int budget, int *flags, int epoch, int *ticket, int *err,
                                                   uint4 *tag)
{
    extern __shared__ unsigned char smraw[];
    __shared__ int s_t;
    if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int i = s_t / G, g = s_t % G;
    if (i >= nb || held_back(err, i)) return;
    const int c0 = g * gw, nc = max(0, min(gw, nrhs - c0));
    sweep_row<T, TR, TC, NT, true, sizeof(T) == 8>(i, size[i], size, boff, rptr, ridx, rent, cbo, crk, W,
                                                   x + (int64_t)c0 * n, y + (int64_t)c0 * n, n, nc, budget,
                                                   flags + g * nb, epoch, err, (T *)smraw, 0, nullptr,
                                                   tag + (int64_t)c0 * n);
}

// y = L^{-T} x : y_k = x_k - sum_{j in S_k} W_kj y_j   (Eq. 24); j walked downwards
template <class T, int TR, int TC, int NT>
__global__ void __launch_bounds__(256) k_sweep_bwd(int nb, const int *size, const int *boff, const int *sptr,
                                                   const int *sidx, const int64_t *cbo, const int *crk,
                                                   const T *W, const T *x, T *y, int n, int nrhs, int G, int gw,
                                                   int budget, int *flags, int epoch, int *ticket, int *err,
                                                   uint4 *tag)
{
    extern __shared__ unsigned char smraw[];
    __shared__ int s_t;
    if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int k = nb - 1 - s_t / G, g = s_t % G;
    if (k < 0 || held_back(err, k)) return;
    const int c0 = g * gw, nc = max(0, min(gw, nrhs - c0));
    sweep_row<T, TR, TC, NT, false, sizeof(T) == 8>(k, size[k], size, boff, sptr, sidx, nullptr, cbo, crk, W,
                                                    x + (int64_t)c0 * n, y + (int64_t)c0 * n, n, nc, budget,
                                                    flags + g * nb, epoch, err, (T *)smraw, 0, nullptr,
                                                    tag + (int64_t)c0 * n);
}

// Cluster-chained complex-FP32 sweeps (kinds 5, 6; see CLink): the cluster's first CTA takes
// C tickets at once, every CTA of the cluster takes its own from them, and all wait at a
// cluster barrier before exiting.  FWD as k_sweep_fwd (lptr/lidx/lent = rptr/ridx/rent), else
// as k_sweep_bwd (sptr/sidx).
template <int TR, int TC, int NT, bool FWD>
__global__ void __launch_bounds__(256) k_sweep_cl(int nb, const int *size, const int *boff, const int *lptr,
                                                  const int *lidx, const int *lent, const int64_t *cbo,
                                                  const int *crk, const float2 *W, const float2 *x, float2 *y, int n,
                                                  int nrhs, int G, int gw, int budget, int *flags, int epoch,
                                                  int *ticket, int *err, uint4 *tag)
{
    extern __shared__ unsigned char smraw[];
    __shared__ int s_t;
    __shared__ unsigned s_ready;
    const unsigned cr = cluster_rank();
    if (threadIdx.x == 0) {
        s_ready = 0;   // launch epochs start at 1
        if (cr == 0) s_t = atomicAdd(ticket, (int)cluster_size());
    }
    cluster_sync();
    const int t0 = (int)ld_cluster_u32(cluster_map(smem_addr(&s_t), 0));
    const int t = t0 + (int)cr, pos = t / G, g = t % G;
    const int o = FWD ? pos : nb - 1 - pos;
    if (pos < nb && !held_back(err, o)) {
        const int c0 = g * gw, nc = max(0, min(gw, nrhs - c0));
        const CLink lk{t0, G, g, nb, smem_addr(smraw), smem_addr(&s_ready)};
        sweep_row<float2, TR, TC, NT, FWD, true, true>(o, size[o], size, boff, lptr, lidx, lent, cbo, crk, W,
                                                       x + (int64_t)c0 * n, y + (int64_t)c0 * n, n, nc, budget,
                                                       flags + g * nb, epoch, err, (float2 *)smraw, 0, nullptr,
                                                       tag + (int64_t)c0 * n, lk);
    }
    cluster_sync();   // the finished rows stay readable until every CTA of the cluster is done
}

// Chain-and-helpers sweep.  The dependencies of block row b are split: the `recent` ones,
// at most SWEEP_T positions before b in sweep order, come last in b's walk; the others are
// added by a helper CTA (sweep_row with the recent ones cut off), which leaves the partial
// sum in y and raises b's partial flag.  One chain CTA per column group then walks the
// block rows in sweep order: it continues b's sum from the partial, adds the recent
// dependencies from a shared-memory ring of the last SWEEP_T + 1 results (their coefficient
// blocks read through L1), stores y_b and raises its final flag, which the helpers wait on.
// The chain CTAs take the first tickets, so they are resident before any helper; every
// output adds its terms in the same order as with one block row per CTA.
// number of recent dependencies at the end of b's walk (|dependency - b| <= SWEEP_T)
template <bool FWD>
__device__ __forceinline__ int recent_count(int b, const int *lptr, const int *lidx)
{
    int c = 0;
    if (FWD)
        for (int p = lptr[b + 1] - 1; p >= lptr[b] && lidx[p] >= b - SWEEP_T; --p) ++c;
    else
        for (int p = lptr[b]; p < lptr[b + 1] && lidx[p] <= b + SWEEP_T; ++p) ++c;
    return c;
}

constexpr int CHAIN_WCAP = 4096;   // entries of each coefficient staging buffer of a chain CTA


// What the chain CTA needs about one block row: loaded one step ahead (independent loads),
// so that their latency overlaps the current step.
struct ChainMeta {
    int b, nb, o, nrec;
    int k[SWEEP_T], nk[SWEEP_T];
    int64_t src[SWEEP_T];   // entry offset of each recent coefficient block in W
};

template <bool FWD>
__device__ __forceinline__ ChainMeta chain_meta(int b, const int *size, const int *boff, const int *rec,
                                                const int *reccol, const int64_t *coff)
{
    ChainMeta m;
    m.b = b;
    m.nb = size[b];
    m.o = boff[b];
    m.nrec = 0;
    int col[SWEEP_T];
#pragma unroll
    for (int j = 0; j < SWEEP_T; ++j) {
        m.k[j] = rec[b * SWEEP_T + j];
        col[j] = reccol[b * SWEEP_T + j];
    }
    const int64_t cb = coff[b];
#pragma unroll
    for (int j = 0; j < SWEEP_T; ++j) {
        const int k = m.k[j] < 0 ? b : m.k[j];
        m.nk[j] = size[k];
        const int64_t ck = coff[k];
        m.src[j] = FWD ? ck + (int64_t)col[j] * m.nk[j] : cb + (int64_t)col[j] * m.nb;
        if (m.k[j] >= 0) m.nrec = j + 1;
    }
    return m;
}

template <class T, int TR, int TC, int NT, bool FWD>
__device__ void chain_run(int nb, const int *size, const int *boff, const int *rec, const int *reccol,
                          const int64_t *coff, const T *W, T *y, int n, int nc, int *fpart, int *ffin, int epoch,
                          int *err, T *ring)
{
    const int slot_sz = 64 * nc;
    T *wbuf[2] = {ring + (SWEEP_T + 1) * slot_sz, ring + (SWEEP_T + 1) * slot_sz + CHAIN_WCAP};
    // copy the recent coefficient blocks of m (concatenated) into buffer `which`; false (nothing
    // copied) when they do not fit
    auto stage = [&](const ChainMeta &m, int which) {
        int tot = 0;
#pragma unroll
        for (int j = 0; j < SWEEP_T; ++j)
            if (j < m.nrec) tot += m.nk[j] * m.nb;
        bool ok = tot <= CHAIN_WCAP;
        if (ok) {
            int off = 0;
#pragma unroll
            for (int j = 0; j < SWEEP_T; ++j)
                if (j < m.nrec) {
                    const int cnt = m.nk[j] * m.nb;
                    for (int e = threadIdx.x; e < cnt; e += blockDim.x)
                        cp_async_el(wbuf[which] + off + e, W + m.src[j] + e);
                    off += cnt;
                }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        return ok;
    };
    ChainMeta m = chain_meta<FWD>(FWD ? 0 : nb - 1, size, boff, rec, reccol, coff);
    bool staged = stage(m, 0);
    for (int q = 0; q < nb; ++q) {
        const int b = m.b, nb_ = m.nb, o = m.o;
        const int nrt = (nb_ + TR - 1) / TR, ntiles = nrt * ((nc + TC - 1) / TC);
        const bool last = q + 1 == nb;
        ChainMeta mn = chain_meta<FWD>(last ? b : (FWD ? q + 1 : nb - 2 - q), size, boff, rec, reccol, coff);
        if (threadIdx.x == 0) wait_ready(fpart, b, epoch, err);
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        const bool here = staged;
        if (!last) staged = stage(mn, (q + 1) & 1);   // the next block's coefficients, other buffer
        Tile<T, TR, TC, NT> acc;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const TileRC tm = tile_rc<TR, TC>(threadIdx.x + t * blockDim.x, nrt, ntiles);
            const int row0 = tm.row0, r0 = tm.c0;
#pragma unroll
            for (int a = 0; a < TR; ++a)
#pragma unroll
                for (int c = 0; c < TC; ++c)
                    acc.v[t][a][c] = (tm.ok && row0 + a < nb_ && r0 + c < nc)
                                         ? ldcg(y + o + row0 + a + (int64_t)(r0 + c) * n)
                                         : czero(T());
        }
        int woff = 0;
#pragma unroll
        for (int j = 0; j < SWEEP_T; ++j) {
            if (j >= m.nrec) break;
            const int k = m.k[j], nk = m.nk[j];
            const int qk = FWD ? k : nb - 1 - k;   // sweep position of k
            const T *Ys = ring + (qk % (SWEEP_T + 1)) * slot_sz;   // Ys[r * nk + qq]
            // M(row, qq) = Mb[row * mr + qq * mq]
            const T *Mb = here ? wbuf[q & 1] + woff : W + m.src[j];
            const int mr = FWD ? nk : 1, mq = FWD ? 1 : nb_;
            woff += nk * nb_;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const TileRC tm = tile_rc<TR, TC>(threadIdx.x + t * blockDim.x, nrt, ntiles);
                if (tm.ok) {
                    const int row0 = tm.row0, r0 = tm.c0;
#pragma unroll 4
                    for (int qq = 0; qq < nk; ++qq) {
                        T w[TR], yv[TC];
#pragma unroll
                        for (int a = 0; a < TR; ++a)
                            w[a] = row0 + a < nb_ ? Mb[(row0 + a) * mr + qq * mq] : czero(T());
#pragma unroll
                        for (int c = 0; c < TC; ++c) yv[c] = Ys[(r0 + c) * nk + qq];
#pragma unroll
                        for (int a = 0; a < TR; ++a)
#pragma unroll
                            for (int c = 0; c < TC; ++c) acc.v[t][a][c] = cfms(w[a], yv[c], acc.v[t][a][c]);
                    }
                }
            }
        }
        // y_b: to the ring (as a vector block, r * nb_ + row) and to global memory
        T *slot = ring + (q % (SWEEP_T + 1)) * slot_sz;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const TileRC tm = tile_rc<TR, TC>(threadIdx.x + t * blockDim.x, nrt, ntiles);
            const int row0 = tm.row0, r0 = tm.c0;
#pragma unroll
            for (int a = 0; a < TR; ++a)
#pragma unroll
                for (int c = 0; c < TC; ++c)
                    if (tm.ok && row0 + a < nb_ && r0 + c < nc) {
                        slot[(r0 + c) * nb_ + row0 + a] = acc.v[t][a][c];
                        y[o + row0 + a + (int64_t)(r0 + c) * n] = acc.v[t][a][c];
                    }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            *(volatile int *)(ffin + b) = epoch;
        }
        m = mn;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <class T, int TR, int TC, int NT, bool FWD>
__global__ void __launch_bounds__(256) k_sweep_ch(int nb, const int *size, const int *boff, const int *lptr,
                                                  const int *lidx, const int *lcol, const int *rec, const int *reccol,
                                                  const int64_t *coff, const int *lent, const int64_t *cbo,
                                                  const int *crk, const T *W,
                                                  const T *x, T *y, int n, int nrhs, int G, int gw, int budget,
                                                  int *flags, int epoch, int *ticket, int *err)
{
    extern __shared__ unsigned char smraw[];
    __shared__ int s_t;
    if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int t = s_t;
    if (t >= G * (nb + 1)) return;
    const int g = t < G ? t : (t - G) % G;
    const int c0 = g * gw, nc = max(0, min(gw, nrhs - c0));
    int *ffin = flags + g * nb, *fpart = flags + (SWEEP_GMAX + g) * nb;
    if (t < G) {
        chain_run<T, TR, TC, NT, FWD>(nb, size, boff, rec, reccol, coff, W, y + (int64_t)c0 * n, n, nc, fpart, ffin,
                                      epoch, err, (T *)smraw);
        return;
    }
    const int qpos = (t - G) / G, b = FWD ? qpos : nb - 1 - qpos;
    if (held_back(err, b)) return;
    const int cut = recent_count<FWD>(b, lptr, lidx);
    sweep_row<T, TR, TC, NT, FWD>(b, size[b], size, boff, lptr, lidx, lent, cbo, crk, W, x + (int64_t)c0 * n,
                                  y + (int64_t)c0 * n, n, nc, budget, ffin, epoch, err, (T *)smraw, cut, fpart);
}

// Super-row sweep (both directions): one CTA computes the SR consecutive blocks (sweep
// order) of super-row r for one column group.  The members' external dependencies are
// added chunk by chunk as in sweep_row (members without a coefficient block for a
// dependency get zero rows, which leave their sums unchanged); then member s is final,
// stored and published, and its product with the later members' coefficient blocks is
// taken from shared memory before the next member is published.  Every output therefore
// adds its terms in the same order as with one block per CTA.
template <class T, int TR, int TC, int NT, bool FWD>
__global__ void __launch_bounds__(256) k_sweep_sr(int nb, int nsr, const int *size, const int *boff, const int *xptr,
                                                  const int *xdep, const int *xoff, const int *xint,
                                                  const int64_t *coff, const T *W, const T *x, T *y, int n, int nrhs,
                                                  int G, int gw, int budget, int *flags, int epoch, int *ticket,
                                                  int *err)
{
    constexpr int SR = SWEEP_SR;
    extern __shared__ unsigned char smraw[];
    T *buf = (T *)smraw;
    __shared__ int s_t;
    if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int r = s_t / G, g = s_t % G;
    if (r >= nsr) return;
    const int c0 = g * gw, nc = max(0, min(gw, nrhs - c0));
    x += (int64_t)c0 * n;
    y += (int64_t)c0 * n;
    flags += g * nb;
    int mb[SR], R[SR + 1], nm = 0;
    R[0] = 0;
#pragma unroll
    for (int s = 0; s < SR; ++s) {
        const int q = r * SR + s;
        mb[s] = q < nb ? (FWD ? q : nb - 1 - q) : -1;
        if (q < nb) nm = s + 1;
        R[s + 1] = R[s] + (q < nb ? size[mb[s]] : 0);
    }
#pragma unroll
    for (int s = 0; s < SR; ++s)
        if (mb[s] >= 0 && held_back(err, mb[s])) return;
    const int no = R[nm];
    const int nrt = (no + TR - 1) / TR, ntiles = nrt * ((nc + TC - 1) / TC);
    const int ldw = stage_ldw(no, TR);
    auto member = [&](int row) {
        int s = 0;
#pragma unroll
        for (int t = 1; t < SR; ++t)
            if (row >= R[t]) s = t;
        return s;
    };
    Tile<T, TR, TC, NT> acc;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const TileRC tm = tile_rc<TR, TC>(threadIdx.x + t * blockDim.x, nrt, ntiles);
        const int row0 = tm.row0, q0 = tm.c0;
#pragma unroll
        for (int a = 0; a < TR; ++a) {
            const int row = row0 + a, s = member(row);
            const int64_t gr = row < no ? boff[mb[s]] + row - R[s] : 0;
#pragma unroll
            for (int c = 0; c < TC; ++c)
                acc.v[t][a][c] = (tm.ok && row < no && q0 + c < nc) ? x[gr + (int64_t)(q0 + c) * n] : czero(T());
        }
    }
    // external dependencies, in the stored order
    const int pa = xptr[r], pend = xptr[r + 1];
    for (int p = pa; p != pend;) {
        const int q = next_chunk<TR, TC>(p, pend, 1, xdep, size, no, nc, budget, nullptr, nullptr);
        int off = 0;
        for (int b = p; b != q; ++b) {
            const int k = xdep[b], nq = size[k];
            T *Ws = buf + off;
            const int *xo = xoff + (int64_t)b * SR;
            stage_copy(nq * no, [&](int e) {
                const int qq = e % nq, row = e / nq, s = member(row), o = xo[s], rr = row - R[s];
                if (o < 0) return czero(T());
                // forward: W_{k,m_s} (nq x n_s) element (qq, rr); backward: W_{m_s,k} (n_s x nq) element (rr, qq)
                const int ns = R[s + 1] - R[s];
                return FWD ? W[coff[k] + (int64_t)o * nq + qq + (int64_t)rr * nq]
                           : W[coff[mb[s]] + (int64_t)o * ns + rr + (int64_t)qq * ns];
            }, [&](int e, T v) { Ws[(e % nq) * ldw + e / nq] = v; });
            off += stage_need(no, nq, nc, TR, TC);
        }
        if (threadIdx.x == 0)
            for (int b = p; b != q; ++b) wait_ready(flags, xdep[b], epoch, err);
        __syncthreads();
        off = 0;
        for (int b = p; b != q; ++b) {
            const int k = xdep[b], nq = size[k], ok = boff[k];
            T *Ys = buf + off + nq * ldw;
            stage_copy(nq * nc, [&](int e) { return ldcg(y + ok + e % nq + (int64_t)(e / nq) * n); },
                       [&](int e, T v) { Ys[e] = v; });
            off += stage_need(no, nq, nc, TR, TC);
        }
        __syncthreads();
        off = 0;
        for (int b = p; b != q; ++b) {
            const int nq = size[xdep[b]];
            tile_mac<true>(acc, buf + off, ldw, buf + off + nq * ldw, 1, nq, nq, nrt, ntiles);
            off += stage_need(no, nq, nc, TR, TC);
        }
        __syncthreads();
        p = q;
    }
    // members in sweep order: store and publish member s, then apply it to the later members
    for (int s = 0; s < nm; ++s) {
        const int ns = R[s + 1] - R[s];
        T *Yint = buf + ns * ldw;   // member s's entries as the vector block (nc x ns)
        const bool more = s + 1 < nm;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const TileRC tm = tile_rc<TR, TC>(threadIdx.x + t * blockDim.x, nrt, ntiles);
            const int row0 = tm.row0, q0 = tm.c0;
#pragma unroll
            for (int a = 0; a < TR; ++a) {
                const int row = row0 + a;
                if (tm.ok && row >= R[s] && row < R[s + 1]) {
                    const int64_t gr = boff[mb[s]] + row - R[s];
#pragma unroll
                    for (int c = 0; c < TC; ++c)
                        if (q0 + c < nc) {
                            y[gr + (int64_t)(q0 + c) * n] = acc.v[t][a][c];
                            if (more) Yint[(q0 + c) * ns + row - R[s]] = acc.v[t][a][c];
                        }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            *(volatile int *)(flags + mb[s]) = epoch;
        }
        if (!more) break;
        // coefficients of member s for the later members: rows of member s2 > s from the
        // block coupling them (forward W_{m_s, m_s2} in panel m_s, backward W_{m_s2, m_s} in
        // panel m_s2), zero elsewhere
        stage_copy(ns * no, [&](int e) {
            const int qq = e % ns, row = e / ns, s2 = member(row);
            const int o = s2 > s ? xint[((int64_t)r * SR + s) * SR + s2] : -1;
            if (o < 0) return czero(T());
            const int rr = row - R[s2], n2 = R[s2 + 1] - R[s2];
            return FWD ? W[coff[mb[s]] + (int64_t)o * ns + qq + (int64_t)rr * ns]
                       : W[coff[mb[s2]] + (int64_t)o * n2 + rr + (int64_t)qq * n2];
        }, [&](int e, T v) { buf[(e % ns) * ldw + e / ns] = v; });
        __syncthreads();
        tile_mac<true>(acc, buf, ldw, Yint, 1, ns, ns, nrt, ntiles);
        __syncthreads();
    }
}

// dst[i*nrhs + r] = src[idx[i] + r*n]   (right-hand sides interleaved)
template <class T>
__global__ void k_gather_il(int n, int nrhs, const int *idx, const T *src, T *dst)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nrhs) return;
    int i = (int)(e / nrhs), r = (int)(e % nrhs);
    dst[e] = src[idx[i] + (int64_t)r * n];
}

// dst[idx[i] + r*ldd] = src[i + r*n]
__global__ void k_scatter_cols(int n, int nrhs, const int *idx, const double2 *src, double2 *dst, int64_t ldd)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nrhs) return;
    int i = (int)(e % n), r = (int)(e / n);
    dst[idx[i] + r * ldd] = src[e];
}

// dst[i + r*n] = src[idx[i] + r*lds]
__global__ void k_gather_cols(int n, int nrhs, const int *idx, const double2 *src, int64_t lds, double2 *dst)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nrhs) return;
    int i = (int)(e % n), r = (int)(e / n);
    dst[e] = src[idx[i] + r * lds];
}

__global__ void k_narrow(int64_t len, const double2 *src, float2 *dst)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < len) dst[e] = make_float2((float)src[e].x, (float)src[e].y);
}

__global__ void k_widen(int64_t len, const float2 *src, double2 *dst)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < len) dst[e] = make_double2((double)src[e].x, (double)src[e].y);
}

// Block-diagonal operations (Eq. 28), one CTA per block:
//   mode 0: y = D^{-1} (D x + w);  mode 1: y = D^{-1} x;  mode 2: y = D x
template <class T>
__global__ void __launch_bounds__(256) k_diag(int mode, int nb, const int *size, const int *boff,
                                              const int64_t *doff, const T *D, const T *Dinv, const T *x,
                                              const T *w, T *y, int n, int nrhs)
{
    extern __shared__ unsigned char smraw[];
    T *xs = (T *)smraw, *ts = xs + 64 * nrhs;
    const int k = blockIdx.x;
    if (k >= nb) return;
    const int nk = size[k], o = boff[k];
    for (int e = threadIdx.x; e < nk * nrhs; e += blockDim.x) {
        const int rw = e % nk, r = e / nk;
        xs[e] = x[o + rw + (int64_t)r * n];
    }
    __syncthreads();
    const T *Dk = D + doff[k], *Ik = Dinv + doff[k];
    if (mode == 0) {
        for (int e = threadIdx.x; e < nk * nrhs; e += blockDim.x) {
            const int rw = e % nk, r = e / nk;
            T acc = w[o + rw + (int64_t)r * n];
            for (int c = 0; c < nk; ++c) acc = cfma(Dk[rw + c * nk], xs[c + r * nk], acc);
            ts[e] = acc;
        }
        __syncthreads();
        xs = ts;
    }
    const T *Mk = (mode == 2) ? Dk : Ik;
    for (int e = threadIdx.x; e < nk * nrhs; e += blockDim.x) {
        const int rw = e % nk, r = e / nk;
        T acc = czero(T());
        for (int c = 0; c < nk; ++c) acc = cfma(Mk[rw + c * nk], xs[c + r * nk], acc);
        y[o + rw + (int64_t)r * n] = acc;
    }
}

// Near-field product for the refinement residual: y += Z_N u, u in cluster order, y in solve
// order.  One CTA per leaf, summing near blocks (t, s) and mirrored (s, t) blocks (FP64).
__global__ void __launch_bounds__(128) k_near_mv(int nl, const int *leaf_ptr, const int *nptr, const int *nent,
                                                 const int *near_t, const int *near_s, const int64_t *near_off,
                                                 const double2 *near, const double2 *u, const int *cl2new, int n,
                                                 int nrhs, double2 *y)
{
    const int l = blockIdx.x;
    if (l >= nl) return;
    const int a = leaf_ptr[l], ni = leaf_ptr[l + 1] - a;
    const int on = cl2new[a];
    for (int e = threadIdx.x; e < ni * nrhs; e += blockDim.x) {
        const int i = e % ni, r = e / ni;
        double2 acc = y[on + i + (int64_t)r * n];
        for (int p = nptr[l]; p < nptr[l + 1]; ++p) {
            const int b = nent[p] >> 1, side = nent[p] & 1;
            const int t = near_t[b], s = near_s[b];
            const int mt = leaf_ptr[t + 1] - leaf_ptr[t];
            const double2 *B = near + near_off[b];
            if (side == 0) {   // row l = t: sum_c B[i, c] u_s[c]
                const int ms = leaf_ptr[s + 1] - leaf_ptr[s];
                const double2 *us = u + (int64_t)leaf_ptr[s] * nrhs + r;
                for (int c = 0; c < ms; ++c) acc = cfma(B[i + (int64_t)c * mt], us[(int64_t)c * nrhs], acc);
            } else {           // row l = s (t != s): sum_q B[q, i] u_t[q]
                const double2 *ut = u + (int64_t)leaf_ptr[t] * nrhs + r;
                for (int q = 0; q < mt; ++q) acc = cfma(B[q + (int64_t)i * mt], ut[(int64_t)q * nrhs], acc);
            }
        }
        y[on + i + (int64_t)r * n] = acc;
    }
}

// ---- host side -------------------------------------------------------------------------
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <class T> struct OpData {
    const T *W, *Ad, *Dinv, *U, *V;
    T *t, *s, *work;
};

static OpData<double2> data64(hm_ctx *h)
{
    return {h->d_Wc, h->d_Ad, h->d_Dinv, h->d_farU, h->d_farV, h->d_t, h->d_s, h->d_work};
}
static OpData<float2> data32(hm_ctx *h)
{
    return {h->d_Wc32, h->d_Ad32, h->d_Dinv32, h->d_farU32, h->d_farV32, h->d_t32, h->d_s32, h->d_work32};
}

// Widest column batch one sweep launch takes (wider requests are split into slices).
template <class T> static int max_cols() { return sizeof(T) == 16 ? 16 : 64; }

// Register tile per group width: (TR, TC, NT) = (1, 1, 1) up to 4 columns, (2, 2, 1) up
// to 16, (2, 4, 2) up to 64 (complex FP32 only); 256 threads cover every output tile of a
// 64-row block (a 2 x 2 tile at 17-32 columns measured 2% slower).  Shared memory: FP64,
// one chunk (at least one 64 x 64 coefficient block with its vector block); complex FP32,
// see SW_WCAP.
template <class T, int TR, int TC, int NT>
static cudaError_t sweep_shape(hm_ctx *h, const OpData<T> &d, bool forward, const T *x, T *y, int nrhs, int G,
                               int gw, int ep, int maxw)
{
    Plan &P = h->plan;
    // complex FP32: two coefficient buffers and a vector area (sweep_row); FP64: one chunk
    auto need = [](int w) {
        return sizeof(T) == 8 ? 2 * SW_WCAP + 64 * stage_ldr(w, TC) : stage_need(64, 64, w, TR, TC);
    };
    const int budget = need(gw);
    const size_t smem = sizeof(T) * (size_t)budget;
    static DeviceOnce attr;
    if (attr.need()) {
        const int smax = (int)(sizeof(T) * (size_t)need(maxw));
        cudaFuncSetAttribute(k_sweep_fwd<T, TR, TC, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        cudaFuncSetAttribute(k_sweep_bwd<T, TR, TC, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        attr.done();
    }
    const unsigned grid = (unsigned)(P.nb * G);
    if (forward)
        HM_LAUNCH(h, K_SWEEP_FWD,
                  (k_sweep_fwd<T, TR, TC, NT><<<grid, 256, smem, h->stream>>>(
                      P.nb, h->d_size, h->d_boff, h->d_rptr, h->d_ridx, h->d_rent, h->d_cboff, h->d_crank, d.W, x, y,
                      P.n, nrhs, G, gw, budget, h->d_flags, ep, h->d_ticket, h->d_err, h->d_ytag)));
    else
        HM_LAUNCH(h, K_SWEEP_BWD,
                  (k_sweep_bwd<T, TR, TC, NT><<<grid, 256, smem, h->stream>>>(
                      P.nb, h->d_size, h->d_boff, h->d_sptr, h->d_sidx, h->d_cboff, h->d_crank, d.W, x, y, P.n, nrhs,
                      G, gw, budget, h->d_flags, ep, h->d_ticket, h->d_err, h->d_ytag)));
    return cudaGetLastError();
}

// Cluster-chained launch (complex FP32): the shared memory of sweep_shape, clusters of C CTAs
// (8, or 16 where the device allows it), the grid rounded up to whole clusters.  Both kernels
// of a tile shape get the shared-memory limit of the shape's widest group (maxw) once.
template <int TR, int TC, int NT> static size_t sweep_cl_smem(int w)
{
    return sizeof(float2) * (size_t)(2 * SW_WCAP + 64 * stage_ldr(w, TC));
}
template <int TR, int TC, int NT> static void sweep_cl_attrs(int maxw)
{
    static DeviceOnce attr;
    if (!attr.need()) return;
    for (auto k : {k_sweep_cl<TR, TC, NT, true>, k_sweep_cl<TR, TC, NT, false>}) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_cl_smem<TR, TC, NT>(maxw));
        cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
    attr.done();
}

template <int TR, int TC, int NT>
static cudaError_t sweep_cl_shape(hm_ctx *h, const OpData<float2> &d, bool forward, const float2 *x, float2 *y,
                                  int nrhs, int G, int gw, int ep, int maxw, int C)
{
    Plan &P = h->plan;
    sweep_cl_attrs<TR, TC, NT>(maxw);
    const int budget = 2 * SW_WCAP + 64 * stage_ldr(gw, TC);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(((int64_t)P.nb * G + C - 1) / C * C));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = sweep_cl_smem<TR, TC, NT>(gw);
    cfg.stream = h->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (forward)
        HM_LAUNCH(h, K_SWEEP_FWD,
                  e = cudaLaunchKernelEx(&cfg, k_sweep_cl<TR, TC, NT, true>, P.nb, (const int *)h->d_size,
                                         (const int *)h->d_boff, (const int *)h->d_rptr, (const int *)h->d_ridx,
                                         (const int *)h->d_rent, (const int64_t *)h->d_cboff,
                                         (const int *)h->d_crank, d.W, x, y, P.n, nrhs, G, gw, budget, h->d_flags, ep,
                                         h->d_ticket, h->d_err, h->d_ytag));
    else
        HM_LAUNCH(h, K_SWEEP_BWD,
                  e = cudaLaunchKernelEx(&cfg, k_sweep_cl<TR, TC, NT, false>, P.nb, (const int *)h->d_size,
                                         (const int *)h->d_boff, (const int *)h->d_sptr, (const int *)h->d_sidx,
                                         (const int *)nullptr, (const int64_t *)h->d_cboff, (const int *)h->d_crank,
                                         d.W, x, y, P.n, nrhs, G, gw, budget, h->d_flags, ep, h->d_ticket, h->d_err,
                                         h->d_ytag));
    if (e) return e;
    return cudaGetLastError();
}

// Largest cluster (16 or 8 CTAs; 0: neither) with which a cluster-chained sweep of the tile
// shape fits the device at the shape's widest group (maxw); asked once per shape and device.
template <int TR, int TC, int NT>
static int sweep_cl_max(int maxw)
{
    static std::atomic<int> cache[64];   // per device: the answer + 1, 0 = not asked yet
    const int dev = DeviceOnce::device();
    if (dev >= 0 && dev < 64 && cache[dev].load() > 0) return cache[dev].load() - 1;
    sweep_cl_attrs<TR, TC, NT>(maxw);
    int cached = 0;
    for (int C = 16; C >= 8; C /= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = sweep_cl_smem<TR, TC, NT>(maxw);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_sweep_cl<TR, TC, NT, true>, &cfg) == cudaSuccess &&
            nclusters > 0) {
            cached = C;
            break;
        }
        cudaGetLastError();
    }
    if (dev >= 0 && dev < 64) cache[dev].store(cached + 1);
    return cached;
}

// Super-row launch: (TR, TC, NT) = (1, 1, 2) up to 4 columns per group, else (2, 2, 2) up to 16.
template <class T, int TR, int TC, int NT>
static cudaError_t sweep_sr_shape(hm_ctx *h, const OpData<T> &d, bool forward, const T *x, T *y, int nrhs, int G,
                                  int gw, int ep, int maxw)
{
    Plan &P = h->plan;
    const int budget = stage_need(64 * SWEEP_SR, 64, gw, TR, TC);
    const size_t smem = sizeof(T) * (size_t)budget;
    static DeviceOnce attr;
    if (attr.need()) {
        const int smax = (int)(sizeof(T) * (size_t)stage_need(64 * SWEEP_SR, 64, maxw, TR, TC));
        cudaFuncSetAttribute(k_sweep_sr<T, TR, TC, NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        cudaFuncSetAttribute(k_sweep_sr<T, TR, TC, NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        attr.done();
    }
    const int nsr = (P.nb + SWEEP_SR - 1) / SWEEP_SR, dir = forward ? 0 : 1;
    const unsigned grid = (unsigned)(nsr * G);
    if (forward)
        HM_LAUNCH(h, K_SWEEP_FWD,
                  (k_sweep_sr<T, TR, TC, NT, true><<<grid, 256, smem, h->stream>>>(
                      P.nb, nsr, h->d_size, h->d_boff, h->d_xptr[dir], h->d_xdep[dir], h->d_xoff[dir], h->d_xint[dir],
                      h->d_coff, d.W, x, y, P.n, nrhs, G, gw, budget, h->d_flags, ep, h->d_ticket, h->d_err)));
    else
        HM_LAUNCH(h, K_SWEEP_BWD,
                  (k_sweep_sr<T, TR, TC, NT, false><<<grid, 256, smem, h->stream>>>(
                      P.nb, nsr, h->d_size, h->d_boff, h->d_xptr[dir], h->d_xdep[dir], h->d_xoff[dir], h->d_xint[dir],
                      h->d_coff, d.W, x, y, P.n, nrhs, G, gw, budget, h->d_flags, ep, h->d_ticket, h->d_err)));
    return cudaGetLastError();
}

// Chain-and-helpers launch: one chain CTA per column group plus one helper per block row
// and group; (TR, TC, NT) = (1, 1, 1) up to 4 columns per group, else (2, 2, 1) up to 16.
template <class T, int TR, int TC, int NT>
static cudaError_t sweep_ch_shape(hm_ctx *h, const OpData<T> &d, bool forward, const T *x, T *y, int nrhs, int G,
                                  int gw, int ep, int maxw)
{
    Plan &P = h->plan;
    const int budget = std::max(stage_need(64, 64, gw, TR, TC), (SWEEP_T + 1) * 64 * gw + 2 * CHAIN_WCAP);
    const size_t smem = sizeof(T) * (size_t)budget;
    static DeviceOnce attr;
    if (attr.need()) {
        const int smax = (int)(sizeof(T) * (size_t)std::max(stage_need(64, 64, maxw, TR, TC),
                                                            (SWEEP_T + 1) * 64 * maxw + 2 * CHAIN_WCAP));
        cudaFuncSetAttribute(k_sweep_ch<T, TR, TC, NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        cudaFuncSetAttribute(k_sweep_ch<T, TR, TC, NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        attr.done();
    }
    const unsigned grid = (unsigned)(G * (P.nb + 1));
    if (forward)
        HM_LAUNCH(h, K_SWEEP_FWD,
                  (k_sweep_ch<T, TR, TC, NT, true><<<grid, 256, smem, h->stream>>>(
                      P.nb, h->d_size, h->d_boff, h->d_rptr, h->d_ridx, h->d_rcol, h->d_rec[0], h->d_reccol[0],
                      h->d_coff, h->d_rent, h->d_cboff, h->d_crank, d.W, x, y, P.n, nrhs, G, gw, budget, h->d_flags, ep,
                      h->d_ticket, h->d_err)));
    else
        HM_LAUNCH(h, K_SWEEP_BWD,
                  (k_sweep_ch<T, TR, TC, NT, false><<<grid, 256, smem, h->stream>>>(
                      P.nb, h->d_size, h->d_boff, h->d_sptr, h->d_sidx, h->d_srow, h->d_rec[1], h->d_reccol[1],
                      h->d_coff, (const int *)nullptr, h->d_cboff, h->d_crank, d.W, x, y, P.n, nrhs, G, gw, budget,
                      h->d_flags, ep, h->d_ticket, h->d_err)));
    return cudaGetLastError();
}

// Complex-FP32 sweep on the tensor cores (k_sweep_tc): shared memory = the operand planes
// and drained accumulator, two raw coefficient buffers, alignment slack.
static cudaError_t sweep_tc_launch(hm_ctx *h, const OpData<float2> &d, bool forward, const float2 *x, float2 *y,
                                   int nrhs, int G, int gw, int ep)
{
    Plan &P = h->plan;
    const size_t smem = tc::REGION_BYTES + 2 * TCW_BYTES + 1024;
    static DeviceOnce attr;
    if (attr.need()) {
        cudaFuncSetAttribute(k_sweep_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_sweep_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr.done();
    }
    const unsigned grid = (unsigned)(P.nb * G);
    if (forward)
        HM_LAUNCH(h, K_SWEEP_FWD,
                  (k_sweep_tc<true><<<grid, 256, smem, h->stream>>>(P.nb, h->d_size, h->d_boff, h->d_rptr, h->d_ridx,
                                                                    h->d_rcol, h->d_coff, d.W, x, y, P.n, nrhs, G, gw,
                                                                    ep, h->d_ticket, h->d_err, h->d_ytag)));
    else
        HM_LAUNCH(h, K_SWEEP_BWD,
                  (k_sweep_tc<false><<<grid, 256, smem, h->stream>>>(P.nb, h->d_size, h->d_boff, h->d_sptr, h->d_sidx,
                                                                     h->d_srow, h->d_coff, d.W, x, y, P.n, nrhs, G, gw,
                                                                     ep, h->d_ticket, h->d_err, h->d_ytag)));
    return cudaGetLastError();
}

static int width_class(int w) { return w <= 4 ? 0 : w <= 8 ? 1 : w <= 16 ? 2 : w <= 32 ? 3 : 4; }

// Number of column groups for a sweep of nrhs columns: the tuned choice of the width class,
// or the next untried candidate (then *tu / *slot let the caller time the launch).
static int sweep_groups(hm_ctx *h, bool fp32, bool forward, int nrhs, SweepTune **tu, int *slot)
{
    *tu = nullptr;
    if (h->sweep_fixed) return h->sweep_fixed;
    SweepTune &t = h->sweep_tune[fp32][forward][width_class(nrhs)];
    if (t.best) return t.best;
    if (t.ncand == 0) {
        for (int G = 1; G <= SWEEP_GMAX; G *= 2) {
            const int gw = (nrhs + G - 1) / G;
            if (G > 1 && gw < 4) continue;
            // one block row per CTA; the super-row and chain-and-helpers kinds compute the same
            // sums but measured slower on every width, and so did the tensor-core kind for the
            // complex-FP32 sweeps (8.7 against 6.1 ms per 64-column launch on the 30,720-unknown
            // sphere: its chunks of 32 are staged and multiplied one after the other); they stay
            // selectable.  Each group width tries its register-tile shapes (sweep_tile_shapes):
            // the same sums, more or fewer threads busy on small block rows.
            for (int tv = 0; tv < (gw > 4 ? 3 : 1); ++tv) t.cand[t.ncand++] = G | (1 << 4) | (tv << 8);
        }
        // The cluster-chained kinds (5, 6) stay selectable but are not tried: on the
        // 30,720-unknown sphere they measured 8-14% slower than kind 1 at every width (1: 3.69
        // against 3.24 ms per forward sweep; 64 in two groups: 5.74 against 5.18 ms) -- a
        // finished CTA holds its slot until the whole cluster is done, and a row's wait is not
        // dominated by the L2 round trip that distributed shared memory removes.
    }
    if (t.ncand == 1) return t.best = t.cand[0];
    if (t.trial < t.ncand) {
        if (!t.ev[0])
            for (cudaEvent_t &e : t.ev) cudaEventCreate(&e);
        *tu = &t;
        *slot = t.trial;
        t.width[t.trial] = nrhs;
        return t.cand[t.trial++];
    }
    // every candidate has run once: keep the fastest per column
    float best = 0;
    for (int c = 0; c < t.ncand; ++c) {
        float ms = 0;
        cudaEventSynchronize(t.ev[2 * c + 1]);
        cudaEventElapsedTime(&ms, t.ev[2 * c], t.ev[2 * c + 1]);
        ms /= (float)t.width[c];
        if (c == 0 || ms < best) {
            best = ms;
            t.best = t.cand[c];
        }
    }
    for (cudaEvent_t &e : t.ev) cudaEventDestroy(e), e = nullptr;
    return t.best;
}

void sweep_tune_release(hm_ctx *h)
{
    for (auto &a : h->sweep_tune)
        for (auto &b : a)
            for (SweepTune &t : b)
                for (cudaEvent_t &e : t.ev)
                    if (e) cudaEventDestroy(e), e = nullptr;
}

template <class T>
static cudaError_t sweep(hm_ctx *h, const OpData<T> &d, bool forward, const T *x, T *y, int nrhs)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(h->d_ticket, 0, sizeof(int), h->stream))) return e;
    const int ep = ++h->epoch;
    h->prof.cols[forward ? K_SWEEP_FWD : K_SWEEP_BWD] += nrhs;
    SweepTune *tu;
    int slot = 0;
    const int code = sweep_groups(h, sizeof(T) == 8, forward, nrhs, &tu, &slot);
    const int G = std::min(code & 15, nrhs), tv = (code >> 8) & 3;
    // the super-row, chain-and-helpers and tensor-core kinds read the dense panel layout; with
    // compressed fill-in blocks stored as factors they take kind 1 (the cluster kinds read both)
    const int kind = (code >> 4) & 15;
    const int sr = h->lowrank && kind < 5 ? 1 : kind;
    const int gw = (nrhs + G - 1) / G;
    if (tu) cudaEventRecord(tu->ev[2 * slot], h->stream);
    if constexpr (sizeof(T) == 8) {
        if (sr == 4) {
            e = sweep_tc_launch(h, d, forward, x, y, nrhs, G, gw, ep);
            if (tu) cudaEventRecord(tu->ev[2 * slot + 1], h->stream);
            return e;
        }
        if (sr == 5 || sr == 6) {
            // kind 6 asks for clusters of 16 (non-portable): 8 where the device cannot fit them
            int C = 8;
            if (sr == 6)
                C = (gw <= 4 ? sweep_cl_max<1, 1, 1>(4)
                             : gw <= 16 ? sweep_cl_max<2, 2, 1>(16) : sweep_cl_max<2, 4, 2>(64)) >= 16 ? 16 : 8;
            if (gw <= 4) e = sweep_cl_shape<1, 1, 1>(h, d, forward, x, y, nrhs, G, gw, ep, 4, C);
            else if (gw <= 16) e = sweep_cl_shape<2, 2, 1>(h, d, forward, x, y, nrhs, G, gw, ep, 16, C);
            else e = sweep_cl_shape<2, 4, 2>(h, d, forward, x, y, nrhs, G, gw, ep, 64, C);
            if (tu) cudaEventRecord(tu->ev[2 * slot + 1], h->stream);
            return e;
        }
    }
    if (sr == 3 && gw <= 16) {
        if (gw <= 4) e = sweep_ch_shape<T, 1, 1, 1>(h, d, forward, x, y, nrhs, G, gw, ep, 4);
        else e = sweep_ch_shape<T, 2, 2, 1>(h, d, forward, x, y, nrhs, G, gw, ep, 16);
    } else if (sr == 2 && gw <= 16) {
        if (gw <= 4) e = sweep_sr_shape<T, 1, 1, 2>(h, d, forward, x, y, nrhs, G, gw, ep, 4);
        else e = sweep_sr_shape<T, 2, 2, 2>(h, d, forward, x, y, nrhs, G, gw, ep, 16);
    } else if (gw <= 4) e = sweep_shape<T, 1, 1, 1>(h, d, forward, x, y, nrhs, G, gw, ep, 4);
    else if (gw <= 16 || sizeof(T) == 16) {
        // register-tile shapes (TR, TC, NT) for up to 16 columns per group: every one covers a
        // 64 x 16 output block with 256 threads
        if (tv == 1) e = sweep_shape<T, 1, 2, 2>(h, d, forward, x, y, nrhs, G, gw, ep, 16);
        else if (tv == 2) e = sweep_shape<T, 1, 1, 4>(h, d, forward, x, y, nrhs, G, gw, ep, 16);
        else e = sweep_shape<T, 2, 2, 1>(h, d, forward, x, y, nrhs, G, gw, ep, 16);
    } else if constexpr (sizeof(T) == 8) {
        // up to 64 columns per group (complex FP32): 64 x 64 output blocks
        if (tv == 1) e = sweep_shape<T, 2, 2, 4>(h, d, forward, x, y, nrhs, G, gw, ep, 64);
        else if (tv == 2) e = sweep_shape<T, 1, 4, 4>(h, d, forward, x, y, nrhs, G, gw, ep, 64);
        else e = sweep_shape<T, 2, 4, 2>(h, d, forward, x, y, nrhs, G, gw, ep, 64);
    }
    if (tu) cudaEventRecord(tu->ev[2 * slot + 1], h->stream);
    return e;
}

// y (solve order) = Z_F x (solve order); ucl receives the cluster-order copy of x with the
// right-hand sides interleaved (ucl[i*nrhs + r])
template <class T>
static cudaError_t far_apply(hm_ctx *h, const OpData<T> &d, const T *x, T *y, int nrhs, T *ucl)
{
    Plan &P = h->plan;
    FarPlan &F = h->fplan;
    const int n = P.n;
    HM_LAUNCH(h, K_PERMUTE, k_gather_il<T><<<nblk((int64_t)n * nrhs, 256), 256, 0, h->stream>>>(n, nrhs, h->d_cl2new, x,
                                                                                            ucl));
    (void)F;
    cudaError_t e = far_product<T>(h, d.U, d.V, d.t, d.s, ucl, y, nrhs);
    if (e) return e;
    return cudaGetLastError();
}

template <class T>
static cudaError_t diag(hm_ctx *h, const OpData<T> &d, int mode, const T *x, const T *w, T *y, int nrhs)
{
    Plan &P = h->plan;
    HM_LAUNCH(h, K_DIAG,
              k_diag<T><<<P.nb, 256, sizeof(T) * 128 * nrhs, h->stream>>>(mode, P.nb, h->d_size, h->d_boff,
                                                                           h->d_doff, d.Ad, d.Dinv, x, w, y, P.n,
                                                                           nrhs));
    return cudaGetLastError();
}

template <class T>
static void set_attrs()
{
    cudaFuncSetAttribute(k_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(T) * 128 * 64));
}

cudaError_t ensure_solve_workspace(hm_ctx *h, int nrhs)
{
    cudaError_t e;
    const int n = h->plan.n;
    if (!h->d_flags) {
        if ((e = h->arena.alloc((void **)&h->d_flags, sizeof(int) * h->plan.nb * SWEEP_GMAX * 2))) return e;
        if ((e = cudaMemsetAsync(h->d_flags, 0, sizeof(int) * h->plan.nb * SWEEP_GMAX * 2, h->stream))) return e;
        h->epoch = 0;
    }
    const size_t tl = std::max<int64_t>(1, h->fplan.tlen);
    if (h->t_cols < nrhs) {
        if (h->d_t) h->arena.release(h->d_t, 0), h->arena.release(h->d_s, 0);
        h->d_t = h->d_s = nullptr;
        h->t_cols = 0;
        if ((e = h->arena.alloc((void **)&h->d_t, sizeof(double2) * tl * nrhs))) return e;
        if ((e = h->arena.alloc((void **)&h->d_s, sizeof(double2) * tl * nrhs))) return e;
        h->t_cols = nrhs;
    }
    const size_t fpb = (size_t)FAR_PARTS * n * nrhs * sizeof(double2);
    if (h->farpart_bytes < fpb) {
        if (h->d_farpart) h->arena.release(h->d_farpart, 0);
        h->d_farpart = nullptr;
        h->farpart_bytes = 0;
        if ((e = h->arena.alloc(&h->d_farpart, fpb))) return e;
        h->farpart_bytes = fpb;
    }
    if (h->work_cols < 3 * nrhs) {
        if (h->d_work) h->arena.release(h->d_work, 0);
        h->d_work = nullptr;
        h->work_cols = 0;
        if ((e = h->arena.alloc((void **)&h->d_work, sizeof(double2) * (size_t)n * 3 * nrhs))) return e;
        h->work_cols = 3 * nrhs;
    }
    if (h->opts.precision == 1 && h->t32_cols < nrhs) {
        if (h->d_t32) h->arena.release(h->d_t32, 0), h->arena.release(h->d_s32, 0), h->arena.release(h->d_work32, 0);
        h->d_t32 = h->d_s32 = nullptr;
        h->d_work32 = nullptr;
        h->t32_cols = 0;
        if ((e = h->arena.alloc((void **)&h->d_t32, sizeof(float2) * tl * nrhs))) return e;
        if ((e = h->arena.alloc((void **)&h->d_s32, sizeof(float2) * tl * nrhs))) return e;
        if ((e = h->arena.alloc((void **)&h->d_work32, sizeof(float2) * (size_t)n * 5 * nrhs))) return e;
        h->t32_cols = nrhs;
    }
    if (h->opts.precision == 1 && !h->d_ytag) {   // tagged sweep results, 64 columns, epochs start at 1
        if ((e = h->arena.alloc((void **)&h->d_ytag, sizeof(uint4) * (size_t)n * 64))) return e;
        if ((e = cudaMemsetAsync(h->d_ytag, 0, sizeof(uint4) * (size_t)n * 64, h->stream))) return e;
    }
    static DeviceOnce attr;
    if (attr.need()) {
        set_attrs<double2>();
        set_attrs<float2>();
        attr.done();
    }
    return cudaSuccess;
}

// Complex FP32 copies of the far factors for the mixed-precision inner operator (at create).
cudaError_t make_fp32_copies(hm_ctx *h)
{
    cudaError_t e;
    auto narrow = [&](const double2 *src, float2 **dst, size_t len) -> cudaError_t {
        cudaError_t r;
        if (!*dst && (r = h->arena.alloc((void **)dst, sizeof(float2) * std::max<size_t>(len, 1)))) return r;
        if (len)
            HM_LAUNCH(h, K_VEC, k_narrow<<<nblk((int64_t)len, 256), 256, 0, h->stream>>>((int64_t)len, src, *dst));
        return cudaGetLastError();
    };
    if ((e = narrow(h->d_farU, &h->d_farU32, (size_t)h->farU_len))) return e;
    return narrow(h->d_farV, &h->d_farV32, (size_t)h->farV_len);
}

template <class T>
static cudaError_t op_chain(hm_ctx *h, const OpData<T> &d, int op, const T *x, T *y, int nrhs)
{
    const int n = h->plan.n;
    T *w0 = d.work, *w1 = d.work + (size_t)n * nrhs, *w2 = d.work + (size_t)2 * n * nrhs;
    cudaError_t e;
    if constexpr (sizeof(T) == 16) {
        if (h->opts.preconditioner == 1) {   // block Jacobi: no coefficients, L = I
            switch (op) {
            case 0:   // A x = D^{-1} (Z_N + Z_F) x, D = diag(Z_kk)
                if ((e = far_apply<T>(h, d, x, w1, nrhs, w2))) return e;   // w2: cluster-order copy of x
                HM_LAUNCH(h, K_NEAR,
                          k_near_mv<<<h->nl, 128, 0, h->stream>>>(h->nl, h->d_leaf_ptr, h->d_nptr, h->d_nent,
                                                                  h->d_near_t, h->d_near_s, h->d_near_off, h->d_near,
                                                                  w2, h->d_cl2new, n, nrhs, w1));
                return diag<T>(h, d, 1, w1, (const T *)nullptr, y, nrhs);
            case 1:
            case 2:
                return cudaMemcpyAsync(y, x, sizeof(T) * (size_t)n * nrhs, cudaMemcpyDeviceToDevice, h->stream);
            default: break;
            }
        }
        if (h->opts.preconditioner == 2 && op == 0) {
            // null-field comparison: A x = M^{-1} (Z_N + Z_F) x, M^{-1} = L^{-T} D^{-1} L^{-1}
            // with the factors of the elimination without fill
            if ((e = far_apply<T>(h, d, x, w1, nrhs, w2))) return e;   // w2: cluster-order copy of x
            HM_LAUNCH(h, K_NEAR,
                      k_near_mv<<<h->nl, 128, 0, h->stream>>>(h->nl, h->d_leaf_ptr, h->d_nptr, h->d_nent, h->d_near_t,
                                                              h->d_near_s, h->d_near_off, h->d_near, w2, h->d_cl2new,
                                                              n, nrhs, w1));
            if ((e = sweep<T>(h, d, true, w1, w0, nrhs))) return e;
            if ((e = diag<T>(h, d, 1, w0, (const T *)nullptr, w1, nrhs))) return e;
            return sweep<T>(h, d, false, w1, y, nrhs);
        }
    }
    switch (op) {
    case 0:   // A x = D^{-1} [D x + L^{-1} Z_F L^{-T} x]
        if ((e = sweep<T>(h, d, false, x, w0, nrhs))) return e;
        if ((e = far_apply<T>(h, d, w0, w1, nrhs, w2))) return e;
        if ((e = sweep<T>(h, d, true, w1, w0, nrhs))) return e;
        return diag<T>(h, d, 0, x, w0, y, nrhs);
    case 1: return sweep<T>(h, d, true, x, y, nrhs);
    case 2: return sweep<T>(h, d, false, x, y, nrhs);
    case 3: return far_apply<T>(h, d, x, y, nrhs, w2);
    case 4: return diag<T>(h, d, 1, x, (const T *)nullptr, y, nrhs);
    case 6: return diag<T>(h, d, 2, x, (const T *)nullptr, y, nrhs);
    default: return cudaErrorInvalidValue;
    }
}

// op codes as in hm_apply (0-4, plus 6 = D x); FP64 data; columns in slices of max_cols
cudaError_t op_apply(hm_ctx *h, int op, const double2 *x, double2 *y, int nrhs)
{
    cudaError_t e;
    const int w = max_cols<double2>();
    if (nrhs > w) {
        for (int c0 = 0; c0 < nrhs; c0 += w)
            if ((e = op_apply(h, op, x + (size_t)c0 * h->plan.n, y + (size_t)c0 * h->plan.n, std::min(w, nrhs - c0))))
                return e;
        return cudaSuccess;
    }
    if ((e = ensure_solve_workspace(h, nrhs))) return e;
    return op_chain<double2>(h, data64(h), op, x, y, nrhs);
}

// The same operators with complex-FP32 data and arithmetic; x, y stay complex FP64.
cudaError_t op_apply32(hm_ctx *h, int op, const double2 *x, double2 *y, int nrhs)
{
    cudaError_t e;
    const int w = max_cols<float2>();
    if (nrhs > w) {
        for (int c0 = 0; c0 < nrhs; c0 += w)
            if ((e = op_apply32(h, op, x + (size_t)c0 * h->plan.n, y + (size_t)c0 * h->plan.n,
                                std::min(w, nrhs - c0))))
                return e;
        return cudaSuccess;
    }
    if ((e = ensure_solve_workspace(h, nrhs))) return e;
    const int64_t len = (int64_t)h->plan.n * nrhs;
    OpData<float2> d = data32(h);
    float2 *x32 = h->d_work32 + 3 * len, *y32 = h->d_work32 + 4 * len;
    HM_LAUNCH(h, K_VEC, k_narrow<<<nblk(len, 256), 256, 0, h->stream>>>(len, x, x32));
    if ((e = op_chain<float2>(h, d, op, x32, y32, nrhs))) return e;
    HM_LAUNCH(h, K_VEC, k_widen<<<nblk(len, 256), 256, 0, h->stream>>>(len, y32, y));
    return cudaGetLastError();
}

// y = Z x with x, y in the ORIGINAL RWG order (near blocks + far factors, FP64).
cudaError_t z_apply_orig(hm_ctx *h, const double2 *x, double2 *y, int nrhs)
{
    cudaError_t e;
    const int w = max_cols<double2>();
    if (nrhs > w) {
        for (int c0 = 0; c0 < nrhs; c0 += w)
            if ((e = z_apply_orig(h, x + (size_t)c0 * h->plan.n, y + (size_t)c0 * h->plan.n, std::min(w, nrhs - c0))))
                return e;
        return cudaSuccess;
    }
    if ((e = ensure_solve_workspace(h, nrhs))) return e;
    const int n = h->plan.n;
    double2 *w0 = h->d_work, *w1 = h->d_work + (size_t)n * nrhs, *w2 = h->d_work + (size_t)2 * n * nrhs;
    HM_LAUNCH(h, K_PERMUTE,
              k_gather_cols<<<nblk((int64_t)n * nrhs, 256), 256, 0, h->stream>>>(n, nrhs, h->d_new2orig, x, n, w0));
    if ((e = far_apply<double2>(h, data64(h), w0, w1, nrhs, w2))) return e;   // leaves the cluster-order copy in w2
    HM_LAUNCH(h, K_NEAR,
              k_near_mv<<<h->nl, 128, 0, h->stream>>>(h->nl, h->d_leaf_ptr, h->d_nptr, h->d_nent, h->d_near_t,
                                                      h->d_near_s, h->d_near_off, h->d_near, w2, h->d_cl2new, n,
                                                      nrhs, w1));
    HM_LAUNCH(h, K_PERMUTE,
              k_scatter_cols<<<nblk((int64_t)n * nrhs, 256), 256, 0, h->stream>>>(n, nrhs, h->d_new2orig, w1, y, n));
    return cudaGetLastError();
}

// original order (ld ldv) -> solve order (ld n)
cudaError_t to_solve_order(hm_ctx *h, const double2 *src, int64_t lds, double2 *dst, int nrhs)
{
    const int n = h->plan.n;
    HM_LAUNCH(h, K_PERMUTE,
              k_gather_cols<<<nblk((int64_t)n * nrhs, 256), 256, 0, h->stream>>>(n, nrhs, h->d_new2orig, src, lds, dst));
    return cudaGetLastError();
}

// solve order (ld n) -> original order (ld ldd)
cudaError_t to_orig_order(hm_ctx *h, const double2 *src, double2 *dst, int64_t ldd, int nrhs)
{
    const int n = h->plan.n;
    HM_LAUNCH(h, K_PERMUTE,
              k_scatter_cols<<<nblk((int64_t)n * nrhs, 256), 256, 0, h->stream>>>(n, nrhs, h->d_new2orig, src, dst, ldd));
    return cudaGetLastError();
}

}  // namespace hm
