// Far-field product v = Z_F u (Sec. 2 Eq. 9 blocks, Eq. 11), complex FP64 or FP32.
//
// Z_F is stored once per admissible pair (rows r-range, columns c-range, r before c): a
// low-rank block U V^T or a dense block B; the mirrored block is its transpose.  u is given
// in cluster order with the right-hand sides interleaved (u[i * nrhs + r]); v is written
// in solve order, column-major.
//
// Phase 1 (k_far_t): the rank vectors t_b = V_b^T u[c-range] and s_b = U_b^T u[r-range].
// Factor columns that contract over the same index range are stacked (up to 64 per task),
// so one CTA stages each piece of u once for all of them (cp.async, double buffered) and
// runs a register-tiled product (tile.cuh); t and s are stored interleaved like u.
// Phase 2 (k_far_y): one CTA per leaf accumulates, in the order of the leaf's list of
// covering far blocks, U_b t_b (row side), V_b s_b (column side), B u (dense row side) and
// B^T u (dense column side) for the leaf's rows; the host plan cuts the list into
// contraction segments of at most 32, which are staged in shared memory in chunks.  Each
// leaf's list is split into FAR_PARTS consecutive parts of about equal length, one CTA each
// (so that the uneven leaves spread over all SMs); k_far_sum adds the parts in order.  Every output sums its terms in
// one fixed order, so results are deterministic and do not depend on how many right-hand
// sides share the launch.
#include "cplx.cuh"
#include "hm_internal.h"
#include "tc.cuh"
#include "tile.cuh"

namespace hm {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

namespace {
constexpr int SEG = 64;   // longest staged contraction segment
}

// Phase 1: one CTA per task (a range [lo, hi) and up to 64 stacked factor columns).  The
// range is walked in pieces of FAR_T1 rows, each piece's factor rows and vector rows copied
// with cp.async into the two halves of shared memory in turn, so the copy of the next piece
// overlaps the product of the current; every output sums its rows in ascending order.
constexpr int FAR_T1 = 32;

template <class T> __device__ __forceinline__ void far_cp(T *dst, const T *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

template <class T, int TR, int TC, int NT>
__global__ void __launch_bounds__(256) k_far_t(const int *task_lo, const int *task_hi, const int *task_ptr,
                                               const int64_t *item_off, const int *item_ld, const int *item_rank,
                                               const int *item_row, const int *item_isv, const T *U, const T *V,
                                               const T *u, int nrhs, T *t, T *s, int budget)
{
    extern __shared__ unsigned char smraw[];
    __shared__ int s_item[64], s_l[64];
    __shared__ const T *s_src[64];
    __shared__ int s_R;
    const int task = blockIdx.x;
    const int lo = task_lo[task], hi = task_hi[task], i0 = task_ptr[task], i1 = task_ptr[task + 1];
    if (threadIdx.x == 0) {
        int R = 0;
        for (int it = i0; it < i1; ++it)
            for (int l = 0; l < item_rank[it] && R < 64; ++l, ++R) {
                s_item[R] = it;
                s_l[R] = l;
                s_src[R] = (item_isv[it] ? V : U) + item_off[it] + (int64_t)l * item_ld[it];
            }
        s_R = R;
    }
    __syncthreads();
    const int R = s_R;
    const int nrt = (R + TR - 1) / TR, ntiles = nrt * ((nrhs + TC - 1) / TC);
    const int ldw = stage_ldw(R, TR), ldr = stage_ldr(nrhs, TC);
    T *const bufs[2] = {(T *)smraw, (T *)smraw + budget / 2};
    Tile<T, TR, TC, NT> acc;
    tile_load(acc, (const T *)nullptr, 0, 0, R, nrhs, nrt, ntiles);
    // copy piece [c0, c0 + ch) into bufs[which]: Ws[qq*ldw + rr] = factor rr at row c0 + qq,
    // Ys[qq*ldr + r] = u[(c0 + qq) * nrhs + r]
    auto stage = [&](int c0, int which) {
        const int ch = min(FAR_T1, hi - c0);
        T *Ws = bufs[which], *Ys = bufs[which] + ch * ldw;
        for (int e = threadIdx.x; e < ch * R; e += blockDim.x) {
            const int qq = e % ch, rr = e / ch;
            far_cp(Ws + qq * ldw + rr, s_src[rr] + (c0 - lo + qq));
        }
        const T *uc = u + (int64_t)c0 * nrhs;
        for (int e = threadIdx.x; e < ch * nrhs; e += blockDim.x) far_cp(Ys + (e / nrhs) * ldr + e % nrhs, uc + e);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    if (lo < hi) stage(lo, 0);
    for (int c0 = lo, it = 0; c0 < hi; c0 += FAR_T1, ++it) {
        const int ch = min(FAR_T1, hi - c0);
        if (c0 + FAR_T1 < hi) {
            stage(c0 + FAR_T1, (it + 1) & 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        T *Ws = bufs[it & 1];
        tile_mac<false>(acc, Ws, ldw, Ws + ch * ldw, ldr, 1, ch, nrt, ntiles);
        __syncthreads();
    }
#pragma unroll
    for (int tt = 0; tt < NT; ++tt) {
        const TileRC m = tile_rc<TR, TC>(threadIdx.x + tt * blockDim.x, nrt, ntiles);
        const int row0 = m.row0, r0 = m.c0;
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int c = 0; c < TC; ++c)
                if (m.ok && row0 + a < R && r0 + c < nrhs) {
                    const int it = s_item[row0 + a];
                    T *dst = item_isv[it] ? t : s;
                    dst[(int64_t)(item_row[it] + s_l[row0 + a]) * nrhs + r0 + c] = acc.v[tt][a][c];
                }
    }
}

// Phase 2: one CTA per leaf over the leaf's segments (FarSegD, list order, len <= 32).
// Consecutive segments form a chunk while their summed length fits half the staging buffer;
// the chunk's coefficient rows and vector rows are stacked into one contraction, so a
// single tile product per chunk keeps every output's order (segment by segment, k
// ascending).  Chunks are copied with cp.async by one warp per segment into the two halves
// of the buffer in turn, so the copy of the next chunk overlaps the product of the current.
template <class T> __device__ __forceinline__ void cp_async_el(T *dst, const T *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <class T, int TR, int TC, int NT>
__global__ void __launch_bounds__(256) k_far_y(int nl, const int *leaf_ptr, const int *part_ptr, const int *kcum,
                                               const FarSegD *segs, const T *U, const T *V, const T *t, const T *s,
                                               const T *u, const int *cl2new, int n, int nrhs, T *part, int budget)
{
    extern __shared__ unsigned char smraw[];
    const int l = blockIdx.x / FAR_PARTS, pp = blockIdx.x % FAR_PARTS;
    if (l >= nl) return;
    const int a = leaf_ptr[l], ni = leaf_ptr[l + 1] - a;
    const int nrt = (ni + TR - 1) / TR, ntiles = nrt * ((nrhs + TC - 1) / TC);
    const int ldw = stage_ldw(ni, TR), ldr = stage_ldr(nrhs, TC);
    const int half = budget / 2, kmax = half / (ldw + ldr);   // >= 32 for ni <= 64
    T *const bufs[2] = {(T *)smraw, (T *)smraw + half};
    Tile<T, TR, TC, NT> acc;
    tile_load(acc, (const T *)nullptr, 0, 0, ni, nrhs, nrt, ntiles);
    const int w1 = part_ptr[blockIdx.x + 1];
    // segments [p, p + count) of the chunk starting at p: those whose stacked length fits kmax
    auto chunk_count = [&](int p) {
        const int q = p + threadIdx.x;
        const bool fit = q < w1 && kcum[q + 1] - kcum[p] <= kmax;
        return __syncthreads_count(fit);
    };
    // the chunk's stacked contraction rows kk = 0 .. klen-1 (segment q's rows kcum[p+q] - k0 ..)
    // copied by all threads: entry e of the coefficient rows is (kk, i) = (e / ni, e % ni), of
    // the vector rows (e / nrhs, e % nrhs); a thread's kk only grows, so it follows the segments
    // in order and reloads a segment's descriptor when it moves to the next
    auto stage = [&](int p, int cnt, T *buf) {
        const int k0 = kcum[p], klen = kcum[p + cnt] - k0;
        T *Wst = buf, *Yst = buf + kmax * ldw;
        int q = -1, qlo = 0, qhi = 0;
        const T *F = nullptr;
        int64_t fi = 0, fk = 0;
        for (int e = threadIdx.x; e < klen * ni; e += blockDim.x) {
            const int kk = e / ni, i = e - kk * ni;
            while (kk >= qhi) {
                ++q;
                qlo = kcum[p + q] - k0;
                qhi = kcum[p + q + 1] - k0;
                const FarSegD g = segs[p + q];
                F = ((g.src & 1) ? V : U) + g.foff;
                fi = g.fi;
                fk = g.fk;
            }
            cp_async_el(Wst + kk * ldw + i, F + (int64_t)i * fi + (int64_t)(kk - qlo) * fk);
        }
        q = -1;
        qhi = 0;
        const T *Yb = nullptr;
        for (int e = threadIdx.x; e < klen * nrhs; e += blockDim.x) {
            const int kk = e / nrhs, r = e - kk * nrhs;
            while (kk >= qhi) {
                ++q;
                qlo = kcum[p + q] - k0;
                qhi = kcum[p + q + 1] - k0;
                const FarSegD g = segs[p + q];
                const int ys = g.src >> 1;
                Yb = (ys == 0 ? t : (ys == 1 ? s : u)) + g.yrow * nrhs;
            }
            cp_async_el(Yst + kk * ldr + r, Yb + (int64_t)(kk - qlo) * nrhs + r);
        }
        cp_async_commit();
        return klen;
    };
    int p = part_ptr[blockIdx.x];
    if (p < w1) {
        int cnt = chunk_count(p), klen = stage(p, cnt, bufs[0]);
        for (int it = 0;; ++it) {
            const int pn = p + cnt;
            int cntn = 0, klenn = 0;
            if (pn < w1) {
                cntn = chunk_count(pn);
                klenn = stage(pn, cntn, bufs[(it + 1) & 1]);
                cp_async_wait<1>();
            } else
                cp_async_wait<0>();
            __syncthreads();
            T *buf = bufs[it & 1];
            tile_mac<false>(acc, buf, ldw, buf + kmax * ldw, ldr, 1, klen, nrt, ntiles);
            __syncthreads();
            if (pn >= w1) break;
            p = pn;
            cnt = cntn;
            klen = klenn;
        }
    }
    tile_store(acc, part + (size_t)pp * n * nrhs + cl2new[a], 1, n, ni, nrhs, nrt, ntiles);
}

// ---- complex FP32 on the tensor cores ------------------------------------------------------
// The same two phases with the block products on the tensor-core micro-kernel of tc.cuh
// (TF32 operands split into a rounded part and a remainder, FP32 accumulation in tensor
// memory), streamed in chunks of tc::KC2 contraction entries through a three-deep pipeline:
// the raw coefficient and vector entries of chunk c+1 are copied with cp.async while chunk c is
// split into one stage of operand planes and the MMAs of chunk c-1 run on the other stage.
// Fixed chunk order, so every output sums its terms in one order whatever the number of
// right-hand sides.
constexpr int FTC_LD = 64;                                   // raw[kk * FTC_LD + row or column]
constexpr int FTC_RAW = tc::KC2 * FTC_LD * 8;                // one raw buffer (8 KB)
constexpr int FTC_REGION = 2 * tc::STAGE2 + 4 * FTC_RAW;     // planes, then raw A and B x 2
constexpr unsigned long long FTC_WAIT_NS = 2000000000ull;
constexpr size_t FTC_SMEM = (FTC_REGION > tc::REGION_BYTES ? FTC_REGION : tc::REGION_BYTES) + 1024;

// Phase 1: task -> up to 64 factor columns (rows of the product) contracted over [lo, hi)
__global__ void __launch_bounds__(256, 2) k_far_t_tc(const int *task_lo, const int *task_hi, const int *task_ptr,
                                                     const int64_t *item_off, const int *item_ld,
                                                     const int *item_rank, const int *item_row, const int *item_isv,
                                                     const float2 *U, const float2 *V, const float2 *u, int nrhs,
                                                     float2 *t, float2 *s, int *err)
{
    extern __shared__ unsigned char smraw[];
    __shared__ int s_item[64], s_l[64];
    __shared__ const float2 *s_src[64];
    __shared__ int s_R;
    __shared__ uint64_t s_mbar[2];
    __shared__ uint32_t s_tmem;
    const int task = blockIdx.x;
    const int lo = task_lo[task], hi = task_hi[task], i0 = task_ptr[task], i1 = task_ptr[task + 1];
    if (threadIdx.x == 0) {
        int R = 0;
        for (int it = i0; it < i1; ++it)
            for (int l = 0; l < item_rank[it] && R < 64; ++l, ++R) {
                s_item[R] = it;
                s_l[R] = l;
                s_src[R] = (item_isv[it] ? V : U) + item_off[it] + (int64_t)l * item_ld[it];
            }
        s_R = R;
    }
    __syncthreads();
    const int R = s_R;
    if (R == 0) return;
    unsigned char *region = tc::align1024(smraw);
    float2 *rawA = (float2 *)(region + 2 * tc::STAGE2), *rawB = rawA + 2 * tc::KC2 * FTC_LD;
    tc::Acc2 acc;
    acc.planes = region;
    acc.mbar = s_mbar;
    acc.tslot = &s_tmem;
    acc.open(R, nrhs);
    const int nch = (hi - lo + tc::KC2 - 1) / tc::KC2;
    auto fetch = [&](int c) {   // raw entries of chunk c into raw buffer c & 1
        const int c0 = lo + c * tc::KC2, kl = min(tc::KC2, hi - c0), b = c & 1;
        float2 *ra = rawA + b * tc::KC2 * FTC_LD, *rb = rawB + b * tc::KC2 * FTC_LD;
        for (int e = threadIdx.x; e < kl * R; e += blockDim.x) {
            const int kk = e % kl, rr = e / kl;
            cp_async_el(ra + kk * FTC_LD + rr, s_src[rr] + (c0 - lo + kk));
        }
        const float2 *uc = u + (int64_t)c0 * nrhs;
        for (int e = threadIdx.x; e < kl * nrhs; e += blockDim.x) cp_async_el(rb + (e / nrhs) * FTC_LD + e % nrhs, uc + e);
        cp_async_commit();
    };
    if (nch > 0) fetch(0);
    for (int c = 0; c < nch; ++c) {
        const int st = c & 1, kl = min(tc::KC2, hi - (lo + c * tc::KC2));
        if (c + 1 < nch) {
            fetch(c + 1);
            cp_async_wait<1>();
        } else
            cp_async_wait<0>();
        __syncthreads();                       // chunk c's raw entries are visible
        acc.wait(st, err, FTC_WAIT_NS);        // the MMAs of chunk c - 2 have left stage st
        const float2 *ra = rawA + st * tc::KC2 * FTC_LD, *rb = rawB + st * tc::KC2 * FTC_LD;
        for (int e = threadIdx.x; e < acc.m8 * kl; e += blockDim.x) {
            const int r = e % acc.m8, kk = e / acc.m8;
            acc.put_a(st, r, kk, r < R ? ra[kk * FTC_LD + r] : make_float2(0.f, 0.f));
        }
        for (int e = threadIdx.x; e < acc.p * kl; e += blockDim.x) {
            const int col = e % acc.p, kk = e / acc.p;
            acc.put_b(st, col, kk, col < nrhs ? rb[kk * FTC_LD + col] : make_float2(0.f, 0.f));
        }
        acc.zero_pad(st, kl);
        acc.issue(st, kl);
    }
    acc.wait(0, err, FTC_WAIT_NS);
    acc.wait(1, err, FTC_WAIT_NS);
    float *dsm = (float *)region;
    const bool any = acc.drain(dsm);
    for (int e = threadIdx.x; e < R * nrhs; e += blockDim.x) {
        const int rr = e / nrhs, r = e % nrhs, it = s_item[rr];
        float2 *dst = item_isv[it] ? t : s;
        dst[(int64_t)(item_row[it] + s_l[rr]) * nrhs + r] = any ? acc.entry(dsm, rr, r) : make_float2(0.f, 0.f);
    }
    acc.close();
}

// Phase 2: CTA = (leaf, part); the part's segments streamed in chunks of tc::KC2 entries (a
// segment may be split between chunks)
struct FarTcChunk {
    const float2 *f[tc::KC2];   // coefficient entry kk of row i: f[kk][i * fi[kk]]
    int fi[tc::KC2];
    const float2 *y[tc::KC2];   // vector entry kk of column r: y[kk][r]
    int kl;
};

struct FarTcWalk {
    int q, koff;   // next segment and its first entry not yet taken
};

// thread 0: the next chunk of the part's segments [w.q, w1)
__device__ __forceinline__ void far_tc_chunk(FarTcWalk &w, int w1, const FarSegD *segs, const float2 *U,
                                             const float2 *V, const float2 *t, const float2 *s, const float2 *u,
                                             int nrhs, FarTcChunk &c)
{
    int kl = 0;
    while (w.q < w1 && kl < tc::KC2) {
        const FarSegD g = segs[w.q];
        const float2 *F = ((g.src & 1) ? V : U) + g.foff;
        const int ys = g.src >> 1;
        const float2 *Yb = (ys == 0 ? t : (ys == 1 ? s : u)) + g.yrow * nrhs;
        const int take = min(g.len - w.koff, tc::KC2 - kl);
        for (int k = 0; k < take; ++k) {
            const int kk = w.koff + k;
            c.f[kl + k] = F + (int64_t)kk * g.fk;
            c.fi[kl + k] = g.fi;
            c.y[kl + k] = Yb + (int64_t)kk * nrhs;
        }
        kl += take;
        w.koff += take;
        if (w.koff == g.len) {
            ++w.q;
            w.koff = 0;
        }
    }
    c.kl = kl;
}

__global__ void __launch_bounds__(256, 2) k_far_y_tc(int nl, const int *leaf_ptr, const int *part_ptr,
                                                     const int *kcum, const FarSegD *segs, const float2 *U,
                                                     const float2 *V, const float2 *t, const float2 *s,
                                                     const float2 *u, const int *cl2new, int n, int nrhs,
                                                     float2 *part, int *err)
{
    extern __shared__ unsigned char smraw[];
    __shared__ FarTcChunk s_ch[3];
    __shared__ uint64_t s_mbar[2];
    __shared__ uint32_t s_tmem;
    const int l = blockIdx.x / FAR_PARTS, pp = blockIdx.x % FAR_PARTS;
    if (l >= nl) return;
    const int a = leaf_ptr[l], ni = leaf_ptr[l + 1] - a;
    const int p0 = part_ptr[blockIdx.x], w1 = part_ptr[blockIdx.x + 1];
    float2 *out = part + (size_t)pp * n * nrhs + cl2new[a];
    if (p0 >= w1) {   // an empty part still contributes zeros to the sum
        for (int e = threadIdx.x; e < ni * nrhs; e += blockDim.x) out[e % ni + (int64_t)(e / ni) * n] = make_float2(0.f, 0.f);
        return;
    }
    unsigned char *region = tc::align1024(smraw);
    float2 *rawA = (float2 *)(region + 2 * tc::STAGE2), *rawB = rawA + 2 * tc::KC2 * FTC_LD;
    tc::Acc2 acc;
    acc.planes = region;
    acc.mbar = s_mbar;
    acc.tslot = &s_tmem;
    FarTcWalk w{p0, 0};
    if (threadIdx.x == 0) {
        far_tc_chunk(w, w1, segs, U, V, t, s, u, nrhs, s_ch[0]);
        far_tc_chunk(w, w1, segs, U, V, t, s, u, nrhs, s_ch[1]);
    }
    acc.open(ni, nrhs);   // synchronises: s_ch[0], s_ch[1] are visible
    (void)kcum;
    auto fetch = [&](int c) {
        const FarTcChunk &ch = s_ch[c % 3];
        const int b = c & 1;
        float2 *ra = rawA + b * tc::KC2 * FTC_LD, *rb = rawB + b * tc::KC2 * FTC_LD;
        for (int e = threadIdx.x; e < ch.kl * ni; e += blockDim.x) {
            const int i = e % ni, kk = e / ni;
            cp_async_el(ra + kk * FTC_LD + i, ch.f[kk] + (int64_t)i * ch.fi[kk]);
        }
        for (int e = threadIdx.x; e < ch.kl * nrhs; e += blockDim.x)
            cp_async_el(rb + (e / nrhs) * FTC_LD + e % nrhs, ch.y[e / nrhs] + e % nrhs);
        cp_async_commit();
    };
    fetch(0);
    for (int c = 0; s_ch[c % 3].kl > 0; ++c) {
        const int st = c & 1, kl = s_ch[c % 3].kl;
        const bool more = s_ch[(c + 1) % 3].kl > 0;
        if (more) {
            fetch(c + 1);
            cp_async_wait<1>();
        } else
            cp_async_wait<0>();
        __syncthreads();                       // chunk c's raw entries are visible
        // thread 0: the sources of chunk c + 2 (its buffer held chunk c - 1, no longer read)
        if (threadIdx.x == 0) far_tc_chunk(w, w1, segs, U, V, t, s, u, nrhs, s_ch[(c + 2) % 3]);
        acc.wait(st, err, FTC_WAIT_NS);        // the MMAs of chunk c - 2 have left stage st
        const float2 *ra = rawA + st * tc::KC2 * FTC_LD, *rb = rawB + st * tc::KC2 * FTC_LD;
        for (int e = threadIdx.x; e < acc.m8 * kl; e += blockDim.x) {
            const int r = e % acc.m8, kk = e / acc.m8;
            acc.put_a(st, r, kk, r < ni ? ra[kk * FTC_LD + r] : make_float2(0.f, 0.f));
        }
        for (int e = threadIdx.x; e < acc.p * kl; e += blockDim.x) {
            const int col = e % acc.p, kk = e / acc.p;
            acc.put_b(st, col, kk, col < nrhs ? rb[kk * FTC_LD + col] : make_float2(0.f, 0.f));
        }
        acc.zero_pad(st, kl);
        acc.issue(st, kl);                     // barrier inside: s_ch[(c + 2) % 3] is visible after it
    }
    acc.wait(0, err, FTC_WAIT_NS);
    acc.wait(1, err, FTC_WAIT_NS);
    float *dsm = (float *)region;
    const bool any = acc.drain(dsm);
    for (int e = threadIdx.x; e < ni * nrhs; e += blockDim.x) {
        const int i = e % ni, r = e / ni;
        out[i + (int64_t)r * n] = any ? acc.entry(dsm, i, r) : make_float2(0.f, 0.f);
    }
    acc.close();
}

// y = sum of the FAR_PARTS partial products, added in part order
template <class T> __global__ void k_far_sum(int64_t len, const T *part, T *y)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= len) return;
    T v = part[e];
    for (int p = 1; p < FAR_PARTS; ++p) {
        const T w = part[p * len + e];
        v.x += w.x;
        v.y += w.y;
    }
    y[e] = v;
}


namespace {
template <class T> struct FarLaunch {
    hm_ctx *h;
    const T *U, *V;
    T *t, *s;
    const T *ucl;
    T *y;
    int nrhs;
    template <int TR, int TC, int NT> cudaError_t run(int maxw)
    {
        const FarPlan &F = h->fplan;
        const int n = h->plan.n;
        const int budget = stage_need(64, SEG, nrhs, TR, TC);
        const size_t smem = sizeof(T) * (size_t)budget;
        static DeviceOnce attr;   // one per instantiation
        if (attr.need()) {
            const int smax = (int)(sizeof(T) * (size_t)stage_need(64, SEG, maxw, TR, TC));
            cudaError_t e;
            if ((e = cudaFuncSetAttribute(k_far_t<T, TR, TC, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax)) ||
                (e = cudaFuncSetAttribute(k_far_y<T, TR, TC, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax)))
                return e;
            attr.done();
        }
        const int ntask = (int)F.p1_lo.size();
        if (ntask > 0)
            HM_LAUNCH(h, K_FAR1,
                      (k_far_t<T, TR, TC, NT><<<ntask, 256, smem, h->stream>>>(
                          h->d_p1_lo, h->d_p1_hi, h->d_p1_ptr, h->d_p1_off, h->d_p1_ld, h->d_p1_rank, h->d_p1_row,
                          h->d_p1_isv, U, V, ucl, nrhs, t, s, budget)));
        T *part = (T *)h->d_farpart;
        HM_LAUNCH(h, K_FAR2,
                  (k_far_y<T, TR, TC, NT><<<h->nl * FAR_PARTS, 256, smem, h->stream>>>(
                      h->nl, h->d_leaf_ptr, h->d_part_ptr, h->d_seg_kcum, h->d_segs, U, V, t, s, ucl, h->d_cl2new,
                      n, nrhs, part, budget)));
        const int64_t len = (int64_t)n * nrhs;
        HM_LAUNCH(h, K_FAR2, k_far_sum<T><<<nblk(len, 256), 256, 0, h->stream>>>(len, part, y));
        return cudaGetLastError();
    }
};
}  // namespace

// complex FP32 on the tensor cores: phase 1, the phase-2 partial products, their sum
static cudaError_t far_tc_launch(hm_ctx *h, const float2 *U, const float2 *V, float2 *t, float2 *s,
                                 const float2 *ucl, float2 *y, int nrhs)
{
    const FarPlan &F = h->fplan;
    const int n = h->plan.n;
    static DeviceOnce attr;
    if (attr.need()) {
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_far_t_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FTC_SMEM)) ||
            (e = cudaFuncSetAttribute(k_far_y_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FTC_SMEM)))
            return e;
        attr.done();
    }
    const int ntask = (int)F.p1_lo.size();
    if (ntask > 0)
        HM_LAUNCH(h, K_FAR1,
                  (k_far_t_tc<<<ntask, 256, FTC_SMEM, h->stream>>>(h->d_p1_lo, h->d_p1_hi, h->d_p1_ptr, h->d_p1_off,
                                                                   h->d_p1_ld, h->d_p1_rank, h->d_p1_row, h->d_p1_isv,
                                                                   U, V, ucl, nrhs, t, s, h->d_err)));
    float2 *part = (float2 *)h->d_farpart;
    HM_LAUNCH(h, K_FAR2,
              (k_far_y_tc<<<h->nl * FAR_PARTS, 256, FTC_SMEM, h->stream>>>(
                  h->nl, h->d_leaf_ptr, h->d_part_ptr, h->d_seg_kcum, h->d_segs, U, V, t, s, ucl, h->d_cl2new, n, nrhs,
                  part, h->d_err)));
    const int64_t len = (int64_t)n * nrhs;
    HM_LAUNCH(h, K_FAR2, k_far_sum<float2><<<nblk(len, 256), 256, 0, h->stream>>>(len, part, y));
    return cudaGetLastError();
}

template <class T>
cudaError_t far_product(hm_ctx *h, const T *U, const T *V, T *t, T *s, const T *ucl, T *y, int nrhs)
{
    h->prof.cols[K_FAR1] += nrhs;
    h->prof.cols[K_FAR2] += nrhs;
    if constexpr (sizeof(T) == 8)
        if (h->far_kind == 2) return far_tc_launch(h, U, V, t, s, ucl, y, nrhs);
    FarLaunch<T> f{h, U, V, t, s, ucl, y, nrhs};
    return tile_dispatch<T>(nrhs, f);
}

template cudaError_t far_product<double2>(hm_ctx *, const double2 *, const double2 *, double2 *, double2 *,
                                          const double2 *, double2 *, int);
template cudaError_t far_product<float2>(hm_ctx *, const float2 *, const float2 *, float2 *, float2 *,
                                         const float2 *, float2 *, int);

}  // namespace hm
