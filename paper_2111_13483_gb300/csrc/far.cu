// Far-field product v = Z_F u (Sec. 2 Eq. 9 blocks, Eq. 11), complex FP64 or FP32.
//
// Z_F is stored once per admissible pair (rows r-range, columns c-range, r before c): a
// low-rank block U V^T or a dense block B; the mirrored block is its transpose.  u is given
// in cluster order with the right-hand sides interleaved (u[i * nrhs + r]); v is written
// in solve order, column-major.
//
// Phase 1 (k_far_t): the rank vectors t_b = V_b^T u[c-range] and s_b = U_b^T u[r-range].
// Factor columns that contract over the same index range are stacked (up to 64 per task),
// so one CTA stages each 64-row piece of u once for all of them and runs a register-tiled
// product (tile.cuh); t and s are stored interleaved like u.
// Phase 2 (k_far_y): one CTA per leaf accumulates, in the order of the leaf's list of
// covering far blocks, U_b t_b (row side), V_b s_b (column side), B u (dense row side) and
// B^T u (dense column side) for the leaf's rows; the list is cut into contraction segments
// of at most 64 that are staged in shared memory in chunks.  Every output sums its terms in
// one fixed order, so results are deterministic and do not depend on how many right-hand
// sides share the launch.
#include "cplx.cuh"
#include "hm_internal.h"
#include "tile.cuh"

namespace hm {

namespace {
constexpr int SEG = 64;   // longest staged contraction segment
}

template <class T, int TR, int TC, int NT>
__global__ void __launch_bounds__(256) k_far_t(const int *task_lo, const int *task_hi, const int *task_ptr,
                                               const int64_t *item_off, const int *item_ld, const int *item_rank,
                                               const int *item_row, const int *item_isv, const T *U, const T *V,
                                               const T *u, int nrhs, T *t, T *s)
{
    extern __shared__ unsigned char smraw[];
    T *buf = (T *)smraw;
    __shared__ int s_item[64], s_l[64];
    __shared__ int s_R;
    const int task = blockIdx.x;
    const int lo = task_lo[task], hi = task_hi[task], i0 = task_ptr[task], i1 = task_ptr[task + 1];
    if (threadIdx.x == 0) {
        int R = 0;
        for (int it = i0; it < i1; ++it)
            for (int l = 0; l < item_rank[it] && R < 64; ++l, ++R) {
                s_item[R] = it;
                s_l[R] = l;
            }
        s_R = R;
    }
    __syncthreads();
    const int R = s_R;
    const int nrt = (R + TR - 1) / TR, ntiles = nrt * ((nrhs + TC - 1) / TC);
    const int ldw = stage_ldw(R, TR), ldr = stage_ldr(nrhs, TC);
    Tile<T, TR, TC, NT> acc;
    tile_load(acc, (const T *)nullptr, 0, 0, R, nrhs, nrt, ntiles);
    for (int c0 = lo; c0 < hi; c0 += SEG) {
        const int ch = min(SEG, hi - c0);
        T *Ws = buf, *Ys = buf + ch * ldw;
        stage_copy(
            ch * R,
            [&](int e) {
                const int rr = e / ch, it = s_item[rr];
                return ((item_isv[it] ? V : U) + item_off[it] + (int64_t)s_l[rr] * item_ld[it])[c0 - lo + e % ch];
            },
            [&](int e, T v) { Ws[(e % ch) * ldw + e / ch] = v; });
        const T *uc = u + (int64_t)c0 * nrhs;
        stage_copy(ch * nrhs, [&](int e) { return uc[e]; }, [&](int e, T v) { Ys[(e / nrhs) * ldr + e % nrhs] = v; });
        __syncthreads();
        tile_mac<false>(acc, Ws, ldw, Ys, ldr, 1, ch, nrt, ntiles);
        __syncthreads();
    }
#pragma unroll
    for (int tt = 0; tt < NT; ++tt) {
        const int tile = threadIdx.x + tt * blockDim.x;
        const int row0 = (tile % nrt) * TR, r0 = (tile / nrt) * TC;
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int c = 0; c < TC; ++c)
                if (tile < ntiles && row0 + a < R && r0 + c < nrhs) {
                    const int it = s_item[row0 + a];
                    T *dst = item_isv[it] ? t : s;
                    dst[(int64_t)(item_row[it] + s_l[row0 + a]) * nrhs + r0 + c] = acc.v[tt][a][c];
                }
    }
}

// Contraction source of one incidence entry of leaf rows [a, a + ni): coefficient
// F(i, k) = Fb[i * fi + k * fk] and vector Y(k, r) = Yb[k * nrhs + r], k < K.
template <class T> struct FarSeg {
    const T *Fb, *Yb;
    int64_t fi, fk;
    int K;
};

template <class T>
__device__ __forceinline__ FarSeg<T> far_seg(int ent, int a, const int *r0, const int *r1, const int *c0,
                                             const int *c1, const int *rank, const int64_t *uoff,
                                             const int64_t *voff, const int64_t *toff, const T *U, const T *V,
                                             const T *t, const T *s, const T *u, int nrhs)
{
    const int b = ent >> 2, kind = ent & 3;
    const int m = r1[b] - r0[b], nc = c1[b] - c0[b];
    FarSeg<T> g;
    if (kind == 0) {          // low rank, leaf in the row range: U_b t_b
        g.Fb = U + uoff[b] + (a - r0[b]);
        g.fi = 1;
        g.fk = m;
        g.Yb = t + toff[b] * nrhs;
        g.K = rank[b];
    } else if (kind == 1) {   // low rank, leaf in the column range: V_b s_b
        g.Fb = V + voff[b] + (a - c0[b]);
        g.fi = 1;
        g.fk = nc;
        g.Yb = s + toff[b] * nrhs;
        g.K = rank[b];
    } else if (kind == 2) {   // dense, row side: B u[c-range]
        g.Fb = U + uoff[b] + (a - r0[b]);
        g.fi = 1;
        g.fk = m;
        g.Yb = u + (int64_t)c0[b] * nrhs;
        g.K = nc;
    } else {                  // dense, column side: B^T u[r-range]
        g.Fb = U + uoff[b] + (int64_t)(a - c0[b]) * m;
        g.fi = m;
        g.fk = 1;
        g.Yb = u + (int64_t)r0[b] * nrhs;
        g.K = m;
    }
    return g;
}

template <class T, int TR, int TC, int NT>
__global__ void __launch_bounds__(256) k_far_y(int nl, const int *leaf_ptr, const int *lptr, const int *lent,
                                               const int *r0, const int *r1, const int *c0, const int *c1,
                                               const int *rank, const int64_t *uoff, const int64_t *voff,
                                               const int64_t *toff, const T *U, const T *V, const T *t,
                                               const T *s, const T *u, const int *cl2new, int n, int nrhs, T *y,
                                               int budget)
{
    extern __shared__ unsigned char smraw[];
    T *buf = (T *)smraw;
    const int l = blockIdx.x;
    if (l >= nl) return;
    const int a = leaf_ptr[l], ni = leaf_ptr[l + 1] - a;
    const int nrt = (ni + TR - 1) / TR, ntiles = nrt * ((nrhs + TC - 1) / TC);
    const int ldw = stage_ldw(ni, TR), ldr = stage_ldr(nrhs, TC);
    Tile<T, TR, TC, NT> acc;
    tile_load(acc, (const T *)nullptr, 0, 0, ni, nrhs, nrt, ntiles);
    const int p1 = lptr[l + 1];
    int p = lptr[l], k0 = 0;
    while (p < p1) {
        // one chunk: segments (entry, [k0, k0 + len)) while they fit the budget
        int used = 0, pp = p, kk = k0;
        for (int nseg = 0; pp < p1 && nseg < 32;) {
            const FarSeg<T> g = far_seg(lent[pp], a, r0, r1, c0, c1, rank, uoff, voff, toff, U, V, t, s, u, nrhs);
            if (kk >= g.K) {   // entry done (or empty)
                ++pp;
                kk = 0;
                continue;
            }
            const int len = min(SEG, g.K - kk);
            const int need = stage_need(ni, len, nrhs, TR, TC);
            if (nseg > 0 && used + need > budget) break;
            T *Ws = buf + used, *Ys = Ws + len * ldw;
            if (g.fi == 1)
                stage_copy(len * ni, [&](int e) { return g.Fb[e % ni + (int64_t)(kk + e / ni) * g.fk]; },
                           [&](int e, T v) { Ws[(e / ni) * ldw + e % ni] = v; });
            else
                stage_copy(len * ni, [&](int e) { return g.Fb[(int64_t)(e / len) * g.fi + kk + e % len]; },
                           [&](int e, T v) { Ws[(e % len) * ldw + e / len] = v; });
            const T *yb = g.Yb + (int64_t)kk * nrhs;
            stage_copy(len * nrhs, [&](int e) { return yb[e]; },
                       [&](int e, T v) { Ys[(e / nrhs) * ldr + e % nrhs] = v; });
            used += need;
            ++nseg;
            kk += len;
        }
        __syncthreads();
        // replay the chunk's segments in order
        int off = 0;
        while (p != pp || k0 != kk) {
            const FarSeg<T> g = far_seg(lent[p], a, r0, r1, c0, c1, rank, uoff, voff, toff, U, V, t, s, u, nrhs);
            if (k0 >= g.K) {
                ++p;
                k0 = 0;
                continue;
            }
            const int len = min(SEG, g.K - k0);
            tile_mac<false>(acc, buf + off, ldw, buf + off + len * ldw, ldr, 1, len, nrt, ntiles);
            off += stage_need(ni, len, nrhs, TR, TC);
            k0 += len;
        }
        __syncthreads();
    }
    tile_store(acc, y + cl2new[a], 1, n, ni, nrhs, nrt, ntiles);
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

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
        static bool attr = false;   // one per instantiation
        if (!attr) {
            const int smax = (int)(sizeof(T) * (size_t)stage_need(64, SEG, maxw, TR, TC));
            cudaError_t e;
            if ((e = cudaFuncSetAttribute(k_far_t<T, TR, TC, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax)) ||
                (e = cudaFuncSetAttribute(k_far_y<T, TR, TC, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax)))
                return e;
            attr = true;
        }
        const int ntask = (int)F.p1_lo.size();
        if (ntask > 0)
            HM_LAUNCH(h, K_FAR1,
                      (k_far_t<T, TR, TC, NT><<<ntask, 256, smem, h->stream>>>(
                          h->d_p1_lo, h->d_p1_hi, h->d_p1_ptr, h->d_p1_off, h->d_p1_ld, h->d_p1_rank, h->d_p1_row,
                          h->d_p1_isv, U, V, ucl, nrhs, t, s)));
        HM_LAUNCH(h, K_FAR2,
                  (k_far_y<T, TR, TC, NT><<<h->nl, 256, smem, h->stream>>>(
                      h->nl, h->d_leaf_ptr, h->d_flptr, h->d_flent, h->d_far_r0, h->d_far_r1, h->d_far_c0,
                      h->d_far_c1, h->d_far_rank, h->d_far_uoff, h->d_far_voff, h->d_far_toff, U, V, t, s, ucl,
                      h->d_cl2new, n, nrhs, y, budget)));
        return cudaGetLastError();
    }
};
}  // namespace

template <class T>
cudaError_t far_product(hm_ctx *h, const T *U, const T *V, T *t, T *s, const T *ucl, T *y, int nrhs)
{
    FarLaunch<T> f{h, U, V, t, s, ucl, y, nrhs};
    return tile_dispatch<T>(nrhs, f);
}

template cudaError_t far_product<double2>(hm_ctx *, const double2 *, const double2 *, double2 *, double2 *,
                                          const double2 *, double2 *, int);
template cudaError_t far_product<float2>(hm_ctx *, const float2 *, const float2 *, float2 *, float2 *,
                                         const float2 *, float2 *, int);

}  // namespace hm
