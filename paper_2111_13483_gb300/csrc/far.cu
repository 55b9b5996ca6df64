// Far-field product v = Z_F u (Sec. 2 Eq. 9 blocks, Eq. 11), complex FP64 or FP32.
//
// Z_F is stored once per admissible pair (rows r-range, columns c-range, r before c): a
// low-rank block U V^T or a dense block B; the mirrored block is its transpose.  u is given
// in cluster order; v is written in solve order.
//
// Phase 1 (k_far_rank): one warp per (low-rank block b, rank column l) computes
//     t_b[l] = V_b[:, l]^T u[c-range],  s_b[l] = U_b[:, l]^T u[r-range]
// for a group of right-hand sides, loading each factor entry once per group.
// Phase 2 (k_far_gather): one CTA per leaf; its eight warps take the leaf's list of covering
// far blocks round robin (low-rank row side U_b t_b, column side V_b s_b, dense row side
// B u, dense column side B^T u), each warp accumulating partial sums for the leaf's rows,
// which are then added in warp order.  The arithmetic order is fixed, so results are
// deterministic and do not depend on how many right-hand sides share the launch.
#include "cplx.cuh"
#include "hm_internal.h"

namespace hm {

constexpr int FAR_RB = 8;    // right-hand sides per register group
constexpr int FAR_G = 8;     // warps (incidence groups) per leaf CTA

template <class T>
__global__ void __launch_bounds__(256) k_far_rank(int64_t tlen, const int *item_blk, const int64_t *toff,
                                                  const int *r0, const int *r1, const int *c0, const int *c1,
                                                  const int64_t *uoff, const int64_t *voff, const T *U, const T *V,
                                                  const T *u, int n, int nrhs, T *t, T *s)
{
    const int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (item >= tlen) return;
    const int b = item_blk[item];
    const int l = (int)(item - toff[b]);
    const int m = r1[b] - r0[b], nc = c1[b] - c0[b];
    const T *Vl = V + voff[b] + (int64_t)l * nc;
    const T *Ul = U + uoff[b] + (int64_t)l * m;
    for (int rb = 0; rb < nrhs; rb += FAR_RB) {
        const int nr = min(FAR_RB, nrhs - rb);
        const T *uc = u + c0[b] + (int64_t)rb * n, *ur = u + r0[b] + (int64_t)rb * n;
        T a1[FAR_RB], a2[FAR_RB];
#pragma unroll
        for (int q = 0; q < FAR_RB; ++q) a1[q] = a2[q] = czero(T());
        for (int i = lane; i < nc; i += 32) {
            const T v = Vl[i];
#pragma unroll
            for (int q = 0; q < FAR_RB; ++q)
                if (q < nr) a1[q] = cfma(v, uc[i + (int64_t)q * n], a1[q]);
        }
        for (int i = lane; i < m; i += 32) {
            const T v = Ul[i];
#pragma unroll
            for (int q = 0; q < FAR_RB; ++q)
                if (q < nr) a2[q] = cfma(v, ur[i + (int64_t)q * n], a2[q]);
        }
#pragma unroll
        for (int q = 0; q < FAR_RB; ++q) {
            if (q >= nr) break;
            T x1 = a1[q], x2 = a2[q];
            for (int w = 16; w > 0; w >>= 1) {
                x1.x += __shfl_xor_sync(0xffffffffu, x1.x, w);
                x1.y += __shfl_xor_sync(0xffffffffu, x1.y, w);
                x2.x += __shfl_xor_sync(0xffffffffu, x2.x, w);
                x2.y += __shfl_xor_sync(0xffffffffu, x2.y, w);
            }
            if (lane == 0) {
                t[item + (int64_t)(rb + q) * tlen] = x1;
                s[item + (int64_t)(rb + q) * tlen] = x2;
            }
        }
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_far_gather(int nl, const int *leaf_ptr, const int *lptr, const int *lent,
                                                    const int *r0, const int *r1, const int *c0, const int *c1,
                                                    const int *rank, const int64_t *uoff, const int64_t *voff,
                                                    const int64_t *toff, const T *U, const T *V, const T *t,
                                                    const T *s, const T *u, const int *cl2new, int n, int nrhs, T *y,
                                                    int64_t tlen)
{
    extern __shared__ unsigned char smraw[];
    T *part = (T *)smraw;                       // [FAR_G][64][FAR_RB]
    const int l = blockIdx.x;
    if (l >= nl) return;
    const int a = leaf_ptr[l], ni = leaf_ptr[l + 1] - a;
    const int on = cl2new[a];
    const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p0 = lptr[l], p1 = lptr[l + 1];
    for (int rb = 0; rb < nrhs; rb += FAR_RB) {
        const int nr = min(FAR_RB, nrhs - rb);
        for (int i0 = 0; i0 < ni; i0 += 32) {
            const int i = i0 + lane;
            const bool act = i < ni;
            T acc[FAR_RB];
#pragma unroll
            for (int q = 0; q < FAR_RB; ++q) acc[q] = czero(T());
            for (int p = p0 + g; p < p1; p += FAR_G) {
                const int ent = lent[p], b = ent >> 2, kind = ent & 3;
                const int m = r1[b] - r0[b], nc = c1[b] - c0[b];
                if (!act) continue;
                if (kind <= 1) {
                    const int rk = rank[b];
                    const int ld = kind == 0 ? m : nc;
                    const T *F = (kind == 0 ? U + uoff[b] + (a - r0[b]) : V + voff[b] + (a - c0[b])) + i;
                    const T *tb = (kind == 0 ? t : s) + toff[b] + (int64_t)rb * tlen;
                    for (int k = 0; k < rk; ++k) {
                        const T f = F[(int64_t)k * ld];
#pragma unroll
                        for (int q = 0; q < FAR_RB; ++q)
                            if (q < nr) acc[q] = cfma(f, tb[k + (int64_t)q * tlen], acc[q]);
                    }
                } else if (kind == 2) {
                    const T *B = U + uoff[b] + (a - r0[b]) + i;
                    const T *uc = u + c0[b] + (int64_t)rb * n;
                    for (int k = 0; k < nc; ++k) {
                        const T f = B[(int64_t)k * m];
#pragma unroll
                        for (int q = 0; q < FAR_RB; ++q)
                            if (q < nr) acc[q] = cfma(f, uc[k + (int64_t)q * n], acc[q]);
                    }
                } else {
                    const T *B = U + uoff[b] + (int64_t)((a - c0[b]) + i) * m;
                    const T *ur = u + r0[b] + (int64_t)rb * n;
                    for (int k = 0; k < m; ++k) {
                        const T f = B[k];
#pragma unroll
                        for (int q = 0; q < FAR_RB; ++q)
                            if (q < nr) acc[q] = cfma(f, ur[k + (int64_t)q * n], acc[q]);
                    }
                }
            }
            if (act) {
#pragma unroll
                for (int q = 0; q < FAR_RB; ++q) part[(g * 64 + i) * FAR_RB + q] = acc[q];
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < ni * nr; e += blockDim.x) {
            const int i = e % ni, q = e / ni;
            T v = part[i * FAR_RB + q];
            for (int gg = 1; gg < FAR_G; ++gg) {
                const T w = part[(gg * 64 + i) * FAR_RB + q];
                v.x += w.x;
                v.y += w.y;
            }
            y[on + i + (int64_t)(rb + q) * n] = v;
        }
        __syncthreads();
    }
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <class T>
cudaError_t far_product(hm_ctx *h, const T *U, const T *V, T *t, T *s, const T *ucl, T *y, int nrhs)
{
    const FarPlan &F = h->fplan;
    const int n = h->plan.n;
    const int smem = (int)(sizeof(T) * FAR_G * 64 * FAR_RB);
    static bool attr = false;   // one per instantiation
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_far_gather<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e) return e;
        attr = true;
    }
    if (F.nf > 0 && F.tlen > 0)
        HM_LAUNCH(h, K_FAR1,
                  k_far_rank<T><<<nblk(F.tlen * 32, 256), 256, 0, h->stream>>>(
                      F.tlen, h->d_far_item, h->d_far_toff, h->d_far_r0, h->d_far_r1, h->d_far_c0, h->d_far_c1,
                      h->d_far_uoff, h->d_far_voff, U, V, ucl, n, nrhs, t, s));
    HM_LAUNCH(h, K_FAR2,
              k_far_gather<T><<<h->nl, 32 * FAR_G, sizeof(T) * FAR_G * 64 * FAR_RB, h->stream>>>(
                  h->nl, h->d_leaf_ptr, h->d_flptr, h->d_flent, h->d_far_r0, h->d_far_r1, h->d_far_c0, h->d_far_c1,
                  h->d_far_rank, h->d_far_uoff, h->d_far_voff, h->d_far_toff, U, V, t, s, ucl, h->d_cl2new, n, nrhs,
                  y, F.tlen));
    return cudaGetLastError();
}

template cudaError_t far_product<double2>(hm_ctx *, const double2 *, const double2 *, double2 *, double2 *,
                                          const double2 *, double2 *, int);
template cudaError_t far_product<float2>(hm_ctx *, const float2 *, const float2 *, float2 *, float2 *,
                                         const float2 *, float2 *, int);

}  // namespace hm
