// Operator of the preconditioned system (Eq. 28) and restarted GMRES (Sec. 5) on the GPU.
//
//   A x~ = D^{-1} [ D x~ + L^{-1} Z_F L^{-T} x~ ],   c = D^{-1} L^{-1} b,   x = L^{-T} x~
//
// L^{-1} / L^{-T} are the products of the left / right scaling coefficients (Eqs. 20,
// 23, 24) applied as block-triangular sweeps over the coefficient panels W_k
// (L_jk = W_kj^T).  Each sweep is one sync-free launch: a CTA takes the next block from a
// ticket counter (so every block it waits on belongs to a CTA that is already running),
// gathers the finished blocks it depends on as their ready flags appear (bounded waits
// that report HM_ETIMEOUT instead of hanging), and publishes its own block with a flag.
// Z_F is applied in cluster order in two deterministic phases: rank vectors V^T u / U^T u
// per far block (a warp each), then one CTA per leaf summing every far block that covers
// it.  All vectors are complex FP64, column-major n x nrhs (ld n), solve order.
#include <cmath>
#include <cstdio>
#include <vector>

#include "hm_internal.h"

namespace hm {

namespace {

constexpr int ERR_TIMEOUT = 0x40000000;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // 2 s bound on any single wait

__device__ __forceinline__ double2 cfma_(double2 a, double2 b, double2 c)
{
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(a.y, b.x, c.y);
    return c;
}
__device__ __forceinline__ double2 cfms_(double2 a, double2 b, double2 c)
{
    // c - a*b
    c.x = fma(-a.x, b.x, c.x);
    c.x = fma(a.y, b.y, c.x);
    c.y = fma(-a.x, b.y, c.y);
    c.y = fma(-a.y, b.x, c.y);
    return c;
}
// conj(a) * b accumulated
__device__ __forceinline__ double2 cjfma_(double2 a, double2 b, double2 c)
{
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(-a.y, b.x, c.y);
    return c;
}

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One thread waits until flags[k] == epoch; returns false (and records ERR_TIMEOUT) when
// the bound expires or another CTA already failed.
__device__ bool wait_ready(const int *flags, int k, int epoch, int *err)
{
    const volatile int *f = flags + k;
    if (*f == epoch) {
        __threadfence();
        return true;
    }
    unsigned long long t0 = gtimer();
    while (*f != epoch) {
        if (*(volatile int *)err) return false;
        if (gtimer() - t0 > WAIT_NS) {
            atomicCAS(err, 0, ERR_TIMEOUT);
            return false;
        }
        __nanosleep(100);
    }
    __threadfence();
    return true;
}

__device__ __forceinline__ void publish(int *flags, int i, int epoch)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicExch(flags + i, epoch);
}

}  // namespace

// y = L^{-1} x : y_i = x_i - sum_{k < i, i in S_k} W_ki^T y_k   (Eq. 23, forward)
__global__ void __launch_bounds__(256) k_sweep_fwd(int nb, const int *size, const int *boff, const int *rptr,
                                                   const int *ridx, const int *rcol, const int64_t *coff,
                                                   const double2 *W, const double2 *x, double2 *y, int n, int nrhs,
                                                   int *flags, int epoch, int *ticket, int *err)
{
    extern __shared__ double2 sm[];
    __shared__ int s_i;
    if (threadIdx.x == 0) s_i = atomicAdd(ticket, 1);
    __syncthreads();
    const int i = s_i;
    if (i >= nb) return;
    const int ni = size[i], o = boff[i];
    double2 *acc = sm;                    // ni x nrhs
    double2 *vk = acc + 64 * nrhs;        // nk x nrhs
    double2 *wb = vk + 64 * nrhs;         // wb[q*65 + c] = W_ki[q, c]
    for (int e = threadIdx.x; e < ni * nrhs; e += blockDim.x) {
        int c = e % ni, r = e / ni;
        acc[e] = x[o + c + (int64_t)r * n];
    }
    for (int p = rptr[i]; p < rptr[i + 1]; ++p) {
        const int k = ridx[p], nk = size[k];
        const double2 *Wki = W + coff[k] + (int64_t)rcol[p] * nk;
        for (int e = threadIdx.x; e < nk * ni; e += blockDim.x) {
            int q = e % nk, c = e / nk;
            wb[q * 65 + c] = Wki[e];
        }
        if (threadIdx.x == 0) wait_ready(flags, k, epoch, err);
        __syncthreads();
        const int ok = boff[k];
        for (int e = threadIdx.x; e < nk * nrhs; e += blockDim.x) {
            int q = e % nk, r = e / nk;
            vk[e] = __ldcg(y + ok + q + (int64_t)r * n);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < ni * nrhs; e += blockDim.x) {
            int c = e % ni, r = e / ni;
            double2 s = acc[e];
            const double2 *v = vk + r * nk;
            for (int q = 0; q < nk; ++q) s = cfms_(wb[q * 65 + c], v[q], s);
            acc[e] = s;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < ni * nrhs; e += blockDim.x) {
        int c = e % ni, r = e / ni;
        y[o + c + (int64_t)r * n] = acc[e];
    }
    publish(flags, i, epoch);
}

// y = L^{-T} x : y_k = x_k - sum_{j in S_k} W_kj y_j   (Eq. 24, backward)
__global__ void __launch_bounds__(256) k_sweep_bwd(int nb, const int *size, const int *boff, const int *sptr,
                                                   const int *sidx, const int *srow, const int64_t *coff,
                                                   const double2 *W, const double2 *x, double2 *y, int n, int nrhs,
                                                   int *flags, int epoch, int *ticket, int *err)
{
    extern __shared__ double2 sm[];
    __shared__ int s_k;
    if (threadIdx.x == 0) s_k = nb - 1 - atomicAdd(ticket, 1);
    __syncthreads();
    const int k = s_k;
    if (k < 0) return;
    const int nk = size[k], o = boff[k];
    double2 *acc = sm;                    // nk x nrhs
    double2 *vj = acc + 64 * nrhs;        // nj x nrhs
    double2 *wb = vj + 64 * nrhs;         // wb[c*65 + row] = W_kj[row, c]
    for (int e = threadIdx.x; e < nk * nrhs; e += blockDim.x) {
        int rw = e % nk, r = e / nk;
        acc[e] = x[o + rw + (int64_t)r * n];
    }
    for (int p = sptr[k + 1] - 1; p >= sptr[k]; --p) {
        const int j = sidx[p], nj = size[j];
        const double2 *Wkj = W + coff[k] + (int64_t)srow[p] * nk;
        for (int e = threadIdx.x; e < nk * nj; e += blockDim.x) {
            int rw = e % nk, c = e / nk;
            wb[c * 65 + rw] = Wkj[e];
        }
        if (threadIdx.x == 0) wait_ready(flags, j, epoch, err);
        __syncthreads();
        const int oj = boff[j];
        for (int e = threadIdx.x; e < nj * nrhs; e += blockDim.x) {
            int c = e % nj, r = e / nj;
            vj[e] = __ldcg(y + oj + c + (int64_t)r * n);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nk * nrhs; e += blockDim.x) {
            int rw = e % nk, r = e / nk;
            double2 s = acc[e];
            const double2 *v = vj + r * nj;
            for (int c = 0; c < nj; ++c) s = cfms_(wb[c * 65 + rw], v[c], s);
            acc[e] = s;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nk * nrhs; e += blockDim.x) {
        int rw = e % nk, r = e / nk;
        y[o + rw + (int64_t)r * n] = acc[e];
    }
    publish(flags, k, epoch);
}

// dst[i + r*n] = src[idx[i] + r*n]
__global__ void k_gather(int n, int nrhs, const int *idx, const double2 *src, double2 *dst)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nrhs) return;
    int i = (int)(e % n), r = (int)(e / n);
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

// Far phase 1: per low-rank block, t_b = V^T u[c-range], s_b = U^T u[r-range] (one warp).
__global__ void __launch_bounds__(256) k_far1(int nf, const int *r0, const int *r1, const int *c0, const int *c1,
                                              const int *rank, const int64_t *uoff, const int64_t *voff,
                                              const int64_t *toff, const double2 *U, const double2 *V,
                                              const double2 *u, int n, int nrhs, double2 *t, double2 *s,
                                              int64_t tlen)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= nf) return;
    const int b = warp, rk = rank[b];
    if (rk <= 0) return;
    const int m = r1[b] - r0[b], nc = c1[b] - c0[b];
    const double2 *Ub = U + uoff[b], *Vb = V + voff[b];
    for (int r = 0; r < nrhs; ++r) {
        const double2 *uc = u + c0[b] + (int64_t)r * n, *ur = u + r0[b] + (int64_t)r * n;
        for (int l = 0; l < rk; ++l) {
            double2 a1 = make_double2(0, 0), a2 = make_double2(0, 0);
            for (int i = lane; i < nc; i += 32) a1 = cfma_(Vb[i + (int64_t)l * nc], uc[i], a1);
            for (int i = lane; i < m; i += 32) a2 = cfma_(Ub[i + (int64_t)l * m], ur[i], a2);
            for (int w = 16; w > 0; w >>= 1) {
                a1.x += __shfl_xor_sync(0xffffffffu, a1.x, w);
                a1.y += __shfl_xor_sync(0xffffffffu, a1.y, w);
                a2.x += __shfl_xor_sync(0xffffffffu, a2.x, w);
                a2.y += __shfl_xor_sync(0xffffffffu, a2.y, w);
            }
            if (lane == 0) {
                t[toff[b] + l + r * tlen] = a1;
                s[toff[b] + l + r * tlen] = a2;
            }
        }
    }
}

// Far phase 2: one CTA per leaf (cluster order) sums all far blocks covering its rows and
// writes the result at the leaf's solve-order position.
__global__ void __launch_bounds__(128) k_far2(int nl, const int *leaf_ptr, const int *lptr, const int *lent,
                                              const int *r0, const int *r1, const int *c0, const int *c1,
                                              const int *rank, const int64_t *uoff, const int64_t *voff,
                                              const int64_t *toff, const double2 *U, const double2 *V,
                                              const double2 *t, const double2 *s, const double2 *u,
                                              const int *cl2new, int n, int nrhs, double2 *y, int64_t tlen)
{
    const int l = blockIdx.x;
    if (l >= nl) return;
    const int a = leaf_ptr[l], ni = leaf_ptr[l + 1] - a;
    const int on = cl2new[a];
    for (int e = threadIdx.x; e < ni * nrhs; e += blockDim.x) {
        const int i = e % ni, r = e / ni;
        double2 acc = make_double2(0, 0);
        for (int p = lptr[l]; p < lptr[l + 1]; ++p) {
            const int ent = lent[p], b = ent >> 2, kind = ent & 3;
            const int m = r1[b] - r0[b], nc = c1[b] - c0[b];
            if (kind == 0) {
                const int rk = rank[b], off = a - r0[b];
                const double2 *Ub = U + uoff[b] + off + i;
                const double2 *tb = t + toff[b] + r * tlen;
                for (int q = 0; q < rk; ++q) acc = cfma_(Ub[(int64_t)q * m], tb[q], acc);
            } else if (kind == 1) {
                const int rk = rank[b], off = a - c0[b];
                const double2 *Vb = V + voff[b] + off + i;
                const double2 *sb = s + toff[b] + r * tlen;
                for (int q = 0; q < rk; ++q) acc = cfma_(Vb[(int64_t)q * nc], sb[q], acc);
            } else if (kind == 2) {
                const int off = a - r0[b];
                const double2 *B = U + uoff[b] + off + i;
                const double2 *uc = u + c0[b] + (int64_t)r * n;
                for (int q = 0; q < nc; ++q) acc = cfma_(B[(int64_t)q * m], uc[q], acc);
            } else {
                const int off = a - c0[b];
                const double2 *B = U + uoff[b] + (int64_t)(off + i) * m;
                const double2 *ur = u + r0[b] + (int64_t)r * n;
                for (int q = 0; q < m; ++q) acc = cfma_(B[q], ur[q], acc);
            }
        }
        y[on + i + (int64_t)r * n] = acc;
    }
}

// Block-diagonal operations (Eq. 28), one CTA per block:
//   mode 0: y = D^{-1} (D x + w);  mode 1: y = D^{-1} x;  mode 2: y = D x
__global__ void __launch_bounds__(256) k_diag(int mode, int nb, const int *size, const int *boff,
                                              const int64_t *doff, const double2 *D, const double2 *Dinv,
                                              const double2 *x, const double2 *w, double2 *y, int n, int nrhs)
{
    extern __shared__ double2 sm[];
    const int k = blockIdx.x;
    if (k >= nb) return;
    const int nk = size[k], o = boff[k];
    double2 *xs = sm, *ts = sm + 64 * nrhs;
    for (int e = threadIdx.x; e < nk * nrhs; e += blockDim.x) {
        int rw = e % nk, r = e / nk;
        xs[e] = x[o + rw + (int64_t)r * n];
    }
    __syncthreads();
    const double2 *Dk = D + doff[k], *Ik = Dinv + doff[k];
    if (mode == 0) {
        for (int e = threadIdx.x; e < nk * nrhs; e += blockDim.x) {
            int rw = e % nk, r = e / nk;
            double2 acc = w[o + rw + (int64_t)r * n];
            for (int c = 0; c < nk; ++c) acc = cfma_(Dk[rw + c * nk], xs[c + r * nk], acc);
            ts[e] = acc;
        }
        __syncthreads();
        xs = ts;
    }
    const double2 *Mk = (mode == 2) ? Dk : Ik;
    for (int e = threadIdx.x; e < nk * nrhs; e += blockDim.x) {
        int rw = e % nk, r = e / nk;
        double2 acc = make_double2(0, 0);
        for (int c = 0; c < nk; ++c) acc = cfma_(Mk[rw + c * nk], xs[c + r * nk], acc);
        y[o + rw + (int64_t)r * n] = acc;
    }
}

// Near-field product for the refinement residual: y += Z_N u, u in cluster order, y in
// solve order.  One CTA per leaf, summing near blocks (t, s) and mirrored (s, t) blocks.
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
                const double2 *us = u + leaf_ptr[s] + (int64_t)r * n;
                for (int c = 0; c < ms; ++c) acc = cfma_(B[i + (int64_t)c * mt], us[c], acc);
            } else {           // row l = s (t != s): sum_q B[q, i] u_t[q]
                const double2 *ut = u + leaf_ptr[t] + (int64_t)r * n;
                for (int q = 0; q < mt; ++q) acc = cfma_(B[q + (int64_t)i * mt], ut[q], acc);
            }
        }
        y[on + i + (int64_t)r * n] = acc;
    }
}

// ---- GMRES vector kernels (per batch column c, basis V_j at Vb + (j*nc + c)*n) -------
constexpr int DOT_CHUNK = 4096;

// part[((c*(J) + i) * nchunk + chunk)] = sum over chunk rows of conj(V_i) w, i < J
__global__ void __launch_bounds__(256) k_dots(int n, int nc, int J, const double2 *Vb, const double2 *w,
                                              double2 *part, int nchunk)
{
    __shared__ double2 red[8][33];
    const int chunk = blockIdx.x, c = blockIdx.y;
    const int lo = chunk * DOT_CHUNK, hi = min(n, lo + DOT_CHUNK);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const double2 *wc = w + (int64_t)c * n;
    for (int i0 = 0; i0 < J; i0 += 32) {
        const int ni = min(32, J - i0);
        double2 acc[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = make_double2(0, 0);
        for (int row = lo + threadIdx.x; row < hi; row += blockDim.x) {
            double2 wv = wc[row];
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (q < ni) acc[q] = cjfma_(Vb[((int64_t)(i0 + q) * nc + c) * n + row], wv, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            if (q >= ni) break;
            double2 v = acc[q];
            for (int o = 16; o > 0; o >>= 1) {
                v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
            }
            if (lane == 0) red[wp][q] = v;
        }
        __syncthreads();
        if (threadIdx.x < ni) {
            double2 v = make_double2(0, 0);
            for (int q = 0; q < 8; ++q) {
                v.x += red[q][threadIdx.x].x;
                v.y += red[q][threadIdx.x].y;
            }
            part[((int64_t)c * J + i0 + threadIdx.x) * nchunk + chunk] = v;
        }
        __syncthreads();
    }
}

// out[c*ldo + i] (+)= sum_chunk part  (fixed order; accumulate if add)
__global__ void k_dots_final(int nc, int J, int nchunk, const double2 *part, double2 *out, int ldo, int add)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nc * J) return;
    int c = e / J, i = e % J;
    double2 v = make_double2(0, 0);
    const double2 *p = part + (int64_t)e * nchunk;
    for (int q = 0; q < nchunk; ++q) {
        v.x += p[q].x;
        v.y += p[q].y;
    }
    double2 *o = out + (int64_t)c * ldo + i;
    if (add) {
        o->x += v.x;
        o->y += v.y;
    } else
        *o = v;
}

// w[:, c] -= sum_{i<J} h[c*ldh + i] V_i[:, c]
__global__ void k_axpy_basis(int n, int nc, int J, const double2 *Vb, const double2 *h, int ldh, double2 *w)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nc) return;
    int row = (int)(e % n), c = (int)(e / n);
    double2 acc = w[e];
    for (int i = 0; i < J; ++i) acc = cfms_(h[(int64_t)c * ldh + i], Vb[((int64_t)i * nc + c) * n + row], acc);
    w[e] = acc;
}

// x[:, c] += sum_{i<J[c]} y[c*ldy + i] V_i[:, c]
__global__ void k_update_x(int n, int nc, const int *J, const double2 *Vb, const double2 *yv, int ldy, double2 *x)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nc) return;
    int row = (int)(e % n), c = (int)(e / n);
    double2 acc = x[e];
    for (int i = 0; i < J[c]; ++i) acc = cfma_(yv[(int64_t)c * ldy + i], Vb[((int64_t)i * nc + c) * n + row], acc);
    x[e] = acc;
}

// v_out[:, c] = w[:, c] * (1 / nrm[c]) when nrm[c] > 0
__global__ void k_scale(int n, int nc, const double *nrm, const double2 *w, double2 *v)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nc) return;
    int c = (int)(e / n);
    double s = nrm[c] > 0 ? 1.0 / nrm[c] : 0.0;
    double2 a = w[e];
    v[e] = make_double2(a.x * s, a.y * s);
}

// r = c - r (in place on r)
__global__ void k_sub_from(int64_t len, const double2 *c, double2 *r)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= len) return;
    r[e] = make_double2(c[e].x - r[e].x, c[e].y - r[e].y);
}

__global__ void k_add_to(int64_t len, const double2 *a, double2 *x)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= len) return;
    x[e] = make_double2(x[e].x + a[e].x, x[e].y + a[e].y);
}

// GMRES small-matrix state per column c (H: (m+1) x m column-major, ld m+1)
struct GState {
    double2 *H, *g, *sn, *y, *hj;   // hj: current column scratch (m+1)
    double *cs, *nrm, *res, *wn;
    int *J, *active;
};

// Hessenberg column j for each active column: h[0..j] from hj, h[j+1] = nrm; previous
// rotations, new complex Givens rotation (real cosine), residual estimate |g_{j+1}|.
__global__ void k_givens(int nc, int m, int j, GState s, double tol_abs_scale_unused)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc || !s.active[c]) return;
    double2 *H = s.H + (int64_t)c * (m + 1) * m;
    double2 *hj = s.hj + (int64_t)c * (m + 1);
    double2 *g = s.g + (int64_t)c * (m + 1);
    double2 *sn = s.sn + (int64_t)c * m;
    double *cs = s.cs + (int64_t)c * m;
    double2 *col = H + (int64_t)j * (m + 1);
    for (int i = 0; i <= j; ++i) col[i] = hj[i];
    col[j + 1] = make_double2(s.nrm[c], 0.0);
    for (int i = 0; i < j; ++i) {
        double2 a = col[i], b = col[i + 1];
        double ci = cs[i];
        double2 si = sn[i];
        double2 t = make_double2(ci * a.x + (si.x * b.x - si.y * b.y), ci * a.y + (si.x * b.y + si.y * b.x));
        // -conj(s) a + c b
        double2 u = make_double2(-(si.x * a.x + si.y * a.y) + ci * b.x, -(si.x * a.y - si.y * a.x) + ci * b.y);
        col[i] = t;
        col[i + 1] = u;
    }
    double2 a = col[j], b = col[j + 1];
    double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
    double cj;
    double2 sj, rho;
    if (aa == 0.0) {
        cj = 0.0;
        sj = make_double2(1.0, 0.0);
        rho = b;
    } else {
        double r = hypot(aa, bb);
        cj = aa / r;
        double2 ph = make_double2(a.x / aa, a.y / aa);
        // s = ph * conj(b) / r
        sj = make_double2((ph.x * b.x + ph.y * b.y) / r, (ph.y * b.x - ph.x * b.y) / r);
        rho = make_double2(ph.x * r, ph.y * r);
    }
    cs[j] = cj;
    sn[j] = sj;
    col[j] = rho;
    col[j + 1] = make_double2(0, 0);
    double2 gj = g[j];
    // g_{j+1} = -conj(s) g_j ; g_j = c g_j
    g[j + 1] = make_double2(-(sj.x * gj.x + sj.y * gj.y), -(sj.x * gj.y - sj.y * gj.x));
    g[j] = make_double2(cj * gj.x, cj * gj.y);
    s.res[c] = hypot(g[j + 1].x, g[j + 1].y);
    s.J[c] = j + 1;
}

// y = H(1:J,1:J)^{-1} g(1:J) per column (back substitution)
__global__ void k_trisolve(int nc, int m, GState s)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const double2 *H = s.H + (int64_t)c * (m + 1) * m;
    const double2 *g = s.g + (int64_t)c * (m + 1);
    double2 *y = s.y + (int64_t)c * m;
    int J = s.J[c];
    for (int i = J - 1; i >= 0; --i) {
        double2 v = g[i];
        for (int q = i + 1; q < J; ++q) v = cfms_(H[i + (int64_t)q * (m + 1)], y[q], v);
        double2 d = H[i + (int64_t)i * (m + 1)];
        double den = d.x * d.x + d.y * d.y;
        y[i] = make_double2((v.x * d.x + v.y * d.y) / den, (v.y * d.x - v.x * d.y) / den);
    }
}

// ---- host side -------------------------------------------------------------------------
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

static cudaError_t sweep(hm_ctx *h, bool forward, const double2 *x, double2 *y, int nrhs)
{
    Plan &P = h->plan;
    cudaError_t e;
    if ((e = cudaMemsetAsync(h->d_ticket, 0, sizeof(int), h->stream))) return e;
    int ep = ++h->epoch;
    size_t smem = sizeof(double2) * (128 * nrhs + 64 * 65);
    if (forward)
        HM_LAUNCH(h, K_SWEEP_FWD, k_sweep_fwd<<<P.nb, 256, smem, h->stream>>>(P.nb, h->d_size, h->d_boff, h->d_rptr, h->d_ridx, h->d_rcol,
                                                     h->d_coff, h->d_W, x, y, P.n, nrhs, h->d_flags, ep,
                                                     h->d_ticket, h->d_err));
    else
        HM_LAUNCH(h, K_SWEEP_BWD, k_sweep_bwd<<<P.nb, 256, smem, h->stream>>>(P.nb, h->d_size, h->d_boff, h->d_sptr, h->d_sidx, h->d_srow,
                                                     h->d_coff, h->d_W, x, y, P.n, nrhs, h->d_flags, ep,
                                                     h->d_ticket, h->d_err));
    return cudaGetLastError();
}

// y (solve order) = Z_F x (solve order); uses work cols [0, nrhs) of d_work as u_cl
static cudaError_t far_apply(hm_ctx *h, const double2 *x, double2 *y, int nrhs, double2 *ucl)
{
    Plan &P = h->plan;
    FarPlan &F = h->fplan;
    const int n = P.n;
    // u_cl[i] = x[cl2new[i]]: cluster-order copy of the solve-order input
    HM_LAUNCH(h, K_PERMUTE, k_gather<<<nblk((int64_t)n * nrhs, 256), 256, 0, h->stream>>>(n, nrhs, h->d_cl2new, x, ucl));
    if (F.nf > 0 && F.tlen > 0)
        HM_LAUNCH(h, K_FAR1, k_far1<<<nblk((int64_t)F.nf * 32, 256), 256, 0, h->stream>>>(
            F.nf, h->d_far_r0, h->d_far_r1, h->d_far_c0, h->d_far_c1, h->d_far_rank, h->d_far_uoff, h->d_far_voff,
            h->d_far_toff, h->d_farU, h->d_farV, ucl, n, nrhs, h->d_t, h->d_s, F.tlen));
    HM_LAUNCH(h, K_FAR2, k_far2<<<h->nl, 128, 0, h->stream>>>(h->nl, h->d_leaf_ptr, h->d_flptr, h->d_flent, h->d_far_r0, h->d_far_r1,
                                         h->d_far_c0, h->d_far_c1, h->d_far_rank, h->d_far_uoff, h->d_far_voff,
                                         h->d_far_toff, h->d_farU, h->d_farV, h->d_t, h->d_s, ucl, h->d_cl2new, n,
                                         nrhs, y, F.tlen));
    return cudaGetLastError();
}

static cudaError_t diag(hm_ctx *h, int mode, const double2 *x, const double2 *w, double2 *y, int nrhs)
{
    Plan &P = h->plan;
    HM_LAUNCH(h, K_DIAG, k_diag<<<P.nb, 256, sizeof(double2) * 128 * nrhs, h->stream>>>(mode, P.nb, h->d_size, h->d_boff, h->d_doff,
                                                                    h->d_Ad, h->d_Dinv, x, w, y, P.n, nrhs));
    return cudaGetLastError();
}

cudaError_t ensure_solve_workspace(hm_ctx *h, int nrhs)
{
    cudaError_t e;
    const int n = h->plan.n;
    if (!h->d_flags) {
        if ((e = h->arena.alloc((void **)&h->d_flags, sizeof(int) * h->plan.nb))) return e;
        if ((e = cudaMemsetAsync(h->d_flags, 0, sizeof(int) * h->plan.nb, h->stream))) return e;
        h->epoch = 0;
    }
    if (h->t_cols < nrhs) {
        if (h->d_t) h->arena.release(h->d_t, 0), h->arena.release(h->d_s, 0);
        size_t len = std::max<int64_t>(1, h->fplan.tlen) * (size_t)nrhs;
        if ((e = h->arena.alloc((void **)&h->d_t, sizeof(double2) * len))) return e;
        if ((e = h->arena.alloc((void **)&h->d_s, sizeof(double2) * len))) return e;
        h->t_cols = nrhs;
    }
    if (h->work_cols < 3 * nrhs) {
        if (h->d_work) h->arena.release(h->d_work, 0);
        if ((e = h->arena.alloc((void **)&h->d_work, sizeof(double2) * (size_t)n * 3 * nrhs))) return e;
        h->work_cols = 3 * nrhs;
    }
    static bool attr = false;
    if (!attr) {
        int smax = (int)(sizeof(double2) * (128 * 64 + 64 * 65));
        cudaFuncSetAttribute(k_sweep_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        cudaFuncSetAttribute(k_sweep_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        cudaFuncSetAttribute(k_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double2) * 128 * 64));
        attr = true;
    }
    return cudaSuccess;
}

// y = Z x with x, y in the ORIGINAL RWG order (near blocks + far factors, FP64).
cudaError_t z_apply_orig(hm_ctx *h, const double2 *x, double2 *y, int nrhs)
{
    cudaError_t e;
    if ((e = ensure_solve_workspace(h, nrhs))) return e;
    const int n = h->plan.n;
    double2 *w0 = h->d_work, *w1 = h->d_work + (size_t)n * nrhs, *w2 = h->d_work + (size_t)2 * n * nrhs;
    HM_LAUNCH(h, K_PERMUTE, k_gather_cols<<<nblk((int64_t)n * nrhs, 256), 256, 0, h->stream>>>(n, nrhs, h->d_new2orig, x, n, w0));
    if ((e = far_apply(h, w0, w1, nrhs, w2))) return e;   // leaves the cluster-order copy in w2
    HM_LAUNCH(h, K_NEAR, k_near_mv<<<h->nl, 128, 0, h->stream>>>(h->nl, h->d_leaf_ptr, h->d_nptr, h->d_nent, h->d_near_t, h->d_near_s,
                                            h->d_near_off, h->d_near, w2, h->d_cl2new, n, nrhs, w1));
    HM_LAUNCH(h, K_PERMUTE, k_scatter_cols<<<nblk((int64_t)n * nrhs, 256), 256, 0, h->stream>>>(n, nrhs, h->d_new2orig, w1, y, n));
    return cudaGetLastError();
}

// op codes as in hm_apply; nrhs <= 64
cudaError_t op_apply(hm_ctx *h, int op, const double2 *x, double2 *y, int nrhs)
{
    cudaError_t e;
    if ((e = ensure_solve_workspace(h, nrhs))) return e;
    const int n = h->plan.n;
    double2 *w0 = h->d_work, *w1 = h->d_work + (size_t)n * nrhs, *w2 = h->d_work + (size_t)2 * n * nrhs;
    switch (op) {
    case 0:   // A x = D^{-1} [D x + L^{-1} Z_F L^{-T} x]
        if ((e = sweep(h, false, x, w0, nrhs))) return e;
        if ((e = far_apply(h, w0, w1, nrhs, w2))) return e;
        if ((e = sweep(h, true, w1, w0, nrhs))) return e;
        return diag(h, 0, x, w0, y, nrhs);
    case 1: return sweep(h, true, x, y, nrhs);
    case 2: return sweep(h, false, x, y, nrhs);
    case 3: return far_apply(h, x, y, nrhs, w2);
    case 4: return diag(h, 1, x, nullptr, y, nrhs);
    case 6: return diag(h, 2, x, nullptr, y, nrhs);
    default: return cudaErrorInvalidValue;
    }
}

// dst[c] = sqrt(max(0, Re src[c*lds]))
__global__ void k_sqrt_re(int nc, const double2 *src, int lds, double *dst)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nc) dst[c] = sqrt(fmax(0.0, src[(int64_t)c * lds].x));
}

// dst[c*ldd + i] += src[c*lds + i], i < J
__global__ void k_hfold(int nc, int J, const double2 *src, int lds, double2 *dst, int ldd)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nc * J) return;
    int c = e / J, i = e % J;
    dst[(int64_t)c * ldd + i].x += src[(int64_t)c * lds + i].x;
    dst[(int64_t)c * ldd + i].y += src[(int64_t)c * lds + i].y;
}

// Batched GMRES(m) on Eq. 28 for nc <= 64 columns in solve order: c (rhs), x (in/out).
// Arnoldi by classical Gram-Schmidt applied twice (CGS2; the oracle's modified
// Gram-Schmidt gives the same basis up to rounding).  One host synchronisation per
// Arnoldi step reads the residual estimates; columns that converge stop taking steps.
static int gmres_batch(hm_ctx *h, const double2 *cvec, double2 *x, int nc, double tol, int m, int maxit,
                       int *iters, double *relres)
{
    cudaStream_t st = h->stream;
    const int n = h->plan.n;
    const int nchunk = (n + DOT_CHUNK - 1) / DOT_CHUNK;
    cudaError_t e = cudaSuccess;
    std::vector<void *> allocs;
    auto A = [&](void **p, size_t bytes) {
        cudaError_t r = h->arena.alloc(p, bytes);
        if (r == cudaSuccess) allocs.push_back(*p);
        return r;
    };
    double2 *Vb, *w, *part, *hcol, *h2, *r;
    GState s{};
    if ((e = A((void **)&Vb, sizeof(double2) * (size_t)n * nc * (m + 1))) ||
        (e = A((void **)&w, sizeof(double2) * (size_t)n * nc)) ||
        (e = A((void **)&r, sizeof(double2) * (size_t)n * nc)) ||
        (e = A((void **)&part, sizeof(double2) * (size_t)nchunk * nc * (m + 1))) ||
        (e = A((void **)&hcol, sizeof(double2) * (size_t)nc * (m + 1))) ||
        (e = A((void **)&h2, sizeof(double2) * (size_t)nc * (m + 1))) ||
        (e = A((void **)&s.H, sizeof(double2) * (size_t)nc * (m + 1) * m)) ||
        (e = A((void **)&s.g, sizeof(double2) * (size_t)nc * (m + 1))) ||
        (e = A((void **)&s.sn, sizeof(double2) * (size_t)nc * m)) ||
        (e = A((void **)&s.y, sizeof(double2) * (size_t)nc * m)) ||
        (e = A((void **)&s.cs, sizeof(double) * (size_t)nc * m)) ||
        (e = A((void **)&s.nrm, sizeof(double) * nc)) || (e = A((void **)&s.res, sizeof(double) * nc)) ||
        (e = A((void **)&s.wn, sizeof(double) * nc)) || (e = A((void **)&s.J, sizeof(int) * nc)) ||
        (e = A((void **)&s.active, sizeof(int) * nc))) {
        for (void *p : allocs) h->arena.release(p, 0);
        h->err = "GMRES workspace allocation failed";
        return HM_ENOMEM;
    }
    s.hj = hcol;
    // ||v[:, c]|| for all columns -> out (device) and returned to the host
    auto norms = [&](const double2 *v, double *out) {
        HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, nc), 256, 0, st>>>(n, nc, 1, v, v, part, nchunk));
        HM_LAUNCH(h, K_SMALL, k_dots_final<<<nblk(nc, 128), 128, 0, st>>>(nc, 1, nchunk, part, h2, 1, 0));
        HM_LAUNCH(h, K_SMALL, k_sqrt_re<<<nblk(nc, 128), 128, 0, st>>>(nc, h2, 1, out));
        std::vector<double> nv(nc);
        cudaMemcpyAsync(nv.data(), out, sizeof(double) * nc, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        return nv;
    };
    std::vector<double> cn = norms(cvec, s.res);
    std::vector<int> conv(nc, 0), it(nc, 0);
    std::vector<double> rr(nc, 0.0);
    for (int c = 0; c < nc; ++c)
        if (cn[c] == 0.0) conv[c] = 1;
    int status = HM_OK;
    bool first = true;
    while (true) {
        // r = c - A x (x = 0 on the first cycle): the true residual at every restart
        if (first)
            cudaMemcpyAsync(r, cvec, sizeof(double2) * (size_t)n * nc, cudaMemcpyDeviceToDevice, st);
        else {
            if ((e = op_apply(h, 0, x, r, nc))) break;
            HM_LAUNCH(h, K_VEC, k_sub_from<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>((int64_t)n * nc, cvec, r));
        }
        first = false;
        std::vector<double> beta = norms(r, s.nrm);
        std::vector<int> act(nc, 0);
        bool any = false;
        for (int c = 0; c < nc; ++c) {
            if (conv[c]) continue;
            if (beta[c] <= tol * cn[c]) {
                conv[c] = 1;
                rr[c] = beta[c] / cn[c];
                continue;
            }
            if (it[c] >= maxit) {
                rr[c] = beta[c] / cn[c];
                continue;
            }
            act[c] = 1;
            any = true;
        }
        if (!any) break;
        cudaMemcpyAsync(s.active, act.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st);
        HM_LAUNCH(h, K_VEC, k_scale<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, s.nrm, r, Vb));   // V_0 = r / beta
        std::vector<double2> g0((size_t)nc * (m + 1), make_double2(0, 0));
        for (int c = 0; c < nc; ++c) g0[(size_t)c * (m + 1)] = make_double2(beta[c], 0);
        cudaMemcpyAsync(s.g, g0.data(), sizeof(double2) * g0.size(), cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(s.J, 0, sizeof(int) * nc, st);
        std::vector<int> done(nc, 0);
        for (int c = 0; c < nc; ++c) done[c] = !act[c];
        std::vector<double> res(nc), wpre(nc), wn(nc);
        for (int j = 0; j < m; ++j) {
            double2 *vj = Vb + (size_t)j * nc * n, *vj1 = Vb + (size_t)(j + 1) * nc * n;
            if ((e = op_apply(h, 0, vj, w, nc))) break;
            // ||w|| before orthogonalisation (happy-breakdown reference)
            HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, nc), 256, 0, st>>>(n, nc, 1, w, w, part, nchunk));
            HM_LAUNCH(h, K_SMALL, k_dots_final<<<nblk(nc, 128), 128, 0, st>>>(nc, 1, nchunk, part, h2, 1, 0));
            HM_LAUNCH(h, K_SMALL, k_sqrt_re<<<nblk(nc, 128), 128, 0, st>>>(nc, h2, 1, s.wn));
            // CGS2: h = V^H w, w -= V h, twice; h accumulated in hcol
            HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, nc), 256, 0, st>>>(n, nc, j + 1, Vb, w, part, nchunk));
            HM_LAUNCH(h, K_SMALL, k_dots_final<<<nblk(nc * (j + 1), 128), 128, 0, st>>>(nc, j + 1, nchunk, part, hcol, m + 1, 0));
            HM_LAUNCH(h, K_VEC, k_axpy_basis<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, j + 1, Vb, hcol, m + 1, w));
            HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, nc), 256, 0, st>>>(n, nc, j + 1, Vb, w, part, nchunk));
            HM_LAUNCH(h, K_SMALL, k_dots_final<<<nblk(nc * (j + 1), 128), 128, 0, st>>>(nc, j + 1, nchunk, part, h2, m + 1, 0));
            HM_LAUNCH(h, K_VEC, k_axpy_basis<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, j + 1, Vb, h2, m + 1, w));
            HM_LAUNCH(h, K_SMALL, k_hfold<<<nblk(nc * (j + 1), 128), 128, 0, st>>>(nc, j + 1, h2, m + 1, hcol, m + 1));
            // h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
            HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, nc), 256, 0, st>>>(n, nc, 1, w, w, part, nchunk));
            HM_LAUNCH(h, K_SMALL, k_dots_final<<<nblk(nc, 128), 128, 0, st>>>(nc, 1, nchunk, part, h2, 1, 0));
            HM_LAUNCH(h, K_SMALL, k_sqrt_re<<<nblk(nc, 128), 128, 0, st>>>(nc, h2, 1, s.nrm));
            HM_LAUNCH(h, K_VEC, k_scale<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, s.nrm, w, vj1));
            HM_LAUNCH(h, K_SMALL, k_givens<<<nblk(nc, 64), 64, 0, st>>>(nc, m, j, s, 0.0));
            cudaMemcpyAsync(res.data(), s.res, sizeof(double) * nc, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(wpre.data(), s.wn, sizeof(double) * nc, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(wn.data(), s.nrm, sizeof(double) * nc, cudaMemcpyDeviceToHost, st);
            if ((e = cudaStreamSynchronize(st))) break;
            bool all = true;
            std::vector<int> act2(nc, 0);
            for (int c = 0; c < nc; ++c) {
                if (done[c]) continue;
                it[c]++;
                bool brk = wn[c] <= 1e-14 * wpre[c];
                rr[c] = res[c] / cn[c];
                if (res[c] <= tol * cn[c] || brk) {
                    done[c] = 1;
                    conv[c] = 1;
                } else if (it[c] >= maxit)
                    done[c] = 1;
                if (!done[c]) {
                    all = false;
                    act2[c] = 1;
                }
            }
            if (all) break;
            cudaMemcpyAsync(s.active, act2.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st);
        }
        if (e) break;
        // x += V y per column (J[c] = steps of this cycle, 0 for columns that sat it out)
        HM_LAUNCH(h, K_SMALL, k_trisolve<<<nblk(nc, 64), 64, 0, st>>>(nc, m, s));
        HM_LAUNCH(h, K_VEC, k_update_x<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, s.J, Vb, s.y, m, x));
        if ((e = cudaStreamSynchronize(st))) break;
        bool all_done = true;
        for (int c = 0; c < nc; ++c)
            if (!conv[c] && it[c] < maxit) all_done = false;
        if (all_done) break;
    }
    for (void *p : allocs) h->arena.release(p, 0);
    if (e) {
        h->err = std::string("CUDA error in GMRES: ") + cudaGetErrorString(e);
        return HM_ECUDA;
    }
    int herr = 0;
    cudaMemcpy(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (herr & ERR_TIMEOUT) {
        h->err = "device-side wait in a triangular sweep timed out";
        return HM_ETIMEOUT;
    }
    for (int c = 0; c < nc; ++c) {
        iters[c] = it[c];
        relres[c] = rr[c];
        if (!conv[c]) status = HM_ENOCONV;
    }
    return status;
}

int gmres_solve(hm_ctx *h, const double2 *dV, int nrhs, int64_t ldv, double tol, int restart, int maxit, double2 *dI,
                int64_t ldi, int *iters, double *relres)
{
    const int n = h->plan.n;
    const int BATCH = 16;
    cudaStream_t st = h->stream;
    double2 *bnew = nullptr, *cvec = nullptr, *xt = nullptr;
    int status = HM_OK;
    cudaError_t e;
    const int nb = std::min(nrhs, BATCH);
    if ((e = h->arena.alloc((void **)&bnew, sizeof(double2) * (size_t)n * nb)) ||
        (e = h->arena.alloc((void **)&cvec, sizeof(double2) * (size_t)n * nb)) ||
        (e = h->arena.alloc((void **)&xt, sizeof(double2) * (size_t)n * nb))) {
        h->err = "solve workspace allocation failed";
        return HM_ENOMEM;
    }
    cudaMemsetAsync(h->d_err, 0, sizeof(int), st);
    for (int c0 = 0; c0 < nrhs && status != HM_ECUDA && status != HM_ETIMEOUT; c0 += BATCH) {
        const int nc = std::min(BATCH, nrhs - c0);
        // b (original order) -> solve order; c = D^{-1} L^{-1} b
        HM_LAUNCH(h, K_PERMUTE, k_gather_cols<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, h->d_new2orig, dV + c0 * ldv, ldv, bnew));
        if ((e = op_apply(h, 1, bnew, xt, nc)) || (e = op_apply(h, 4, xt, cvec, nc))) {
            status = HM_ECUDA;
            break;
        }
        cudaMemsetAsync(xt, 0, sizeof(double2) * (size_t)n * nc, st);
        int s = gmres_batch(h, cvec, xt, nc, tol, restart, maxit, iters + c0, relres + c0);
        if (s == HM_ECUDA || s == HM_ENOMEM || s == HM_ETIMEOUT) {
            status = s;
            break;
        }
        if (s == HM_ENOCONV) status = HM_ENOCONV;
        // x = L^{-T} x~ -> original order
        if ((e = op_apply(h, 2, xt, bnew, nc))) {
            status = HM_ECUDA;
            break;
        }
        HM_LAUNCH(h, K_PERMUTE, k_scatter_cols<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, h->d_new2orig, bnew, dI + c0 * ldi, ldi));
    }
    if (status != HM_ECUDA && (e = cudaStreamSynchronize(st))) status = HM_ECUDA;
    int herr = 0;
    cudaMemcpy(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (status == HM_OK && (herr & ERR_TIMEOUT)) {
        h->err = "device-side wait in a triangular sweep timed out";
        status = HM_ETIMEOUT;
    }
    if (status == HM_ECUDA && h->err.empty()) h->err = cudaGetErrorString(e);
    h->arena.release(bnew, 0);
    h->arena.release(cvec, 0);
    h->arena.release(xt, 0);
    return status;
}

}  // namespace hm
