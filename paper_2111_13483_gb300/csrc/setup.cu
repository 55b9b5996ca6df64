// Symmetric near-field Schur-complement setup (Sec. 3.1-3.2, Eqs. 12-21) on the GPU.
//
// Storage (solve order, blocks k = 0..nb-1 of n_k <= 64 unknowns):
//   Ad + doff[k]        A_kk, n_k x n_k; after the step it is D_k (Eq. 21);
//   A  + coff[k]        stacked column k: the blocks A_jk, j in S_k, one under the other,
//                       (M_k x n_k, ld M_k), the lower half of the symmetric near field
//                       plus its fill (scratch during setup);
//   W  + coff[k]        coefficient panel W_k = D_k^{-1} [A_kj]_{j in S_k} (n_k x M_k,
//                       ld n_k): W_kj = -alpha_kj of Eq. 14, the left coefficients being
//                       their transposes (Sec. 3.2);
//   Dinv + doff[k]      D_k^{-1} for the Eq. 28 preconditioner.
// Step k: pivot inverse (one CTA), panel (M_k/64 CTAs), Schur updates
// A_ij -= A_ik W_kj for i >= j in S_k (Eq. 19; diagonal blocks in full; one CTA per block
// pair in FP64, one CTA per row block and group of up to 8 column blocks in FP32).  Stream
// order gives the step dependencies.
//
// S is the storage and arithmetic type of A, the diagonal blocks and W: complex FP64, or
// complex FP32 in the mixed-precision setup, where the pivot blocks are still inverted in
// FP64 (their inverse is kept in FP64 and as an FP32 copy for the panels and the inner
// operator) and everything else stays FP32, so no step converts between the two.
#include <cstdio>

#include "cluster.cuh"
#include "cplx.cuh"
#include "hm_internal.h"
#include "tc.cuh"
#include "tile.cuh"

namespace hm {

// row offset of block i inside stacked column j (binary search in S_j); -1 if absent
__device__ __forceinline__ int find_row(const int *sptr, const int *sidx, const int *srow, int j, int i)
{
    int lo = sptr[j], hi = sptr[j + 1];
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = sidx[mid];
        if (v == i) return srow[mid];
        if (v < i) lo = mid + 1; else hi = mid;
    }
    return -1;
}

// Near-field blocks (cluster leaves t <= s) into the solve-order workspace.
template <class S>
__global__ void k_scatter_near(int n_near, const int *near_t, const int *near_s, const int64_t *near_off,
                               const double2 *near, const int *leaf_ptr, const int *pos, const int *sptr,
                               const int *sidx, const int *srow, const int *M, const int64_t *coff,
                               const int64_t *doff, S *A, S *Ad, int *err, bool diag_only = false)
{
    int b = blockIdx.x;
    if (b >= n_near) return;
    int t = near_t[b], s = near_s[b];
    if (diag_only && t != s) return;
    int m = leaf_ptr[t + 1] - leaf_ptr[t], n = leaf_ptr[s + 1] - leaf_ptr[s];
    const double2 *B = near + near_off[b];
    int i = pos[t], j = pos[s];
    S *dst;
    int ld;
    bool tr;
    if (i == j) {
        dst = Ad + doff[i];
        ld = m;
        tr = false;
    } else if (i > j) {
        int r = find_row(sptr, sidx, srow, j, i);
        if (r < 0) { atomicExch(err, 0x7fffffff); return; }
        dst = A + coff[j] + r;
        ld = M[j];
        tr = false;
    } else {
        int r = find_row(sptr, sidx, srow, i, j);
        if (r < 0) { atomicExch(err, 0x7fffffff); return; }
        dst = A + coff[i] + r;
        ld = M[i];
        tr = true;
    }
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
        int rr = e % m, cc = e / m;
        const S v = cconv<S>(B[e]);
        if (!tr) dst[rr + (int64_t)cc * ld] = v;
        else dst[cc + (int64_t)rr * ld] = v;
    }
}

// Pivot search of Gauss-Jordan step c by one warp over rows r >= c of column `col` of a
// (row-major, leading dimension ld): the largest |a_rc|^2, the lowest row on ties.  The
// squares are compared as the integer bit patterns of non-negative doubles (same order as
// the values), which keeps the compares off the slow FP64 pipe.  Lane 0 returns the row p,
// 1 / pivot in *d, and whether the pivot is singular (|pivot|^2 <= 1e-300 or not finite).
__device__ __forceinline__ int gj_pivot(const double2 *a, int ld, int col, int c, int n, double2 *d, bool *bad)
{
    const int lane = threadIdx.x & 31;
    unsigned long long best = 0;
    int bi = n;
    for (int r = c + lane; r < n; r += 32) {
        double2 v = a[r * ld + col];
        unsigned long long key = (unsigned long long)__double_as_longlong(fma(v.x, v.x, v.y * v.y));
        if (key > best || (key == best && r < bi) || bi == n) { best = key; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi < n && (ob > best || (ob == best && oi < bi) || bi == n)) { best = ob; bi = oi; }
    }
    const double pv = __longlong_as_double((long long)best);
    *bad = !(pv > 1e-300) || best >= 0x7ff0000000000000ull;
    const double2 pvv = a[bi * ld + col];
    *d = make_double2(pvv.x / pv, -pvv.y / pv);
    return bi;
}

// Entry (r, j) of Gauss-Jordan step c: row c takes the scaled pivot row rc; column c becomes
// -f d; every other entry cur - f rc (f = entry r of the pivot column after the interchange,
// d = 1 / pivot).  Both inverse kernels use these two functions, so their results agree bit
// for bit.
__device__ __forceinline__ double2 gj_row(double2 ap, double2 d, bool pivot_col) { return pivot_col ? d : cmul(ap, d); }
__device__ __forceinline__ double2 gj_entry(bool is_row, bool is_col, double2 rc, double2 f, double2 d, double2 cur)
{
    if (is_row) return rc;
    if (is_col) return make_double2(-(f.x * d.x - f.y * d.y), -(f.x * d.y + f.y * d.x));
    return make_double2(fma(-f.x, rc.x, fma(f.y, rc.y, cur.x)), fma(-f.x, rc.y, fma(-f.y, rc.x, cur.y)));
}

// In-place Gauss-Jordan inverse with partial pivoting (largest modulus, lowest row on
// ties) of D_k = Ad[k], in FP64 whatever S is; result to Dinv[k] (and its FP32 copy when
// Dinv32 is given).  err <- k+1 on a singular pivot.  Per column: one warp finds the pivot;
// one pass forms the scaled pivot row and the pivot column and moves the old row c into
// the pivot's row; one pass eliminates (four fused multiply-adds per entry) and writes the
// new row c.
template <class S>
__global__ void __launch_bounds__(256) k_pivot_inverse(int kbase, const int *size, const int64_t *doff, const S *Ad,
                                                       double2 *Dinv, float2 *Dinv32, int *err)
{
    const int k = kbase + blockIdx.x;   // one block per CTA (block Jacobi inverts all at once)
    extern __shared__ double2 sm[];
    const int n = size[k];
    const int ld = n + 1;                      // padded
    double2 *a = sm;                           // n x ld, row-major a[r*ld + c]
    double2 *rowc = sm + n * ld;               // n: pivot row after scaling
    double2 *colc = rowc + n;                  // n: pivot column (rows after the interchange)
    __shared__ int piv[64];
    __shared__ int s_p;
    __shared__ double2 s_d;
    const S *D = Ad + doff[k];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int r = e % n, c = e / n;
        a[r * ld + c] = cwiden(D[e]);
    }
    __syncthreads();
    for (int c = 0; c < n; ++c) {
        if (threadIdx.x < 32) {
            double2 d;
            bool bad;
            const int bi = gj_pivot(a, ld, c, c, n, &d, &bad);
            if (threadIdx.x == 0) {
                s_p = bi;
                piv[c] = bi;
                s_d = d;
                if (bad) atomicCAS(err, 0, k + 1);
            }
        }
        __syncthreads();
        const int p = s_p;
        const double2 d = s_d;
        // rows c and p interchanged: the new row c is the old row p
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const double2 ap = a[p * ld + j];
            rowc[j] = gj_row(ap, d, j == c);
            colc[j] = a[(j == p ? c : j) * ld + c];
            if (p != c) a[p * ld + j] = a[c * ld + j];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int r = e / n, j = e % n;
            a[r * ld + j] = gj_entry(r == c, j == c, rowc[j], colc[r], d, a[r * ld + j]);
        }
        __syncthreads();
    }
    // undo the row interchanges as column interchanges, last first
    for (int c = n - 1; c >= 0; --c) {
        int p = piv[c];
        if (p != c)
            for (int r = threadIdx.x; r < n; r += blockDim.x) {
                double2 t = a[r * ld + c];
                a[r * ld + c] = a[r * ld + p];
                a[r * ld + p] = t;
            }
        __syncthreads();
    }
    double2 *out = Dinv + doff[k];
    float2 *out32 = Dinv32 ? Dinv32 + doff[k] : nullptr;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int r = e % n, c = e / n;
        const double2 v = a[r * ld + c];
        out[e] = v;
        if (out32) out32[e] = make_float2((float)v.x, (float)v.y);
    }
}

// The same inverse on a cluster of CL CTAs (one block per cluster), so that the FP64 pipes of
// CL SMs share the elimination.  CTA q keeps the columns j = q, q + CL, ... of the in-place
// array (row-major, n x nloc).  Step c: the CTA that owns column c finds the pivot and
// stores p, 1 / pivot and the interchanged column c into every CTA of the cluster (two
// alternating buffers, distributed shared memory), then one cluster barrier; every CTA then
// interchanges, scales and eliminates its own columns with gj_row / gj_entry, entry for entry
// the operations of k_pivot_inverse, so the inverse is bitwise the same.  The row
// interchanges are undone by writing column x of the result from the column the interchanges
// moved there.  Every CTA takes all n + 1 cluster barriers (a CTA without columns too).
// Buffer b = c & 1 is rewritten at step c + 2 only after every CTA has passed the barrier of
// step c + 1, which it reaches after its elimination of step c.
template <class S, int CL>
__global__ void __launch_bounds__(128) k_pivot_inverse_cl(int kbase, const int *size, const int64_t *doff, const S *Ad,
                                                          double2 *Dinv, float2 *Dinv32, int *err)
{
    const int q = (int)cluster_rank();
    const int k = kbase + (int)(blockIdx.x / CL);
    extern __shared__ double2 sm[];
    const int n = size[k];
    const int nloc = (n - q + CL - 1) / CL;    // columns q, q + CL, ... below n
    const int ld = nloc + 1;
    double2 *a = sm;                           // n x ld, a[r * ld + jl] = column jl * CL + q
    double2 *rowc = sm + n * ld;               // nloc: the scaled pivot row
    __shared__ double2 s_col[2][64];           // pivot column after the interchange (pushed)
    __shared__ double2 s_d[2];                 // 1 / pivot (pushed)
    __shared__ int s_p[2];                     // pivot row (pushed)
    __shared__ int piv[64];
    __shared__ int at[64];
    const S *D = Ad + doff[k];
    for (int e = threadIdx.x; e < n * nloc; e += blockDim.x) {
        const int r = e % n, jl = e / n;
        a[r * ld + jl] = cwiden(D[r + (int64_t)(jl * CL + q) * n]);
    }
    cluster_sync();   // every CTA of the cluster is running before any remote store
    for (int c = 0; c < n; ++c) {
        const int b = c & 1;
        if (q == c % CL) {
            const int col = c / CL;
            __shared__ int o_p;
            __shared__ double2 o_d;
            if (threadIdx.x < 32) {
                double2 d;
                bool bad;
                const int bi = gj_pivot(a, ld, col, c, n, &d, &bad);
                if (threadIdx.x == 0) {
                    o_p = bi;
                    o_d = d;
                    if (bad) atomicCAS(err, 0, k + 1);
                }
            }
            __syncthreads();
            const int p = o_p;
            for (int x = threadIdx.x; x < CL * (n + 1); x += blockDim.x) {
                const int dst = x / (n + 1), r = x % (n + 1);
                if (r < n)
                    st_remote_d2(cluster_map(smem_addr(&s_col[b][r]), (unsigned)dst), a[(r == p ? c : r) * ld + col]);
                else {
                    st_remote_d2(cluster_map(smem_addr(&s_d[b]), (unsigned)dst), o_d);
                    st_remote_s32(cluster_map(smem_addr(&s_p[b]), (unsigned)dst), p);
                }
            }
        }
        cluster_sync();
        const int p = s_p[b];
        const double2 d = s_d[b];
        if (threadIdx.x == 0) piv[c] = p;
        for (int jl = threadIdx.x; jl < nloc; jl += blockDim.x) {
            const int j = jl * CL + q;
            rowc[jl] = gj_row(a[p * ld + jl], d, j == c);
            if (p != c) a[p * ld + jl] = a[c * ld + jl];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < n * nloc; e += blockDim.x) {
            const int r = e / nloc, jl = e % nloc;
            a[r * ld + jl] = gj_entry(r == c, jl * CL + q == c, rowc[jl], s_col[b][r], d, a[r * ld + jl]);
        }
        __syncthreads();
    }
    // at[x] = the column of the array that the interchanges (undone last first) move to x
    if (threadIdx.x == 0) {
        for (int x = 0; x < n; ++x) at[x] = x;
        for (int c = n - 1; c >= 0; --c) {
            const int t = at[c];
            at[c] = at[piv[c]];
            at[piv[c]] = t;
        }
    }
    __syncthreads();
    double2 *out = Dinv + doff[k];
    float2 *out32 = Dinv32 ? Dinv32 + doff[k] : nullptr;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e % n, x = e / n, src = at[x];
        if (src % CL != q) continue;
        const double2 v = a[r * ld + src / CL];
        out[e] = v;
        if (out32) out32[e] = make_float2((float)v.x, (float)v.y);
    }
}

// W_k[:, c0:c0+64] = D_k^{-1} (A_col_k[c0:c0+64, :])^T in S arithmetic
template <class S>
__global__ void __launch_bounds__(256) k_panel(int k, const int *size, const int *M, const int64_t *coff,
                                               const int64_t *doff, const S *Dinv, const S *A, S *W)
{
    extern __shared__ unsigned char psraw[];
    S *dinv = (S *)psraw;             // dinv[r*65 + q] = D_k^{-1}[r, q]
    S *ac = dinv + 64 * 65;           // ac[q*65 + col] = A_col[c0+col, q]
    const int n = size[k], Mk = M[k];
    const int c0 = blockIdx.x * 64;
    const int nc = min(64, Mk - c0);
    const S *Di = Dinv + doff[k];
    const S *Ac = A + coff[k];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int r = e % n, q = e / n;
        dinv[r * 65 + q] = Di[e];
    }
    for (int e = threadIdx.x; e < nc * n; e += blockDim.x) {
        int col = e % nc, q = e / nc;
        ac[q * 65 + col] = Ac[(c0 + col) + (int64_t)q * Mk];
    }
    __syncthreads();
    S *Wk = W + coff[k];
    for (int e = threadIdx.x; e < n * nc; e += blockDim.x) {
        int r = e % n, col = e / n;
        S acc = czero(S());
        for (int q = 0; q < n; ++q) acc = cfma(dinv[r * 65 + q], ac[q * 65 + col], acc);
        Wk[r + (int64_t)(c0 + col) * n] = acc;
    }
}

// Schur updates of step k (Eq. 19), FP64 setup: one CTA per pair (a >= b) of S_k,
// A_ij -= A_ik W_kj, in S arithmetic (the FP32 setup uses k_update_grp below).  C (ni x nj) -= A (ni x nk) W (nk x nj) on a 16U x 16U tile: thread
// (tx, ty) owns rows tx + 16u and columns ty + 16v (u, v < U).  The shared tiles are
// zero-padded to the tile size, so every thread runs the same unpredicated FMA sequence;
// padded outputs are dropped.
template <class S, int QC, int U>
__device__ __forceinline__ void update_tile(S (*As)[65], S (*Ws)[65], const S *Aik, int Mk, const S *Wkj, int nk,
                                            int ni, int nj, S *C, int ldc)
{
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    constexpr int TS = 16 * U;
    S acc[U][U];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v] = czero(S());
    for (int q0 = 0; q0 < nk; q0 += QC) {
        const int nq = min(QC, nk - q0);
        stage_copy<4>(
            TS * nq, [&](int e) { return e % TS < ni ? Aik[e % TS + (int64_t)(q0 + e / TS) * Mk] : czero(S()); },
            [&](int e, S v) { As[e / TS][e % TS] = v; });
        stage_copy<4>(
            nq * TS, [&](int e) { return e / nq < nj ? Wkj[(q0 + e % nq) + (int64_t)(e / nq) * nk] : czero(S()); },
            [&](int e, S v) { Ws[e % nq][e / nq] = v; });
        __syncthreads();
        for (int q = 0; q < nq; ++q) {
            S av[U], wv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) av[u] = As[q][tx + 16 * u];
#pragma unroll
            for (int v = 0; v < U; ++v) wv[v] = Ws[q][ty + 16 * v];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int v = 0; v < U; ++v) acc[u][v] = cfma(av[u], wv[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) {
            const int r = tx + 16 * u, c = ty + 16 * v;
            if (r < ni && c < nj) {
                S *p = C + r + (int64_t)c * ldc;
                S o = *p;
                o.x -= acc[u][v].x;
                o.y -= acc[u][v].y;
                *p = o;
            }
        }
}

template <class S>
__global__ void __launch_bounds__(256) k_update(int k, int ns, const int *size, const int *sptr, const int *sidx,
                                                const int *srow, const int *M, const int64_t *coff,
                                                const int64_t *doff, const S *W, S *A, S *Ad)
{
    constexpr int QC = sizeof(S) == 16 ? 16 : 32;
    __shared__ S As[QC][65];   // As[q][r] = A_ik[r, q0+q]
    __shared__ S Ws[QC][65];   // Ws[q][c] = W_kj[q0+q, c]
    // triangular index -> (a, b), a >= b (integer arithmetic only)
    const long t = blockIdx.x;
    int a = (int)sqrtf(2.0f * (float)t);
    while ((long)(a + 1) * (a + 2) / 2 <= t) ++a;
    while ((long)a * (a + 1) / 2 > t) --a;
    int b = (int)(t - (long)a * (a + 1) / 2);
    if (a >= ns) return;
    const int e0 = sptr[k];
    const int i = sidx[e0 + a], j = sidx[e0 + b];
    const int nk = size[k], ni = size[i], nj = size[j];
    const int Mk = M[k];
    const S *Aik = A + coff[k] + srow[e0 + a];                 // ld Mk
    const S *Wkj = W + coff[k] + (int64_t)srow[e0 + b] * nk;   // ld nk
    S *C;
    int ldc;
    if (i == j) {
        C = Ad + doff[i];
        ldc = ni;
    } else {
        int r = find_row(sptr, sidx, srow, j, i);
        if (r < 0) return;   // cannot happen when S is the symbolic fill (i in S_j)
        C = A + coff[j] + r;
        ldc = M[j];
    }
    if (ni <= 32 && nj <= 32)
        update_tile<S, QC, 2>(As, Ws, Aik, Mk, Wkj, nk, ni, nj, C, ldc);
    else
        update_tile<S, QC, 4>(As, Ws, Aik, Mk, Wkj, nk, ni, nj, C, ldc);
}

// Grouped Schur updates of step k for the complex-FP32 setup.  CTA -> (a, g): row block a
// of S_k and the column blocks b = g*gb .. min(a, g*gb + gb - 1).  For each, C_ij -= A_ik W_kj
// with the thread layout and q order of update_tile, so the result is bitwise that of
// k_update, on a tile fitted to the block in steps of 16 rows and columns (update_tile pads
// to 32 x 32 or 64 x 64: up to 5x the useful FMAs for uneven pairs).  A_ik is staged once
// per CTA, the W_kj blocks stream through two cp.async buffers (the copy of the next overlaps
// the product of the current) and each C block's old values are loaded before its product,
// so their latency hides behind the FMAs.
constexpr int UPD_LD = 65;
constexpr size_t UPD_SMEM = sizeof(float2) * 3 * 64 * UPD_LD;   // A_ik + two W_kj buffers

// CTAs of the rows a' < a: sum over m = 1..a of ceil(m / gb)
__host__ __device__ __forceinline__ long upd_first(int a, int gb)
{
    const long q = a / gb, r = a % gb;
    return (long)gb * q * (q + 1) / 2 + r * (q + 1);
}

__device__ __forceinline__ void upd_cp(float2 *dst, const float2 *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// C (ni x nj) -= A W on a (16 UR) x (16 UC) tile, UR = ceil(ni / 16), UC = ceil(nj / 16):
// thread (tx, ty) owns rows tx + 16u and columns ty + 16v, as in update_tile.
template <int UR, int UC>
__device__ __forceinline__ void upd_product(const float2 (*As)[UPD_LD], const float2 (*Ws)[UPD_LD], int nk, int ni,
                                            int nj, float2 *C, int ldc)
{
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float2 old[UR][UC], acc[UR][UC];
#pragma unroll
    for (int u = 0; u < UR; ++u)
#pragma unroll
        for (int v = 0; v < UC; ++v) {
            const int r = tx + 16 * u, c = ty + 16 * v;
            old[u][v] = (r < ni && c < nj) ? C[r + (int64_t)c * ldc] : czero(float2());
            acc[u][v] = czero(float2());
        }
    for (int q = 0; q < nk; ++q) {
        float2 av[UR], wv[UC];
#pragma unroll
        for (int u = 0; u < UR; ++u) av[u] = As[q][tx + 16 * u];
#pragma unroll
        for (int v = 0; v < UC; ++v) wv[v] = Ws[q][ty + 16 * v];
#pragma unroll
        for (int u = 0; u < UR; ++u)
#pragma unroll
            for (int v = 0; v < UC; ++v) acc[u][v] = cfma(av[u], wv[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < UR; ++u)
#pragma unroll
        for (int v = 0; v < UC; ++v) {
            const int r = tx + 16 * u, c = ty + 16 * v;
            if (r < ni && c < nj) {
                float2 o = old[u][v];
                o.x -= acc[u][v].x;
                o.y -= acc[u][v].y;
                C[r + (int64_t)c * ldc] = o;
            }
        }
}

__global__ void __launch_bounds__(256, 2) k_update_grp(int k, int ns, int gb, const int *size, const int *sptr,
                                                       const int *sidx, const int *srow, const int *M,
                                                       const int64_t *coff, const int64_t *doff, const float2 *W,
                                                       float2 *A, float2 *Ad)
{
    extern __shared__ float2 upd_sm[];
    float2(*As)[UPD_LD] = (float2(*)[UPD_LD])upd_sm;   // As[q][r] = A_ik[r, q], rows >= n_i zero
    // W buffer w: Ws[q][c] = W_kj[q, c], columns >= n_j zero up to the tile size
    auto wbuf = [&](int w) { return (float2(*)[UPD_LD])(upd_sm + (1 + w) * 64 * UPD_LD); };
    const long t = blockIdx.x;
    int lo = 0, hi = ns;   // largest a with upd_first(a) <= t
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (upd_first(mid, gb) <= t) lo = mid;
        else hi = mid;
    }
    const int a = lo, b0 = (int)(t - upd_first(a, gb)) * gb, b1 = min(a + 1, b0 + gb);
    if (b0 > a) return;   // cannot happen: row a has ceil((a + 1) / gb) groups
    const int e0 = sptr[k], i = sidx[e0 + a], nk = size[k], ni = size[i], Mk = M[k];
    const float2 *Aik = A + coff[k] + srow[e0 + a];   // ld Mk; panel k is not written in this step
    for (int e = threadIdx.x; e < 64 * nk; e += blockDim.x) {
        const int r = e & 63, q = e >> 6;
        if (r < ni) upd_cp(&As[q][r], Aik + r + (int64_t)q * Mk);
        else As[q][r] = czero(float2());
    }
    auto stage_w = [&](int b, int buf) {
        const int nj = size[sidx[e0 + b]];
        const float2 *Wkj = W + coff[k] + (int64_t)srow[e0 + b] * nk;   // ld nk
        const int ts = (nj + 15) / 16 * 16;
        float2(*Ws)[UPD_LD] = wbuf(buf);
        for (int e = threadIdx.x; e < nk * ts; e += blockDim.x) {
            const int q = e % nk, c = e / nk;
            if (c < nj) upd_cp(&Ws[q][c], Wkj + q + (int64_t)c * nk);
            else Ws[q][c] = czero(float2());
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    stage_w(b0, 0);   // one group with the A_ik copies
    for (int b = b0, it = 0; b < b1; ++b, ++it) {
        if (b + 1 < b1) {
            stage_w(b + 1, (it + 1) & 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        const int j = sidx[e0 + b], nj = size[j];
        float2 *C = nullptr;
        int ldc = 0;
        if (i == j) {
            C = Ad + doff[i];
            ldc = ni;
        } else {
            const int r = find_row(sptr, sidx, srow, j, i);   // >= 0 when S is the symbolic fill
            if (r >= 0) {
                C = A + coff[j] + r;
                ldc = M[j];
            }
        }
        if (C) {
            const float2(*Ws)[UPD_LD] = wbuf(it & 1);
            switch (((ni - 1) >> 4) * 4 + ((nj - 1) >> 4)) {   // (UR - 1) * 4 + (UC - 1)
#define HM_UPD(R, C_) \
    case (R - 1) * 4 + (C_ - 1): upd_product<R, C_>(As, Ws, nk, ni, nj, C, ldc); break;
                HM_UPD(1, 1) HM_UPD(1, 2) HM_UPD(1, 3) HM_UPD(1, 4)
                HM_UPD(2, 1) HM_UPD(2, 2) HM_UPD(2, 3) HM_UPD(2, 4)
                HM_UPD(3, 1) HM_UPD(3, 2) HM_UPD(3, 3) HM_UPD(3, 4)
                HM_UPD(4, 1) HM_UPD(4, 2) HM_UPD(4, 3) HM_UPD(4, 4)
#undef HM_UPD
            default: break;   // block sizes are 1..64
            }
        }
        __syncthreads();   // the buffer is restaged two products later
    }
}

// Schur updates of step k on the tensor cores (complex-FP32 setup, update kind 2).  The step's
// products are one lower-triangular product of the stacked column [A_ik; i in S_k] (M_k x n_k)
// with the panel W_k (n_k x M_k): CTA t takes row block a of S_k (i = S_k[a], n_i rows) and 64
// consecutive columns of W_k among those of blocks b <= a (tasks of row a: ceil((srow_a + n_i) /
// 64), ucum[e0 + a] the tasks before row a).  C = A_ik W_k[:, c0 : c0 + nc] runs as tcgen05
// MMAs on 3xTF32 operands (tc::Acc, chunks of tc::KC along n_k); every output column is then
// subtracted from its block A_ij (j = the S_k block holding the column; the diagonal block in Ad
// when j = i).  Each output adds its n_k terms in one fixed order.
__global__ void __launch_bounds__(256) k_update_tc(int k, int ns, const int *ucum, const int *size, const int *sptr,
                                                   const int *sidx, const int *srow, const int *M, const int64_t *coff,
                                                   const int64_t *doff, const float2 *W, float2 *A, float2 *Ad,
                                                   int *err, unsigned long long bound)
{
    extern __shared__ unsigned char smraw[];
    __shared__ uint64_t s_mbar;
    __shared__ uint32_t s_tslot;
    __shared__ float2 *s_col[64];
    const int e0 = sptr[k], t = blockIdx.x;
    int lo = 0, hi = ns;   // row a: the largest with ucum[e0 + a] <= t
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ucum[e0 + mid] <= t) lo = mid;
        else hi = mid;
    }
    const int a = lo, i = sidx[e0 + a], ni = size[i], nk = size[k], Mk = M[k];
    const int c0 = (t - ucum[e0 + a]) * 64, nc = min(64, srow[e0 + a] + ni - c0);
    if (threadIdx.x < nc) {   // where output column c0 + x goes
        const int c = c0 + threadIdx.x;
        int l2 = 0, h2 = a + 1;   // block b holding column c: the largest with srow[e0 + b] <= c
        while (h2 - l2 > 1) {
            const int mid = (l2 + h2) >> 1;
            if (srow[e0 + mid] <= c) l2 = mid;
            else h2 = mid;
        }
        const int j = sidx[e0 + l2], cl = c - srow[e0 + l2];
        float2 *dst = nullptr;
        if (j == i) {
            dst = Ad + doff[i] + (int64_t)cl * ni;
        } else {
            const int r = find_row(sptr, sidx, srow, j, i);   // >= 0 when S is the symbolic fill
            if (r >= 0) dst = A + coff[j] + r + (int64_t)cl * M[j];
        }
        s_col[threadIdx.x] = dst;
    }
    tc::Acc acc;
    unsigned char *base = tc::align1024(smraw);
    acc.planes = base;
    acc.mbar = &s_mbar;
    acc.tslot = &s_tslot;
    acc.open(ni, nc);
    const float2 *Aik = A + coff[k] + srow[e0 + a];        // n_i x n_k, ld M_k (panel k is not written)
    const float2 *Wc = W + coff[k] + (int64_t)c0 * nk;     // n_k x nc, ld n_k
    for (int q0 = 0; q0 < nk; q0 += tc::KC) {
        const int kl = min(tc::KC, nk - q0);
        acc.wait(err, bound);   // the previous chunk's MMAs have read the planes
        for (int e = threadIdx.x; e < ni * kl; e += blockDim.x) {
            const int r = e % ni, q = e / ni;
            acc.put_a(r, q, Aik[r + (int64_t)(q0 + q) * Mk]);
        }
        for (int e = threadIdx.x; e < kl * nc; e += blockDim.x) {
            const int q = e % kl, c = e / kl;
            acc.put_b(c, q, Wc[(q0 + q) + (int64_t)c * nk]);
        }
        acc.zero_pad(kl);
        acc.issue(kl);
    }
    acc.wait(err, bound);
    float *dsm = (float *)base;
    if (acc.drain(dsm)) {
        for (int e = threadIdx.x; e < ni * nc; e += blockDim.x) {
            const int r = e % ni, c = e / ni;
            float2 *dst = s_col[c];
            if (dst) {
                const float2 v = acc.entry(dsm, r, c);
                float2 o = dst[r];
                o.x -= v.x;
                o.y -= v.y;
                dst[r] = o;
            }
        }
    }
    acc.close();
}

// Column blocks per CTA of the grouped update: the most (up to 8) that still leaves at least
// four CTAs per SM.
static int upd_group(int ns, int nsm)
{
    int gb = 8;
    while (gb > 1 && upd_first(ns, gb) < 4L * nsm) gb >>= 1;
    return gb;
}

// one pivot block on a cluster of h->pivot_cl CTAs (2, 4 or 8)
template <class S>
static cudaError_t pivot_cluster(hm_ctx *h, int k, int nk, const S *Ad, float2 *Dinv32)
{
    const int C = h->pivot_cl;
    const int nloc = (nk + C - 1) / C;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    cfg.blockDim = dim3(128, 1, 1);
    cfg.dynamicSmemBytes = sizeof(double2) * ((size_t)nk * (nloc + 1) + nloc);
    cfg.stream = h->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaSuccess;
    const int *sz = h->d_size;
    const int64_t *dof = h->d_doff;
    double2 *Dinv = h->d_Dinv;
    int *err = h->d_err;
    if (C == 2)
        HM_LAUNCH(h, K_PIVOT, e = cudaLaunchKernelEx(&cfg, k_pivot_inverse_cl<S, 2>, k, sz, dof, Ad, Dinv, Dinv32, err));
    else if (C == 4)
        HM_LAUNCH(h, K_PIVOT, e = cudaLaunchKernelEx(&cfg, k_pivot_inverse_cl<S, 4>, k, sz, dof, Ad, Dinv, Dinv32, err));
    else
        HM_LAUNCH(h, K_PIVOT, e = cudaLaunchKernelEx(&cfg, k_pivot_inverse_cl<S, 8>, k, sz, dof, Ad, Dinv, Dinv32, err));
    if (e) return e;
    return cudaGetLastError();
}

template <class S>
static cudaError_t setup_typed(hm_ctx *h, S *A, S *Ad, S *W, S *DinvS, float2 *Dinv32, int *bad_block)
{
    Plan &P = h->plan;
    cudaStream_t st = h->stream;
    cudaError_t e;
    *bad_block = -1;
    if ((e = cudaMemsetAsync(A, 0, sizeof(S) * P.coef_entries, st))) return e;
    if ((e = cudaMemsetAsync(Ad, 0, sizeof(S) * P.diag_entries, st))) return e;
    if ((e = cudaMemsetAsync(h->d_err, 0, sizeof(int), st))) return e;
    HM_LAUNCH(h, K_SCATTER,
              k_scatter_near<S><<<(int)h->near_t.size(), 128, 0, st>>>(
                  (int)h->near_t.size(), h->d_near_t, h->d_near_s, h->d_near_off, h->d_near, h->d_leaf_ptr, h->d_pos,
                  h->d_sptr, h->d_sidx, h->d_srow, h->d_M, h->d_coff, h->d_doff, A, Ad, h->d_err));
    if ((e = cudaGetLastError())) return e;
    const size_t inv_smem = sizeof(double2) * (64 * 65 + 128);
    const size_t panel_smem = sizeof(S) * (2 * 64 * 65);
    if ((e = cudaFuncSetAttribute(k_pivot_inverse<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(k_panel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(k_update_grp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)UPD_SMEM))) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))) return e;
    if (sizeof(S) == 8 && h->update_kind == 2) {
        if (!h->d_ucum) {   // tensor-core update tasks: per row a of S_k, 64-column pieces of W_k
            std::vector<int> uc(std::max<size_t>(P.sidx.size(), 1));
            h->utot.assign(P.nb, 0);
            for (int k = 0; k < P.nb; ++k) {
                int c = 0;
                for (int x = P.sptr[k]; x < P.sptr[k + 1]; ++x) {
                    uc[x] = c;
                    c += (P.srow[x] + P.size[P.sidx[x]] + 63) / 64;
                }
                h->utot[k] = c;
            }
            if ((e = h->arena.alloc((void **)&h->d_ucum, sizeof(int) * uc.size())) ||
                (e = cudaMemcpyAsync(h->d_ucum, uc.data(), sizeof(int) * uc.size(), cudaMemcpyHostToDevice, st)) ||
                (e = cudaStreamSynchronize(st)))
                return e;
        }
        if ((e = cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM_BYTES)))
            return e;
    }
    for (int k = 0; k < P.nb; ++k) {
        int nk = P.size[k];
        if (h->pivot_cl > 1) {
            if ((e = pivot_cluster<S>(h, k, nk, Ad, Dinv32))) return e;
        } else
            HM_LAUNCH(h, K_PIVOT,
                      k_pivot_inverse<S><<<1, 256, sizeof(double2) * (nk * (nk + 1) + 2 * nk), st>>>(
                          k, h->d_size, h->d_doff, Ad, h->d_Dinv, Dinv32, h->d_err));
        int ns = P.sptr[k + 1] - P.sptr[k];
        if (ns > 0) {
            int Mk = P.M[k];
            HM_LAUNCH(h, K_PANEL,
                      k_panel<S><<<(Mk + 63) / 64, 256, panel_smem, st>>>(k, h->d_size, h->d_M, h->d_coff, h->d_doff,
                                                                          DinvS, A, W));
            if (h->opts.compress_in_setup && (e = compress_step<S>(h, k, W))) return e;
            if constexpr (sizeof(S) == 8) {
                if (h->update_kind == 2) {
                    HM_LAUNCH(h, K_UPDATE,
                              k_update_tc<<<(unsigned)h->utot[k], 256, tc::SMEM_BYTES, st>>>(
                                  k, ns, h->d_ucum, h->d_size, h->d_sptr, h->d_sidx, h->d_srow, h->d_M, h->d_coff,
                                  h->d_doff, W, A, Ad, h->d_err, WAIT_NS_DEFAULT));
                    if ((e = cudaGetLastError())) return e;
                    continue;
                }
                const int gb = upd_group(ns, nsm);
                HM_LAUNCH(h, K_UPDATE,
                          k_update_grp<<<(unsigned)upd_first(ns, gb), 256, UPD_SMEM, st>>>(
                              k, ns, gb, h->d_size, h->d_sptr, h->d_sidx, h->d_srow, h->d_M, h->d_coff, h->d_doff,
                              W, A, Ad));
            } else {
                long nt = (long)ns * (ns + 1) / 2;
                HM_LAUNCH(h, K_UPDATE,
                          k_update<S><<<(unsigned)nt, 256, 0, st>>>(k, ns, h->d_size, h->d_sptr, h->d_sidx,
                                                                    h->d_srow, h->d_M, h->d_coff, h->d_doff, W, A,
                                                                    Ad));
            }
        }
        if ((e = cudaGetLastError())) return e;
    }
    int herr = 0;
    if ((e = cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    if (herr == 0x7fffffff) return cudaErrorInvalidValue;   // plan / pattern mismatch
    if (herr == ERR_TIMEOUT) return cudaErrorLaunchTimeout;   // a tensor-core wait gave up
    if (herr > 0) *bad_block = herr - 1;
    return cudaSuccess;
}

// Block Jacobi (Sec. 1's block diagonal preconditioner): D_k = Z_kk, all inverted at once.
cudaError_t block_jacobi_setup(hm_ctx *h, int *bad_block)
{
    Plan &P = h->plan;
    cudaStream_t st = h->stream;
    cudaError_t e;
    *bad_block = -1;
    if ((e = cudaMemsetAsync(h->d_Ad, 0, sizeof(double2) * P.diag_entries, st))) return e;
    if ((e = cudaMemsetAsync(h->d_err, 0, sizeof(int), st))) return e;
    HM_LAUNCH(h, K_SCATTER,
              k_scatter_near<double2><<<(int)h->near_t.size(), 128, 0, st>>>(
                  (int)h->near_t.size(), h->d_near_t, h->d_near_s, h->d_near_off, h->d_near, h->d_leaf_ptr, h->d_pos,
                  h->d_sptr, h->d_sidx, h->d_srow, h->d_M, h->d_coff, h->d_doff, (double2 *)nullptr, h->d_Ad, h->d_err,
                  true));
    const size_t inv_smem = sizeof(double2) * (64 * 65 + 128);
    if ((e = cudaFuncSetAttribute(k_pivot_inverse<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)inv_smem)))
        return e;
    HM_LAUNCH(h, K_PIVOT,
              k_pivot_inverse<double2><<<P.nb, 256, inv_smem, st>>>(0, h->d_size, h->d_doff, h->d_Ad, h->d_Dinv,
                                                                    nullptr, h->d_err));
    if ((e = cudaGetLastError())) return e;
    int herr = 0;
    if ((e = cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    if (herr > 0 && herr != 0x7fffffff) *bad_block = herr - 1;
    return cudaSuccess;
}

cudaError_t setup_run(hm_ctx *h, int *bad_block)
{
    if (h->opts.precision == 1)
        return setup_typed<float2>(h, h->d_A32, h->d_Ad32, h->d_W32, h->d_Dinv32, h->d_Dinv32, bad_block);
    return setup_typed<double2>(h, h->d_A, h->d_Ad, h->d_W, h->d_Dinv, nullptr, bad_block);
}

}  // namespace hm
