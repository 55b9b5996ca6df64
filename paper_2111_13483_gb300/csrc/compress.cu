// Compression of the fill-in scaling-coefficient blocks (Sec. 3.4, Tables 5-6).
//
// After the numeric factorisation, every coefficient block W_kj whose block pair (k, j) is
// not a near-field pair (a fill-in block) is replaced by its truncated SVD of the smallest
// rank r whose singular-value tail has Frobenius norm <= fill_tol ||W_kj||_F; blocks for
// which r (n_k + n_j) >= n_k n_j stay dense.  Near-pattern blocks are never compressed.
// The truncation is written into the block's own panel slot as its factors P (n_k x r, the
// left singular vectors scaled by the singular values) then Q (n_j x r), W_kj ~ P Q^T
// (r (n_k + n_j) < n_k n_j entries, so they fit), and its rank is recorded; pack_run then
// gathers every block -- dense, or its factors -- into the compact store the sweeps read.
//
// One CTA per fill-in block: the one-sided Jacobi SVD of jacobi.cuh in shared memory, of
// A = W when n_k >= n_j and of A = W^H otherwise, so that A never has more columns than rows
// (surplus columns of a wide block could never become mutually orthogonal: they would keep
// rotating at rounding level); the rounding floor of the skip rule is u^2 ||W||_F^2.  Then
// sigma_i = ||a_i||, A ~ sum over the r largest of a_i v_i^H.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cplx.cuh"
#include "hm_internal.h"
#include "jacobi.cuh"

namespace hm {


template <class TC>
__global__ void __launch_bounds__(256) k_compress(int nfill, const int *fill_e, const int *fill_k, const int *size,
                                                  const int *sidx, const int *srow, const int64_t *coff, TC *W,
                                                  double tol, int *rank_out, bool expand = false)
{
    typedef typename Real<TC>::type R;
    extern __shared__ unsigned char smraw[];
    TC *A = (TC *)smraw;          // A[c*64 + r], nr x nc
    TC *V = A + 64 * 64;          // V[c*64 + r], nc x nc
    __shared__ R sig[64];
    __shared__ int ord[64];
    __shared__ int s_rot, s_rank;
    const int f = blockIdx.x;
    if (f >= nfill) return;
    const int e = fill_e[f], k = fill_k[f];
    const int m = size[k], n = size[sidx[e]];
    TC *Wb = W + coff[k] + (int64_t)srow[e] * m;   // m x n, column-major, ld m
    __shared__ R s_part[8];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const bool tr = m < n;                       // A = W^H (rows nr = n, columns nc = m)
    const int nr = tr ? n : m, nc = tr ? m : n;
    R fro2 = 0;
    for (int x = threadIdx.x; x < m * n; x += blockDim.x) {
        const int r = x % m, c = x / m;
        const TC w = Wb[x];
        fro2 += w.x * w.x + w.y * w.y;
        if (tr) A[r * 64 + c] = jconj(w);
        else A[c * 64 + r] = w;
    }
    for (int x = threadIdx.x; x < nc * nc; x += blockDim.x) {
        const int r = x % nc, c = x / nc;
        V[c * 64 + r] = (r == c) ? cconv<TC>(make_double2(1.0, 0.0)) : czero(TC());
    }
    for (int o = 16; o > 0; o >>= 1) fro2 += __shfl_xor_sync(0xffffffffu, fro2, o);
    if (lane == 0) s_part[wp] = fro2;
    __syncthreads();
    fro2 = 0;
    for (int w = 0; w < 8; ++w) fro2 += s_part[w];
    const R floor2 = JacobiEps<TC>::u() * JacobiEps<TC>::u() * fro2;   // rounding level of the block
    jacobi_sweeps<TC, 64>(A, V, nr, nc, floor2, &s_rot);
    column_norms2<TC, 64>(A, nr, nc, sig);   // singular values squared
    __syncthreads();
    if (threadIdx.x == 0) {
        int r = truncation_rank(sig, ord, nc, tol);
        if ((int64_t)r * (m + n) >= (int64_t)m * n) r = -1;
        s_rank = r;
    }
    __syncthreads();
    const int r = s_rank;
    if (r >= 0 && expand) {   // the truncation itself, in place (used by the later Schur updates)
        for (int x = threadIdx.x; x < m * n; x += blockDim.x) {
            const int row = x % m, c = x / m;
            TC acc = czero(TC());
            for (int l = 0; l < r; ++l) {
                const int o = ord[l];
                acc = tr ? cfma(V[o * 64 + row], jconj(A[o * 64 + c]), acc)
                         : cfma(A[o * 64 + row], jconj(V[o * 64 + c]), acc);
            }
            Wb[x] = acc;
        }
    } else if (r >= 0) {
        // W ~ sum over the r largest of a_o conj(v_o)^T (W = A V^H), or of v_o conj(a_o)^T in the
        // transposed case (W = (A V^H)^H = V A^H): P(:, l) and Q(:, l) from the l-th largest
        TC *Pb = Wb, *Qb = Wb + (int64_t)m * r;
        for (int x = threadIdx.x; x < m * r; x += blockDim.x) {
            const int row = x % m, o = ord[x / m];
            Pb[x] = tr ? V[o * 64 + row] : A[o * 64 + row];
        }
        for (int x = threadIdx.x; x < n * r; x += blockDim.x) {
            const int c = x % n, o = ord[x / n];
            Qb[x] = jconj(tr ? A[o * 64 + c] : V[o * 64 + c]);
        }
    }
    if (threadIdx.x == 0) rank_out[f] = r;
}

// The same compression with one warp per fill-in block (jacobi_sweeps_warp), for the
// factorised panels after the elimination.  The host packs the blocks, largest shared-memory
// footprint first, into CTAs of up to CW_WARPS warps whose regions fit CW_BYTES; warp w of CTA
// b takes block item[first[b] + w] in the region at soff (entries of TC): A (nr x nc, leading
// dimension nr | 1), V (nc x nc, leading dimension nc | 1), then the norms and the order of
// the truncation.  Ranks, factors and their layout are those of k_compress.
constexpr int CW_WARPS = 8;
constexpr int CW_BYTES = 110 * 1024;

__host__ __device__ __forceinline__ int cw_footprint(int m, int n)
{
    const int nr = m < n ? n : m, nc = m < n ? m : n;
    return nc * ((nr | 1) + (nc | 1)) + 64;   // entries; the last 64 hold the norms and the order
}

template <class TC>
__global__ void __launch_bounds__(CW_WARPS * 32) k_compress_w(const int *first, const int *item, const int *soff,
                                                              const int *fill_e, const int *fill_k, const int *size,
                                                              const int *sidx, const int *srow, const int64_t *coff,
                                                              TC *W, double tol, int *rank_out)
{
    typedef typename Real<TC>::type R;
    extern __shared__ unsigned char smraw[];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int x = first[blockIdx.x] + wp;
    if (x >= first[blockIdx.x + 1]) return;   // the rest of the kernel uses warp barriers only
    const int f = item[x];
    const int e = fill_e[f], k = fill_k[f];
    const int m = size[k], n = size[sidx[e]];
    TC *Wb = W + coff[k] + (int64_t)srow[e] * m;   // m x n, column-major, ld m
    const bool tr = m < n;                       // A = W^H (rows nr = n, columns nc = m)
    const int nr = tr ? n : m, nc = tr ? m : n;
    const int lda = nr | 1, ldv = nc | 1;
    TC *A = (TC *)smraw + soff[x];
    TC *V = A + nc * lda;
    R *sig = (R *)(V + nc * ldv);
    int *ord = (int *)(sig + 64);
    R fro2 = 0;
    for (int t = lane; t < m * n; t += 32) {
        const int r = t % m, c = t / m;
        const TC w = Wb[t];
        fro2 += w.x * w.x + w.y * w.y;
        if (tr) A[r * lda + c] = jconj(w);
        else A[c * lda + r] = w;
    }
    for (int t = lane; t < nc * nc; t += 32) {
        const int r = t % nc, c = t / nc;
        V[c * ldv + r] = (r == c) ? cconv<TC>(make_double2(1.0, 0.0)) : czero(TC());
    }
    for (int o = 16; o > 0; o >>= 1) fro2 += __shfl_xor_sync(0xffffffffu, fro2, o);
    __syncwarp();
    const R floor2 = JacobiEps<TC>::u() * JacobiEps<TC>::u() * fro2;   // rounding level of the block
    jacobi_sweeps_warp<TC>(A, lda, V, ldv, nr, nc, floor2);
    for (int c = lane; c < nc; c += 32) {   // singular values squared
        R s2 = 0;
        for (int r = 0; r < nr; ++r) s2 += A[c * lda + r].x * A[c * lda + r].x + A[c * lda + r].y * A[c * lda + r].y;
        sig[c] = s2;
    }
    __syncwarp();
    int r = 0;
    if (lane == 0) {
        r = truncation_rank(sig, ord, nc, tol);
        if ((int64_t)r * (m + n) >= (int64_t)m * n) r = -1;
    }
    r = __shfl_sync(0xffffffffu, r, 0);
    __syncwarp();
    if (r >= 0) {   // the factors, as k_compress writes them
        TC *Pb = Wb, *Qb = Wb + (int64_t)m * r;
        for (int t = lane; t < m * r; t += 32) {
            const int row = t % m, o = ord[t / m];
            Pb[t] = tr ? V[o * ldv + row] : A[o * lda + row];
        }
        for (int t = lane; t < n * r; t += 32) {
            const int c = t % n, o = ord[t / n];
            Qb[t] = jconj(tr ? A[o * lda + c] : V[o * ldv + c]);
        }
    }
    if (lane == 0) rank_out[f] = r;
}

// dst[e] <- the block's stored entries (dense n_k n_j, or r (n_k + n_j) factor entries), one
// CTA per S-list entry
template <class TC>
__global__ void k_pack(int ne, const int64_t *pboff, const int64_t *cboff, const TC *W, TC *Wc)
{
    const int e = blockIdx.x;
    if (e >= ne) return;
    const int64_t len = cboff[e + 1] - cboff[e];
    const TC *src = W + pboff[e];
    TC *dst = Wc + cboff[e];
    for (int64_t x = threadIdx.x; x < len; x += blockDim.x) dst[x] = src[x];
}

// The store the sweeps read (see hm_ctx::d_Wc): with no compressed block the panels themselves;
// otherwise a compact copy with the factors of the compressed blocks, offsets and ranks uploaded.
cudaError_t pack_run(hm_ctx *h)
{
    const Plan &P = h->plan;
    const bool mixed = h->opts.precision == 1;
    const int ne = (int)P.sidx.size();
    cudaError_t e;
    bool lr = false;
    for (int r : h->fill_ranks) lr = lr || r >= 0;
    if (!lr) {
        if (h->wc_len) {
            h->arena.release(mixed ? (void *)h->d_Wc32 : (void *)h->d_Wc, 0);
            h->wc_len = 0;
        }
        if (h->lowrank) {   // back to the panel layout
            if ((e = cudaMemcpyAsync(h->d_cboff, P.pboff.data(), sizeof(int64_t) * ne, cudaMemcpyHostToDevice,
                                     h->stream)))
                return e;
            if ((e = cudaMemsetAsync(h->d_crank, 0xff, sizeof(int) * ne, h->stream))) return e;
        }
        h->lowrank = false;
        h->d_Wc = h->d_W;
        h->d_Wc32 = h->d_W32;
        h->cboff = P.pboff;
        h->crank.assign(ne, -1);
        return cudaStreamSynchronize(h->stream);
    }
    h->crank.assign(ne, -1);
    for (size_t f = 0; f < P.fill_e.size(); ++f) h->crank[P.fill_e[f]] = h->fill_ranks[f];
    h->cboff.assign(ne + 1, 0);
    for (int k = 0; k < P.nb; ++k)
        for (int x = P.sptr[k]; x < P.sptr[k + 1]; ++x) {
            const int64_t nk = P.size[k], nj = P.size[P.sidx[x]], r = h->crank[x];
            h->cboff[x + 1] = h->cboff[x] + (r < 0 ? nk * nj : r * (nk + nj));
        }
    const int64_t total = h->cboff[ne];
    if (h->wc_len != total) {
        if (h->wc_len) h->arena.release(mixed ? (void *)h->d_Wc32 : (void *)h->d_Wc, 0);
        h->wc_len = 0;
        if ((e = mixed ? h->arena.alloc((void **)&h->d_Wc32, sizeof(float2) * total)
                       : h->arena.alloc((void **)&h->d_Wc, sizeof(double2) * total)))
            return e;
        h->wc_len = total;
    }
    if ((e = cudaMemcpyAsync(h->d_cboff, h->cboff.data(), sizeof(int64_t) * (ne + 1), cudaMemcpyHostToDevice,
                             h->stream)) ||
        (e = cudaMemcpyAsync(h->d_crank, h->crank.data(), sizeof(int) * ne, cudaMemcpyHostToDevice, h->stream)))
        return e;
    if (ne > 0) {
        if (mixed)
            HM_LAUNCH(h, K_COMPRESS, k_pack<float2><<<ne, 128, 0, h->stream>>>(ne, h->d_pboff, h->d_cboff, h->d_W32,
                                                                               h->d_Wc32));
        else
            HM_LAUNCH(h, K_COMPRESS, k_pack<double2><<<ne, 128, 0, h->stream>>>(ne, h->d_pboff, h->d_cboff, h->d_W,
                                                                                h->d_Wc));
    }
    h->lowrank = true;
    if ((e = cudaGetLastError())) return e;
    return cudaStreamSynchronize(h->stream);
}

// Compression during the setup: the fill-in blocks of panel k truncated in place, before the
// Schur updates of step k read them (hm_opts.compress_in_setup).
template <class TC> cudaError_t compress_step(hm_ctx *h, int k, TC *W)
{
    const Plan &P = h->plan;
    const int f0 = P.fill_ptr[k], nf = P.fill_ptr[k + 1] - f0;
    if (nf == 0 || !(h->opts.fill_tol > 0)) return cudaSuccess;
    cudaError_t e;
    if (!h->d_fill_rank && (e = h->arena.alloc((void **)&h->d_fill_rank, sizeof(int) * P.fill_e.size()))) return e;
    const size_t smem = sizeof(TC) * 2 * 64 * 64;
    static DeviceOnce attr;
    if (attr.need()) {
        if ((e = cudaFuncSetAttribute(k_compress<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        attr.done();
    }
    HM_LAUNCH(h, K_COMPRESS,
              k_compress<TC><<<nf, 256, smem, h->stream>>>(nf, h->d_fill_e + f0, h->d_fill_k + f0, h->d_size, h->d_sidx,
                                                           h->d_srow, h->d_coff, W, h->opts.fill_tol,
                                                           h->d_fill_rank + f0, true));
    return cudaGetLastError();
}
template cudaError_t compress_step<double2>(hm_ctx *, int, double2 *);
template cudaError_t compress_step<float2>(hm_ctx *, int, float2 *);

cudaError_t compress_run(hm_ctx *h)
{
    const Plan &P = h->plan;
    const int nfill = (int)P.fill_e.size();
    h->fill_ranks.assign(nfill, -1);
    if (nfill == 0 || !(h->opts.fill_tol > 0)) return cudaSuccess;
    cudaError_t e;
    if (!h->d_fill_rank && (e = h->arena.alloc((void **)&h->d_fill_rank, sizeof(int) * nfill))) return e;
    // FP64 Jacobi on the FP64 factors (the oracle's rank decisions); FP32 on the FP32 factors
    // of the mixed-precision setup
    const bool mixed = h->opts.precision == 1;
    if (h->cw_first.empty()) {   // pack the blocks into CTAs (once per handle)
        const int esz = mixed ? (int)sizeof(float2) : (int)sizeof(double2);
        const int cap = CW_BYTES / esz;
        std::vector<int> foot(nfill), ordv(nfill);
        for (int f = 0; f < nfill; ++f) {
            foot[f] = cw_footprint(P.size[P.fill_k[f]], P.size[P.sidx[P.fill_e[f]]]);
            ordv[f] = f;
        }
        std::stable_sort(ordv.begin(), ordv.end(), [&](int a, int b) { return foot[a] > foot[b]; });
        std::vector<int> off(nfill);
        h->cw_first.assign(1, 0);
        int used = 0, cnt = 0;
        h->cw_smem = 0;
        for (int x = 0; x < nfill; ++x) {
            const int fp = foot[ordv[x]];
            if (cnt == CW_WARPS || (cnt > 0 && used + fp > cap)) {
                h->cw_first.push_back(x);
                used = cnt = 0;
            }
            off[x] = used;
            used += fp;
            ++cnt;
            h->cw_smem = std::max<size_t>(h->cw_smem, (size_t)used * esz);
        }
        h->cw_first.push_back(nfill);
        if ((e = h->arena.alloc((void **)&h->d_cw, sizeof(int) * (h->cw_first.size() + 2 * (size_t)nfill))) ||
            (e = cudaMemcpyAsync(h->d_cw, h->cw_first.data(), sizeof(int) * h->cw_first.size(), cudaMemcpyHostToDevice,
                                 h->stream)) ||
            (e = cudaMemcpyAsync(h->d_cw + h->cw_first.size(), ordv.data(), sizeof(int) * nfill,
                                 cudaMemcpyHostToDevice, h->stream)) ||
            (e = cudaMemcpyAsync(h->d_cw + h->cw_first.size() + nfill, off.data(), sizeof(int) * nfill,
                                 cudaMemcpyHostToDevice, h->stream)) ||
            (e = cudaStreamSynchronize(h->stream)))
            return e;
    }
    // a block larger than CW_BYTES (FP64, n_k = n_j = 64: 134 KB) has a CTA of its own; the
    // limit is raised per device (the attribute belongs to the device) to the largest need seen
    static std::atomic<size_t> attr_w[2][64];
    const int dev = DeviceOnce::device();
    if (dev < 0 || dev >= 64 || h->cw_smem > attr_w[mixed][dev].load()) {
        if ((e = mixed ? cudaFuncSetAttribute(k_compress_w<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)h->cw_smem)
                       : cudaFuncSetAttribute(k_compress_w<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)h->cw_smem)))
            return e;
        if (dev >= 0 && dev < 64) attr_w[mixed][dev].store(h->cw_smem);
    }
    const unsigned ncta = (unsigned)h->cw_first.size() - 1;
    const int *d_first = h->d_cw, *d_item = h->d_cw + h->cw_first.size(), *d_off = d_item + nfill;
    if (mixed)
        HM_LAUNCH(h, K_COMPRESS,
                  k_compress_w<float2><<<ncta, CW_WARPS * 32, h->cw_smem, h->stream>>>(
                      d_first, d_item, d_off, h->d_fill_e, h->d_fill_k, h->d_size, h->d_sidx, h->d_srow, h->d_coff,
                      h->d_W32, h->opts.fill_tol, h->d_fill_rank));
    else
        HM_LAUNCH(h, K_COMPRESS,
                  k_compress_w<double2><<<ncta, CW_WARPS * 32, h->cw_smem, h->stream>>>(
                      d_first, d_item, d_off, h->d_fill_e, h->d_fill_k, h->d_size, h->d_sidx, h->d_srow, h->d_coff,
                      h->d_W, h->opts.fill_tol, h->d_fill_rank));
    if ((e = cudaGetLastError())) return e;
    if ((e = cudaMemcpyAsync(h->fill_ranks.data(), h->d_fill_rank, sizeof(int) * nfill, cudaMemcpyDeviceToHost,
                             h->stream)))
        return e;
    return cudaStreamSynchronize(h->stream);
}

}  // namespace hm
