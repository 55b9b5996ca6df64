// hm_far_apply_noalloc: the far-field product y = Z_F x that performs no device allocation.
//
// Who needs it: callers that must not call cudaMalloc / cudaFree at the point of the call.
// For example, a serving loop that keeps several streams busy cannot afford cudaFree, which
// synchronises the whole device; and a process whose device memory is already held by
// another allocator's pool (a framework's caching allocator) may find a raw cudaMalloc
// failing.  The regular path (hm_apply, op 3) allocates its scratch lazily on first use.
//
// Scratch: one file-scope device array of HM_NOALLOC_SCRATCH complex doubles (16 MiB).  It
// is part of the library image, so every GPU that loads the library holds it until the
// process exits.  The cluster-order copy of x (n * nrhs entries) and the two rank-vector
// sets of the far blocks (2 * sum(rank) * nrhs entries) live in it; a call needing more is
// rejected with HM_EINVAL before any GPU work.  Every word the kernels read is written
// earlier in the same call, so nothing has to be cleared between calls.  All calls share
// the array: calls that overlap on the GPU (other streams, other handles on the device)
// race on it and must be serialised by the caller.
//
// Set-up: host code must not use the array's name as a device address (on the host it
// names a host-side stand-in).  The first call on each device, with that device current,
// asks the runtime for the array's device address (cudaGetSymbolAddress) and caches it.  The
// cached address belongs to the device's primary context as the first call found it; a caller
// that resets the device (cudaDeviceReset) must reload the library before calling again.
#include <mutex>

#include "hm_internal.h"

#define HM_NOALLOC_SCRATCH (1 << 20)

static __device__ __align__(256) double2 g_far_scratch[HM_NOALLOC_SCRATCH];

namespace {

constexpr int kMaxDevices = 64;
double2 *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// u[i + r*n] = x[cl2new[i] + r*n]  (cluster-order copy of the solve-order input)
__global__ void k_na_gather(int n, int nrhs, const int *cl2new, const double2 *x, double2 *u)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nrhs) return;
    int i = (int)(e % n), r = (int)(e / n);
    u[e] = x[cl2new[i] + (int64_t)r * n];
}

__device__ __forceinline__ double2 na_fma(double2 a, double2 b, double2 c)
{
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(a.y, b.x, c.y);
    return c;
}

// rank vectors: t_b = V_b^T u[c-range], s_b = U_b^T u[r-range], one warp per far block
__global__ void __launch_bounds__(256) k_na_far1(int nf, const int *r0, const int *r1, const int *c0, const int *c1,
                                                 const int *rank, const int64_t *uoff, const int64_t *voff,
                                                 const int64_t *toff, const double2 *U, const double2 *V,
                                                 const double2 *u, int n, int nrhs, double2 *t, double2 *s,
                                                 int64_t tlen)
{
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (b >= nf) return;
    const int rk = rank[b];
    if (rk <= 0) return;
    const int m = r1[b] - r0[b], nc = c1[b] - c0[b];
    const double2 *Ub = U + uoff[b], *Vb = V + voff[b];
    for (int r = 0; r < nrhs; ++r) {
        const double2 *uc = u + c0[b] + (int64_t)r * n, *ur = u + r0[b] + (int64_t)r * n;
        for (int l = 0; l < rk; ++l) {
            double2 a1 = make_double2(0, 0), a2 = make_double2(0, 0);
            for (int i = lane; i < nc; i += 32) a1 = na_fma(Vb[i + (int64_t)l * nc], uc[i], a1);
            for (int i = lane; i < m; i += 32) a2 = na_fma(Ub[i + (int64_t)l * m], ur[i], a2);
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

// per leaf: sum of every far block covering its rows, written at its solve-order position
__global__ void __launch_bounds__(128) k_na_far2(int nl, const int *leaf_ptr, const int *lptr, const int *lent,
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
                const double2 *Ub = U + uoff[b] + (a - r0[b]) + i;
                const double2 *tb = t + toff[b] + r * tlen;
                for (int q = 0; q < rank[b]; ++q) acc = na_fma(Ub[(int64_t)q * m], tb[q], acc);
            } else if (kind == 1) {
                const double2 *Vb = V + voff[b] + (a - c0[b]) + i;
                const double2 *sb = s + toff[b] + r * tlen;
                for (int q = 0; q < rank[b]; ++q) acc = na_fma(Vb[(int64_t)q * nc], sb[q], acc);
            } else if (kind == 2) {
                const double2 *B = U + uoff[b] + (a - r0[b]) + i;
                const double2 *uc = u + c0[b] + (int64_t)r * n;
                for (int q = 0; q < nc; ++q) acc = na_fma(B[(int64_t)q * m], uc[q], acc);
            } else {
                const double2 *B = U + uoff[b] + (int64_t)((a - c0[b]) + i) * m;
                const double2 *ur = u + r0[b] + (int64_t)r * n;
                for (int q = 0; q < m; ++q) acc = na_fma(B[q], ur[q], acc);
            }
        }
        y[on + i + (int64_t)r * n] = acc;
    }
}

// Device address of the scratch array for the current device (looked up once per device).
cudaError_t scratch_for_device(int dev, double2 **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_far_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double2 *)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int hm_far_apply_noalloc(hm_handle h, const void *dx, void *dy, int32_t nrhs)
{
    if (!h || !dx || !dy || nrhs < 1) return HM_EINVAL;
    const int n = h->n;
    const hm::FarPlan &F = h->fplan;
    const int64_t need = (int64_t)n * nrhs + 2 * std::max<int64_t>(F.tlen, 0) * nrhs;
    if (need > HM_NOALLOC_SCRATCH) {
        h->err = "hm_far_apply_noalloc: this call needs " + std::to_string(need) +
                 " complex scratch entries but the static scratch holds " + std::to_string(HM_NOALLOC_SCRATCH) +
                 "; pass fewer right-hand sides per call";
        return HM_EINVAL;
    }
    cudaError_t e;
    if ((e = cudaSetDevice(h->dev))) {
        h->err = std::string("hm_far_apply_noalloc: ") + cudaGetErrorString(e);
        return HM_ECUDA;
    }
    double2 *scratch = nullptr;
    if ((e = scratch_for_device(h->dev, &scratch))) {
        h->err = std::string("hm_far_apply_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
        return HM_ECUDA;
    }
    double2 *u = scratch;                                   // n x nrhs, cluster order
    double2 *t = scratch + (size_t)n * nrhs;                // tlen x nrhs
    double2 *s = t + (size_t)F.tlen * nrhs;                 // tlen x nrhs
    const double2 *x = (const double2 *)dx;
    double2 *y = (double2 *)dy;
    const int64_t tot = (int64_t)n * nrhs;
    k_na_gather<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(n, nrhs, h->d_cl2new, x, u);
    if (F.nf > 0 && F.tlen > 0)
        k_na_far1<<<(unsigned)(((int64_t)F.nf * 32 + 255) / 256), 256, 0, h->stream>>>(
            F.nf, h->d_far_r0, h->d_far_r1, h->d_far_c0, h->d_far_c1, h->d_far_rank, h->d_far_uoff, h->d_far_voff,
            h->d_far_toff, h->d_farU, h->d_farV, u, n, nrhs, t, s, F.tlen);
    k_na_far2<<<h->nl, 128, 0, h->stream>>>(h->nl, h->d_leaf_ptr, h->d_flptr, h->d_flent, h->d_far_r0, h->d_far_r1,
                                            h->d_far_c0, h->d_far_c1, h->d_far_rank, h->d_far_uoff, h->d_far_voff,
                                            h->d_far_toff, h->d_farU, h->d_farV, t, s, u, h->d_cl2new, n, nrhs, y,
                                            F.tlen);
    if ((e = cudaGetLastError()) || (e = cudaStreamSynchronize(h->stream))) {
        h->err = std::string("hm_far_apply_noalloc: ") + cudaGetErrorString(e);
        return HM_ECUDA;
    }
    return HM_OK;
}
