// Restarted GMRES (Sec. 5) on the preconditioned system of Eq. 28, for batches of columns
// in lockstep (each column its own Krylov space), and the mixed-precision refinement loop.
//
// FP64 mode: GMRES on A x~ = c with the FP64 operator, stop at |g_{j+1}| <= tol ||c||.
// Mixed mode: an outer FP64 loop r = V - Z I (near blocks + far factors in FP64), inner
// GMRES on A d~ = D^{-1} L^{-1} r with the complex-FP32 operator, I += L^{-T} d~, until
// ||V - Z I|| <= tol ||V||.  Arnoldi vectors, Gram-Schmidt, Givens rotations and the
// refinement residual are FP64 in both modes.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "cplx.cuh"
#include "hm_internal.h"

namespace hm {

constexpr int DOT_CHUNK = 4096;

// part[((c*J + i) * nchunk + chunk)] = sum over the chunk's rows of conj(V_i) w (i < J);
// basis V_i of column c at Vb + (i*nc + c)*n
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
                if (q < ni) acc[q] = cjfma(Vb[((int64_t)(i0 + q) * nc + c) * n + row], wv, acc[q]);
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

// out[c*ldo + i] = sum over chunks of part (fixed order)
__global__ void k_dots_final(int nc, int J, int nchunk, const double2 *part, double2 *out, int ldo)
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
    out[(int64_t)c * ldo + i] = v;
}

// w[:, c] -= sum_{i<J} h[c*ldh + i] V_i[:, c]
__global__ void k_axpy_basis(int n, int nc, int J, const double2 *Vb, const double2 *h, int ldh, double2 *w)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nc) return;
    int row = (int)(e % n), c = (int)(e / n);
    double2 acc = w[e];
    for (int i = 0; i < J; ++i) acc = cfms(h[(int64_t)c * ldh + i], Vb[((int64_t)i * nc + c) * n + row], acc);
    w[e] = acc;
}

// x[:, c] += sum_{i<J[c]} y[c*ldy + i] V_i[:, c]
__global__ void k_update_x(int n, int nc, const int *J, const double2 *Vb, const double2 *yv, int ldy, double2 *x)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nc) return;
    int row = (int)(e % n), c = (int)(e / n);
    double2 acc = x[e];
    for (int i = 0; i < J[c]; ++i) acc = cfma(yv[(int64_t)c * ldy + i], Vb[((int64_t)i * nc + c) * n + row], acc);
    x[e] = acc;
}

// v[:, c] = w[:, c] / nrm[c] (0 when nrm[c] = 0)
__global__ void k_scale(int n, int nc, const double *nrm, const double2 *w, double2 *v)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nc) return;
    int c = (int)(e / n);
    double s = nrm[c] > 0 ? 1.0 / nrm[c] : 0.0;
    double2 a = w[e];
    v[e] = make_double2(a.x * s, a.y * s);
}

// r = c - r
__global__ void k_sub_from(int64_t len, const double2 *c, double2 *r)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= len) return;
    r[e] = make_double2(c[e].x - r[e].x, c[e].y - r[e].y);
}

// x += a
__global__ void k_add_to(int64_t len, const double2 *a, double2 *x)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= len) return;
    x[e] = make_double2(x[e].x + a[e].x, x[e].y + a[e].y);
}

// zero the columns whose mask is 0
__global__ void k_mask_cols(int n, int nc, const int *mask, double2 *v)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nc) return;
    if (!mask[e / n]) v[e] = make_double2(0, 0);
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

// GMRES small-matrix state per column c (H: (m+1) x m column-major, ld m+1)
struct GState {
    double2 *H, *g, *sn, *y, *hj;
    double *cs, *nrm, *res, *wn;
    int *J, *active;
};

// Hessenberg column j of each active column: h[0..j] from hj, h[j+1] = nrm; previous
// rotations, a new complex Givens rotation with real cosine, residual estimate |g_{j+1}|.
__global__ void k_givens(int nc, int m, int j, GState s)
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
        // [c s; -conj(s) c] [a; b]
        double2 t = make_double2(ci * a.x + (si.x * b.x - si.y * b.y), ci * a.y + (si.x * b.y + si.y * b.x));
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
        sj = make_double2((ph.x * b.x + ph.y * b.y) / r, (ph.y * b.x - ph.x * b.y) / r);   // ph conj(b) / r
        rho = make_double2(ph.x * r, ph.y * r);
    }
    cs[j] = cj;
    sn[j] = sj;
    col[j] = rho;
    col[j + 1] = make_double2(0, 0);
    double2 gj = g[j];
    g[j + 1] = make_double2(-(sj.x * gj.x + sj.y * gj.y), -(sj.x * gj.y - sj.y * gj.x));   // -conj(s) g_j
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
        for (int q = i + 1; q < J; ++q) v = cfms(H[i + (int64_t)q * (m + 1)], y[q], v);
        double2 d = H[i + (int64_t)i * (m + 1)];
        double den = d.x * d.x + d.y * d.y;
        y[i] = make_double2((v.x * d.x + v.y * d.y) / den, (v.y * d.x - v.x * d.y) / den);
    }
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

static cudaError_t apply_op(hm_ctx *h, bool fp32, int op, const double2 *x, double2 *y, int nrhs)
{
    return fp32 ? op_apply32(h, op, x, y, nrhs) : op_apply(h, op, x, y, nrhs);
}

// Column 2-norms of v (n x nc) -> out (device) and returned to the host.
static std::vector<double> col_norms(hm_ctx *h, const double2 *v, int nc, double2 *part, double2 *tmp, double *out)
{
    const int n = h->plan.n, nchunk = (n + DOT_CHUNK - 1) / DOT_CHUNK;
    cudaStream_t st = h->stream;
    HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, nc), 256, 0, st>>>(n, nc, 1, v, v, part, nchunk));
    HM_LAUNCH(h, K_SMALL, k_dots_final<<<nblk(nc, 128), 128, 0, st>>>(nc, 1, nchunk, part, tmp, 1));
    HM_LAUNCH(h, K_SMALL, k_sqrt_re<<<nblk(nc, 128), 128, 0, st>>>(nc, tmp, 1, out));
    std::vector<double> nv(nc);
    cudaMemcpyAsync(nv.data(), out, sizeof(double) * nc, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return nv;
}

// Batched GMRES(m) on Eq. 28 for nc <= 64 columns in solve order: c (rhs), x (in/out,
// starts at zero).  Column c stops at |g_{j+1}| <= tol[c] ||c_c||.  Arnoldi by classical
// Gram-Schmidt applied twice (the oracle's modified Gram-Schmidt spans the same space up
// to rounding).  One host synchronisation per Arnoldi step reads the residual estimates.
static int gmres_batch(hm_ctx *h, bool fp32, const double2 *cvec, double2 *x, int nc, const std::vector<double> &tol,
                       int m, int maxit, int *iters, double *relres)
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
    std::vector<double> cn = col_norms(h, cvec, nc, part, h2, s.res);
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
            if ((e = apply_op(h, fp32, 0, x, r, nc))) break;
            HM_LAUNCH(h, K_VEC, k_sub_from<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>((int64_t)n * nc, cvec, r));
        }
        first = false;
        std::vector<double> beta = col_norms(h, r, nc, part, h2, s.nrm);
        std::vector<int> act(nc, 0);
        bool any = false;
        for (int c = 0; c < nc; ++c) {
            if (conv[c]) continue;
            if (beta[c] <= tol[c] * cn[c]) {
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
        HM_LAUNCH(h, K_VEC, k_scale<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, s.nrm, r, Vb));   // V_0 = r/beta
        std::vector<double2> g0((size_t)nc * (m + 1), make_double2(0, 0));
        for (int c = 0; c < nc; ++c) g0[(size_t)c * (m + 1)] = make_double2(beta[c], 0);
        cudaMemcpyAsync(s.g, g0.data(), sizeof(double2) * g0.size(), cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(s.J, 0, sizeof(int) * nc, st);
        std::vector<int> done(nc, 0);
        for (int c = 0; c < nc; ++c) done[c] = !act[c];
        std::vector<double> res(nc), wpre(nc), wn(nc);
        for (int j = 0; j < m; ++j) {
            double2 *vj = Vb + (size_t)j * nc * n, *vj1 = Vb + (size_t)(j + 1) * nc * n;
            if ((e = apply_op(h, fp32, 0, vj, w, nc))) break;
            // ||w|| before orthogonalisation (happy-breakdown reference)
            HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, nc), 256, 0, st>>>(n, nc, 1, w, w, part, nchunk));
            HM_LAUNCH(h, K_SMALL, k_dots_final<<<nblk(nc, 128), 128, 0, st>>>(nc, 1, nchunk, part, h2, 1));
            HM_LAUNCH(h, K_SMALL, k_sqrt_re<<<nblk(nc, 128), 128, 0, st>>>(nc, h2, 1, s.wn));
            // CGS2: h = V^H w, w -= V h, twice; coefficients accumulated in hcol
            HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, nc), 256, 0, st>>>(n, nc, j + 1, Vb, w, part, nchunk));
            HM_LAUNCH(h, K_SMALL,
                      k_dots_final<<<nblk(nc * (j + 1), 128), 128, 0, st>>>(nc, j + 1, nchunk, part, hcol, m + 1));
            HM_LAUNCH(h, K_VEC,
                      k_axpy_basis<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, j + 1, Vb, hcol, m + 1, w));
            HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, nc), 256, 0, st>>>(n, nc, j + 1, Vb, w, part, nchunk));
            HM_LAUNCH(h, K_SMALL,
                      k_dots_final<<<nblk(nc * (j + 1), 128), 128, 0, st>>>(nc, j + 1, nchunk, part, h2, m + 1));
            HM_LAUNCH(h, K_VEC,
                      k_axpy_basis<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, j + 1, Vb, h2, m + 1, w));
            HM_LAUNCH(h, K_SMALL, k_hfold<<<nblk(nc * (j + 1), 128), 128, 0, st>>>(nc, j + 1, h2, m + 1, hcol, m + 1));
            // h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
            HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, nc), 256, 0, st>>>(n, nc, 1, w, w, part, nchunk));
            HM_LAUNCH(h, K_SMALL, k_dots_final<<<nblk(nc, 128), 128, 0, st>>>(nc, 1, nchunk, part, h2, 1));
            HM_LAUNCH(h, K_SMALL, k_sqrt_re<<<nblk(nc, 128), 128, 0, st>>>(nc, h2, 1, s.nrm));
            HM_LAUNCH(h, K_VEC, k_scale<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, s.nrm, w, vj1));
            HM_LAUNCH(h, K_SMALL, k_givens<<<nblk(nc, 64), 64, 0, st>>>(nc, m, j, s));
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
                if (res[c] <= tol[c] * cn[c] || brk) {
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

// FP64 mode: GMRES on Eq. 28 with the FP64 operator.
static int solve_fp64(hm_ctx *h, const double2 *dV, int nc, int64_t ldv, double tol, int restart, int maxit,
                      double2 *dI, int64_t ldi, int *iters, double *relres, double2 *bnew, double2 *cvec, double2 *xt)
{
    const int n = h->plan.n;
    cudaError_t e;
    if ((e = to_solve_order(h, dV, ldv, bnew, nc)) || (e = op_apply(h, 1, bnew, xt, nc)) ||
        (e = op_apply(h, 4, xt, cvec, nc))) {
        h->err = cudaGetErrorString(e);
        return HM_ECUDA;
    }
    cudaMemsetAsync(xt, 0, sizeof(double2) * (size_t)n * nc, h->stream);
    int s = gmres_batch(h, false, cvec, xt, nc, std::vector<double>(nc, tol), restart, maxit, iters, relres);
    if (s != HM_OK && s != HM_ENOCONV) return s;
    if ((e = op_apply(h, 2, xt, bnew, nc)) || (e = to_orig_order(h, bnew, dI, ldi, nc))) {
        h->err = cudaGetErrorString(e);
        return HM_ECUDA;
    }
    return s;
}

// Mixed mode: FP64 residual-and-correction loop around the complex-FP32 inner solve.
static int solve_mixed(hm_ctx *h, const double2 *dV, int nc, int64_t ldv, double tol, int restart, int maxit,
                       double2 *dI, int64_t ldi, int *iters, double *relres, double2 *bnew, double2 *cvec,
                       double2 *xt)
{
    const int n = h->plan.n, nchunk = (n + DOT_CHUNK - 1) / DOT_CHUNK;
    cudaStream_t st = h->stream;
    cudaError_t e = cudaSuccess;
    double2 *b = nullptr, *xo = nullptr, *r = nullptr, *part = nullptr, *tmp = nullptr;
    double *nrm = nullptr;
    int *mask = nullptr;
    const size_t vec = sizeof(double2) * (size_t)n * nc;
    if ((e = h->arena.alloc((void **)&b, vec)) || (e = h->arena.alloc((void **)&xo, vec)) ||
        (e = h->arena.alloc((void **)&r, vec)) || (e = h->arena.alloc((void **)&part, sizeof(double2) * nchunk * nc)) ||
        (e = h->arena.alloc((void **)&tmp, sizeof(double2) * nc)) || (e = h->arena.alloc((void **)&nrm, sizeof(double) * nc)) ||
        (e = h->arena.alloc((void **)&mask, sizeof(int) * nc))) {
        for (void *p : {(void *)b, (void *)xo, (void *)r, (void *)part, (void *)tmp, (void *)nrm, (void *)mask})
            h->arena.release(p, 0);
        h->err = "mixed-precision workspace allocation failed";
        return HM_ENOMEM;
    }
    // b: packed copy of V (original order, ld n); xo = 0
    cudaMemcpy2DAsync(b, sizeof(double2) * n, dV, sizeof(double2) * ldv, sizeof(double2) * n, nc,
                      cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(xo, 0, vec, st);
    std::vector<double> bn = col_norms(h, b, nc, part, tmp, nrm);
    std::vector<int> total(nc, 0), done(nc, 0);
    std::vector<double> rel(nc, 0.0);
    int status = HM_OK;
    const int MAX_OUTER = 40;
    for (int outer = 0; outer <= MAX_OUTER; ++outer) {
        // r = b - Z xo in FP64
        if (outer == 0)
            cudaMemcpyAsync(r, b, vec, cudaMemcpyDeviceToDevice, st);
        else {
            if ((e = z_apply_orig(h, xo, r, nc))) break;
            HM_LAUNCH(h, K_VEC, k_sub_from<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>((int64_t)n * nc, b, r));
        }
        std::vector<double> rn = col_norms(h, r, nc, part, tmp, nrm);
        std::vector<int> act(nc, 0);
        std::vector<double> itol(nc, 0.5);
        bool any = false;
        for (int c = 0; c < nc; ++c) {
            rel[c] = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
            if (done[c]) continue;
            if (rel[c] <= tol || bn[c] == 0.0) {
                done[c] = 1;
                continue;
            }
            if (total[c] >= maxit || outer == MAX_OUTER) continue;
            act[c] = 1;
            any = true;
            // ask the inner solve for a little more than what is still missing
            itol[c] = std::min(0.5, std::max(1e-7, 0.3 * tol / rel[c]));
        }
        if (!any) break;
        int left = maxit;
        for (int c = 0; c < nc; ++c)
            if (act[c]) left = std::min(left, maxit - total[c]);
        cudaMemcpyAsync(mask, act.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st);
        HM_LAUNCH(h, K_VEC, k_mask_cols<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, mask, r));
        // inner: c = D^{-1} L^{-1} r (FP32 operators), GMRES on A d~ = c, d = L^{-T} d~
        if ((e = to_solve_order(h, r, n, bnew, nc)) || (e = op_apply32(h, 1, bnew, xt, nc)) ||
            (e = op_apply32(h, 4, xt, cvec, nc)))
            break;
        cudaMemsetAsync(xt, 0, vec, st);
        std::vector<int> it(nc, 0);
        std::vector<double> rr(nc, 0.0);
        int s = gmres_batch(h, true, cvec, xt, nc, itol, restart, std::max(left, 1), it.data(), rr.data());
        if (s != HM_OK && s != HM_ENOCONV) {
            status = s;
            break;
        }
        for (int c = 0; c < nc; ++c) total[c] += it[c];
        if ((e = op_apply32(h, 2, xt, bnew, nc)) || (e = to_orig_order(h, bnew, r, n, nc))) break;
        HM_LAUNCH(h, K_VEC, k_add_to<<<nblk((int64_t)n * nc, 256), 256, 0, st>>>((int64_t)n * nc, r, xo));
    }
    if (!e && status == HM_OK) {
        cudaMemcpy2DAsync(dI, sizeof(double2) * ldi, xo, sizeof(double2) * n, sizeof(double2) * n, nc,
                          cudaMemcpyDeviceToDevice, st);
        e = cudaStreamSynchronize(st);
    }
    for (void *p : {(void *)b, (void *)xo, (void *)r, (void *)part, (void *)tmp, (void *)nrm, (void *)mask})
        h->arena.release(p, 0);
    if (e) {
        h->err = std::string("CUDA error in the refinement loop: ") + cudaGetErrorString(e);
        return HM_ECUDA;
    }
    if (status != HM_OK) return status;
    for (int c = 0; c < nc; ++c) {
        iters[c] = total[c];
        relres[c] = rel[c];
        if (!done[c]) status = HM_ENOCONV;
    }
    return status;
}

int gmres_solve(hm_ctx *h, const double2 *dV, int nrhs, int64_t ldv, double tol, int restart, int maxit, double2 *dI,
                int64_t ldi, int *iters, double *relres)
{
    const int n = h->plan.n;
    // columns solved in lockstep per batch: the FP32 operator takes 64 per sweep launch
    const int BATCH = h->opts.precision == 1 ? 64 : 16;
    cudaStream_t st = h->stream;
    double2 *bnew = nullptr, *cvec = nullptr, *xt = nullptr;
    int status = HM_OK;
    cudaError_t e;
    const int nb = std::min(nrhs, BATCH);
    if ((e = h->arena.alloc((void **)&bnew, sizeof(double2) * (size_t)n * nb)) ||
        (e = h->arena.alloc((void **)&cvec, sizeof(double2) * (size_t)n * nb)) ||
        (e = h->arena.alloc((void **)&xt, sizeof(double2) * (size_t)n * nb))) {
        h->arena.release(bnew, 0);
        h->arena.release(cvec, 0);
        h->err = "solve workspace allocation failed";
        return HM_ENOMEM;
    }
    cudaMemsetAsync(h->d_err, 0, sizeof(int), st);
    for (int c0 = 0; c0 < nrhs; c0 += BATCH) {
        const int nc = std::min(BATCH, nrhs - c0);
        int s = (h->opts.precision == 1)
                    ? solve_mixed(h, dV + c0 * ldv, nc, ldv, tol, restart, maxit, dI + c0 * ldi, ldi, iters + c0,
                                  relres + c0, bnew, cvec, xt)
                    : solve_fp64(h, dV + c0 * ldv, nc, ldv, tol, restart, maxit, dI + c0 * ldi, ldi, iters + c0,
                                 relres + c0, bnew, cvec, xt);
        if (s == HM_ENOCONV) status = HM_ENOCONV;
        else if (s != HM_OK) {
            status = s;
            break;
        }
    }
    if (status != HM_ECUDA && (e = cudaStreamSynchronize(st))) {
        status = HM_ECUDA;
        h->err = cudaGetErrorString(e);
    }
    int herr = 0;
    cudaMemcpy(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if ((status == HM_OK || status == HM_ENOCONV) && (herr & ERR_TIMEOUT)) {
        h->err = "device-side wait in a triangular sweep timed out";
        status = HM_ETIMEOUT;
    }
    h->arena.release(bnew, 0);
    h->arena.release(cvec, 0);
    h->arena.release(xt, 0);
    return status;
}

}  // namespace hm
