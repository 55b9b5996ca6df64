// Restarted GMRES (Sec. 5) on the preconditioned system of Eq. 28 and the mixed-precision
// refinement loop, run by a slot engine.  Every slot holds one right-hand side with its own
// Krylov space, restart cycle and refinement state; one engine tick advances every occupied
// slot by one step, and the operator applications of all slots that need the same operator
// in that tick are packed into one multi-column launch.  A slot freed by a finished solve
// takes a new right-hand side at the next tick (continuous batching), and solve() runs
// through the same engine.  Every per-column reduction has a fixed order that does not
// depend on the other columns of the pack, so a column's result is bitwise the same alone
// and in any mix.
//
// FP64 mode: GMRES on A x~ = c with the FP64 operator, stop at |g_{j+1}| <= tol ||c||.
// Mixed mode: an outer FP64 loop r = V - Z I (near blocks + far factors in FP64), inner
// GMRES on A d~ = D^{-1} L^{-1} r with the complex-FP32 operator, I += L^{-T} d~, until
// ||V - Z I|| <= tol ||V||.  The inner tolerance is clamp(max(0.6 tol ||V|| / ||r||, f),
// 1e-7, 0.5): f = 0.1 rho, rho = ||r|| / ||r_prev|| the contraction the last pass achieved
// (0.1 fill_tol before the first pass).  A pass cannot reduce the true residual by much more
// than the mismatch between the inner operator (FP32, fill-in blocks compressed to fill_tol)
// and Z allows, so solving the inner system further than that only costs iterations.
// Krylov vectors, Gram-Schmidt, Givens rotations and the refinement residual are FP64 in
// both modes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cplx.cuh"
#include "hm_internal.h"

namespace hm {

constexpr int DOT_CHUNK = 4096;
constexpr int MAX_OUTER = 40;

// Packed column p, vector i of a family: base + (idx[p] + i * istep) * n.
struct VRef {
    double2 *base;
    const int *idx;
    int64_t istep, n;
    __device__ __forceinline__ double2 *at(int p, int i = 0) const
    {
        return base + ((int64_t)idx[p] + (int64_t)i * istep) * n;
    }
};

// part[((p*ldp + i) * nchunk + chunk)] = sum over the chunk's rows of conj(basis_i) w, i < J[p]
// (J == nullptr: one vector)
__global__ void __launch_bounds__(256, 2) k_dots(int n, VRef basis, const int *J, VRef w, double2 *part, int nchunk,
                                                 int ldp)
{
    constexpr int QB = 16;   // vectors per pass (16 accumulators per thread: two CTAs per SM)
    __shared__ double2 red[8][QB + 1];
    const int chunk = blockIdx.x, p = blockIdx.y;
    const int lo = chunk * DOT_CHUNK, hi = min(n, lo + DOT_CHUNK);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int Jp = J ? J[p] : 1;
    const double2 *wc = w.at(p);
    for (int i0 = 0; i0 < Jp; i0 += QB) {
        const int ni = min(QB, Jp - i0);
        double2 acc[QB];
#pragma unroll
        for (int q = 0; q < QB; ++q) acc[q] = make_double2(0, 0);
        for (int row = lo + threadIdx.x; row < hi; row += blockDim.x) {
            double2 wv = wc[row];
#pragma unroll
            for (int q = 0; q < QB; ++q)
                if (q < ni) acc[q] = cjfma(basis.at(p, i0 + q)[row], wv, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < QB; ++q) {
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
            part[((int64_t)p * ldp + i0 + threadIdx.x) * nchunk + chunk] = v;
        }
        __syncthreads();
    }
}

// out[oidx[p]*ldo + i] = sum over chunks of part (fixed order), i < J[p]
__global__ void k_dots_final(int k, int ldp, const int *J, int nchunk, const double2 *part, double2 *out, int ldo,
                             const int *oidx)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k * ldp) return;
    const int p = e / ldp, i = e % ldp;
    if (i >= J[p]) return;
    double2 v = make_double2(0, 0);
    const double2 *q = part + (int64_t)e * nchunk;
    for (int c = 0; c < nchunk; ++c) {
        v.x += q[c].x;
        v.y += q[c].y;
    }
    out[(int64_t)oidx[p] * ldo + i] = v;
}

// out[oidx[p]] = sqrt(max(0, Re sum over chunks of part[p]))   (a 2-norm from k_dots with J = 1)
__global__ void k_norm_final(int k, int nchunk, const double2 *part, double *out, const int *oidx)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= k) return;
    double v = 0.0;
    const double2 *q = part + (int64_t)p * nchunk;
    for (int c = 0; c < nchunk; ++c) v += q[c].x;
    out[oidx[p]] = sqrt(fmax(0.0, v));
}

// w_p -= sum_{i<J[p]} h[hidx[p]*ldh + i] basis_i(p)
__global__ void k_axpy_basis(int n, int k, VRef basis, const int *J, const double2 *h, int ldh, const int *hidx,
                             VRef w)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * k) return;
    const int row = (int)(e % n), p = (int)(e / n);
    double2 *wp = w.at(p);
    double2 acc = wp[row];
    const double2 *hp = h + (int64_t)hidx[p] * ldh;
    for (int i = 0; i < J[p]; ++i) acc = cfms(hp[i], basis.at(p, i)[row], acc);
    wp[row] = acc;
}

// dst[idx[p]*ld + i] += src[idx[p]*ld + i], i < J[p]
__global__ void k_hfold(int k, int ldp, const int *J, const int *idx, const double2 *src, double2 *dst, int ld)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k * ldp) return;
    const int p = e / ldp, i = e % ldp;
    if (i >= J[p]) return;
    const int64_t o = (int64_t)idx[p] * ld + i;
    dst[o].x += src[o].x;
    dst[o].y += src[o].y;
}

// v_p = w_p / nrm[nidx[p]] (0 when the norm is 0)
__global__ void k_scale(int n, int k, const double *nrm, const int *nidx, VRef w, VRef v)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * k) return;
    const int row = (int)(e % n), p = (int)(e / n);
    const double r = nrm[nidx[p]];
    const double s = r > 0 ? 1.0 / r : 0.0;
    const double2 a = w.at(p)[row];
    v.at(p)[row] = make_double2(a.x * s, a.y * s);
}

// elementwise column ops on packed families: mode 0 dst = a; 1 dst = a - b; 2 dst += a; 3 dst = 0
__global__ void k_vec(int n, int k, int mode, VRef a, VRef b, VRef dst)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * k) return;
    const int row = (int)(e % n), p = (int)(e / n);
    double2 *d = dst.at(p) + row;
    if (mode == 3) {
        *d = make_double2(0, 0);
        return;
    }
    const double2 x = a.at(p)[row];
    if (mode == 0) *d = x;
    else if (mode == 1) {
        const double2 y = b.at(p)[row];
        *d = make_double2(x.x - y.x, x.y - y.y);
    } else
        *d = make_double2(d->x + x.x, d->y + x.y);
}

// GMRES small-matrix state per slot c (H: (m+1) x m column-major, ld m+1)
struct GState {
    double2 *H, *g, *sn, *y, *hj;
    double *cs, *nrm, *res, *wn;
    int *J;
};

// A new cycle for slot[p]: g = beta e_1 (beta = nrm[slot]), J = 0
__global__ void k_cycle_init(int k, int m, const int *slot, GState s)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k * (m + 1)) return;
    const int p = e / (m + 1), i = e % (m + 1), c = slot[p];
    s.g[(int64_t)c * (m + 1) + i] = make_double2(i == 0 ? s.nrm[c] : 0.0, 0.0);
    if (i == 0) s.J[c] = 0;
}

// Hessenberg column j = J[c] of slot c: h[0..j] from hj, h[j+1] = nrm; previous rotations,
// a new complex Givens rotation with real cosine, residual estimate |g_{j+1}|.
__global__ void k_givens(int k, int m, const int *slot, GState s)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= k) return;
    const int c = slot[p], j = s.J[c];
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

// y = H(1:J,1:J)^{-1} g(1:J) for slot[p] (back substitution)
__global__ void k_trisolve(int k, int m, const int *slot, GState s)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= k) return;
    const int c = slot[p];
    const double2 *H = s.H + (int64_t)c * (m + 1) * m;
    const double2 *g = s.g + (int64_t)c * (m + 1);
    double2 *y = s.y + (int64_t)c * m;
    const int J = s.J[c];
    for (int i = J - 1; i >= 0; --i) {
        double2 v = g[i];
        for (int q = i + 1; q < J; ++q) v = cfms(H[i + (int64_t)q * (m + 1)], y[q], v);
        double2 d = H[i + (int64_t)i * (m + 1)];
        double den = d.x * d.x + d.y * d.y;
        y[i] = make_double2((v.x * d.x + v.y * d.y) / den, (v.y * d.x - v.x * d.y) / den);
    }
}

// x_p += sum_{i<J[c]} y_c[i] basis_i(p), c = slot[p]
__global__ void k_update_x(int n, int k, const int *slot, const int *J, VRef basis, const double2 *yv, int ldy, VRef x)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * k) return;
    const int row = (int)(e % n), p = (int)(e / n), c = slot[p];
    double2 *xp = x.at(p);
    double2 acc = xp[row];
    for (int i = 0; i < J[c]; ++i) acc = cfma(yv[(int64_t)c * ldy + i], basis.at(p, i)[row], acc);
    xp[row] = acc;
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---- the engine ----------------------------------------------------------------------------
enum SlotState { FREE = 0, OUTER, RESTART, ARNOLDI, INNER_END, DONE };

struct Slot {
    int state = FREE;
    int j = 0, it = 0, it_in = 0, in_max = 0, outer = 0, maxit = 0, status = HM_OK;
    bool first = false, conv = false, reported = false;
    double tol = 0, itol = 0, bn = 0, cn = 0, rel = 0, prev_rel = 0;
};

struct Engine {
    hm_ctx *h = nullptr;
    int S = 0, m = 0, n = 0, nchunk = 0;
    bool fp32 = false;
    bool left = false;   // preconditioner applied from the left only (null field): x = x~
    // per-slot vectors (slot stride n): V, I (original order), FP64 residual, c and x~ (solve order)
    double2 *B = nullptr, *XO = nullptr, *R = nullptr, *C = nullptr, *XT = nullptr;
    double2 *Vb = nullptr;                   // Krylov basis: vector i of slot c at (i*S + c) * n
    double2 *PX = nullptr, *PY = nullptr, *PT = nullptr;   // packed operator operands
    double2 *part = nullptr, *h2 = nullptr;
    double *tmp = nullptr;                   // per-slot norms of the control phases
    GState s{};
    int *d_idx = nullptr, *h_idx = nullptr;  // index uploads (pinned ring, NIDX regions of S)
    int *d_iota = nullptr;
    int ring = 0;
    std::vector<void *> allocs;
    std::vector<Slot> sl;
    static constexpr int NIDX = 24;

    static size_t bytes(int n, int S, int m)
    {
        const int nchunk = (n + DOT_CHUNK - 1) / DOT_CHUNK;
        size_t b = sizeof(double2) * (size_t)n * S * (5 + (m + 1) + 3);
        b += sizeof(double2) * (size_t)nchunk * S * (m + 1);
        b += sizeof(double2) * (size_t)S * ((m + 1) * 2 + (m + 1) * m + (m + 1) + 2 * m);
        b += sizeof(double) * (size_t)S * (m + 5) + sizeof(int) * (size_t)S * (NIDX + 2);
        return b;
    }

    cudaError_t open(hm_ctx *hh, int slots, int restart)
    {
        h = hh;
        S = slots;
        m = restart;
        n = h->plan.n;
        nchunk = (n + DOT_CHUNK - 1) / DOT_CHUNK;
        fp32 = h->opts.precision == 1;
        left = h->opts.preconditioner == 2;
        sl.assign(S, Slot());
        cudaError_t e;
        auto A = [&](void **p, size_t b) {
            cudaError_t r = h->arena.alloc(p, b);
            if (r == cudaSuccess) allocs.push_back(*p);
            return r;
        };
        const size_t vs = sizeof(double2) * (size_t)n * S;
        if ((e = A((void **)&B, vs)) || (e = A((void **)&XO, vs)) || (e = A((void **)&R, vs)) ||
            (e = A((void **)&C, vs)) || (e = A((void **)&XT, vs)) || (e = A((void **)&Vb, vs * (m + 1))) ||
            (e = A((void **)&PX, vs)) || (e = A((void **)&PY, vs)) || (e = A((void **)&PT, vs)) ||
            (e = A((void **)&part, sizeof(double2) * (size_t)nchunk * S * (m + 1))) ||
            (e = A((void **)&h2, sizeof(double2) * (size_t)S * (m + 1))) ||
            (e = A((void **)&s.hj, sizeof(double2) * (size_t)S * (m + 1))) ||
            (e = A((void **)&s.H, sizeof(double2) * (size_t)S * (m + 1) * m)) ||
            (e = A((void **)&s.g, sizeof(double2) * (size_t)S * (m + 1))) ||
            (e = A((void **)&s.sn, sizeof(double2) * (size_t)S * m)) ||
            (e = A((void **)&s.y, sizeof(double2) * (size_t)S * m)) ||
            (e = A((void **)&s.cs, sizeof(double) * (size_t)S * m)) || (e = A((void **)&s.nrm, sizeof(double) * S)) ||
            (e = A((void **)&s.res, sizeof(double) * S)) || (e = A((void **)&s.wn, sizeof(double) * S)) ||
            (e = A((void **)&tmp, sizeof(double) * S)) || (e = A((void **)&s.J, sizeof(int) * S)) ||
            (e = A((void **)&d_idx, sizeof(int) * (size_t)S * NIDX)) || (e = A((void **)&d_iota, sizeof(int) * S)))
            return e;
        if ((e = cudaMallocHost((void **)&h_idx, sizeof(int) * (size_t)S * NIDX))) return e;
        std::vector<int> io(S);
        for (int c = 0; c < S; ++c) io[c] = c;
        if ((e = cudaMemcpyAsync(d_iota, io.data(), sizeof(int) * S, cudaMemcpyHostToDevice, h->stream))) return e;
        // the operator workspace for the widest pack
        if ((e = ensure_solve_workspace(h, std::min(S, fp32 ? 64 : 16)))) return e;
        return cudaStreamSynchronize(h->stream);
    }

    void close()
    {
        if (h) cudaStreamSynchronize(h->stream);
        for (void *p : allocs) h->arena.release(p, 0);
        allocs.clear();
        if (h_idx) cudaFreeHost(h_idx);
        h_idx = nullptr;
    }

    // copy an index list to the device (a fresh region of the ring; every tick ends synchronised)
    const int *upload(const std::vector<int> &v)
    {
        int *hp = h_idx + (size_t)ring * S, *dp = d_idx + (size_t)ring * S;
        ring = (ring + 1) % NIDX;
        std::memcpy(hp, v.data(), sizeof(int) * v.size());
        cudaMemcpyAsync(dp, hp, sizeof(int) * v.size(), cudaMemcpyHostToDevice, h->stream);
        return dp;
    }

    VRef ref(double2 *base, const int *idx, int64_t istep = 0) const { return VRef{base, idx, istep, n}; }
    VRef packed(double2 *base, int off = 0) const { return VRef{base, d_iota + off, 0, n}; }

    void vec(int mode, int k, VRef a, VRef b, VRef d)
    {
        HM_LAUNCH(h, K_VEC, k_vec<<<nblk((int64_t)n * k, 256), 256, 0, h->stream>>>(n, k, mode, a, b, d));
    }

    cudaError_t op(int code, const double2 *x, double2 *y, int k)
    {
        return fp32 ? op_apply32(h, code, x, y, k) : op_apply(h, code, x, y, k);
    }

    // 2-norms of k packed vectors v -> out[oidx[p]]
    void norms(int k, VRef v, double *out, const int *oidx)
    {
        HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, k), 256, 0, h->stream>>>(n, v, nullptr, v, part, nchunk, 1));
        HM_LAUNCH(h, K_SMALL, k_norm_final<<<nblk(k, 128), 128, 0, h->stream>>>(k, nchunk, part, out, oidx));
    }

    cudaError_t fetch(const double *d, std::vector<double> &hv)
    {
        hv.resize(S);
        cudaMemcpyAsync(hv.data(), d, sizeof(double) * S, cudaMemcpyDeviceToHost, h->stream);
        return cudaStreamSynchronize(h->stream);
    }

    std::vector<int> in_state(int st) const
    {
        std::vector<int> v;
        for (int c = 0; c < S; ++c)
            if (sl[c].state == st) v.push_back(c);
        return v;
    }

    // take a free slot for the right-hand side V (n entries, original order, host or device
    // memory); returns the slot, -2 when none is free, -1 on a CUDA error
    int submit(const double2 *V, double tol, int maxit)
    {
        for (int c = 0; c < S; ++c)
            if (sl[c].state == FREE) {
                cudaError_t e = cudaMemcpyAsync(B + (size_t)c * n, V, sizeof(double2) * n, cudaMemcpyDefault, h->stream);
                if (!e) e = cudaMemsetAsync(XO + (size_t)c * n, 0, sizeof(double2) * n, h->stream);
                if (e) return -1;
                Slot z;
                z.state = OUTER;
                z.tol = tol;
                z.maxit = maxit;
                sl[c] = z;
                return c;
            }
        return -2;
    }

    // the inner solve of these slots has ended: fold x~ back (mixed) or form the solution (FP64)
    cudaError_t inner_end(const std::vector<int> &E)
    {
        const int k = (int)E.size();
        const int *id = upload(E);
        cudaError_t e;
        vec(0, k, ref(XT, id), ref(XT, id), packed(PX));
        if (left) {   // x = x~
            if ((e = to_orig_order(h, PX, PT, n, k))) return e;
        } else if ((e = op(2, PX, PY, k)) || (e = to_orig_order(h, PY, PT, n, k)))
            return e;
        vec(fp32 ? 2 : 0, k, packed(PT), packed(PT), ref(XO, id));
        for (int c : E) {
            Slot &z = sl[c];
            if (fp32) {
                z.outer++;
                z.state = OUTER;
            } else {
                z.state = DONE;
                z.status = z.conv ? HM_OK : HM_ENOCONV;
            }
        }
        return cudaGetLastError();
    }

    // start (FP64) or continue (mixed) the refinement: residual, stopping test, c = D^{-1} L^{-1} r
    // (null field: c = L^{-T} D^{-1} L^{-1} r)
    cudaError_t outer(const std::vector<int> &O)
    {
        cudaError_t e;
        std::vector<int> go;
        if (fp32) {
            std::vector<int> O0, O1;
            for (int c : O) (sl[c].outer == 0 ? O0 : O1).push_back(c);
            if (!O1.empty()) {   // r = V - Z I in FP64
                const int k = (int)O1.size();
                const int *id = upload(O1);
                vec(0, k, ref(XO, id), ref(XO, id), packed(PX));
                if ((e = z_apply_orig(h, PX, PY, k))) return e;
                vec(1, k, ref(B, id), packed(PY), ref(R, id));
            }
            if (!O0.empty()) {
                const int *id = upload(O0);
                vec(0, (int)O0.size(), ref(B, id), ref(B, id), ref(R, id));
            }
            const int *id = upload(O);
            norms((int)O.size(), ref(R, id), tmp, id);
            std::vector<double> rn;
            if ((e = fetch(tmp, rn))) return e;
            for (int c : O) {
                Slot &z = sl[c];
                if (z.outer == 0) z.bn = rn[c];
                z.rel = z.bn > 0 ? rn[c] / z.bn : 0.0;
                if (z.rel <= z.tol || z.bn == 0.0) {
                    z.state = DONE;
                    z.status = HM_OK;
                } else if (z.it >= z.maxit || z.outer == MAX_OUTER) {
                    z.state = DONE;
                    z.status = HM_ENOCONV;
                } else {
                    // ask the inner solve for a little more than what is still missing, but not
                    // for much more than one pass can gain (the contraction of the last pass, or
                    // the fill compression tolerance before the first)
                    const double rho = z.outer == 0 ? h->opts.fill_tol : std::min(1.0, z.rel / z.prev_rel);
                    z.itol = std::min(0.5, std::max({1e-7, 0.6 * z.tol / z.rel, 0.1 * rho}));
                    z.prev_rel = z.rel;
                    z.in_max = std::max(z.maxit - z.it, 1);
                    go.push_back(c);
                }
            }
        } else {
            go = O;
            for (int c : O) {
                sl[c].itol = sl[c].tol;
                sl[c].in_max = sl[c].maxit;
            }
        }
        if (go.empty()) return cudaSuccess;
        const int k = (int)go.size();
        const int *id = upload(go);
        vec(0, k, ref(fp32 ? R : B, id), ref(B, id), packed(PX));
        if ((e = to_solve_order(h, PX, n, PY, k)) || (e = op(1, PY, PT, k))) return e;
        if (left ? ((e = op(4, PT, PY, k)) || (e = op(2, PY, PX, k))) : (bool)(e = op(4, PT, PX, k))) return e;
        vec(0, k, packed(PX), packed(PX), ref(C, id));
        vec(3, k, packed(PX), packed(PX), ref(XT, id));
        norms(k, ref(C, id), tmp, id);
        std::vector<double> cn;
        if ((e = fetch(tmp, cn))) return e;
        for (int c : go) {
            Slot &z = sl[c];
            z.cn = cn[c];
            z.it_in = 0;
            z.first = true;
            z.conv = false;
            z.state = RESTART;
        }
        return cudaSuccess;
    }

    // true residual c - A x~ at a restart (c itself at the first), stopping test, v_0 = r / beta
    cudaError_t restart(const std::vector<int> &Rs)
    {
        cudaError_t e;
        std::vector<int> Rn, Rf;
        for (int c : Rs) {
            Slot &z = sl[c];
            if (z.cn == 0.0) {   // zero right-hand side of the inner system
                z.conv = true;
                if (!fp32) z.rel = 0.0;
                z.state = INNER_END;
                continue;
            }
            (z.first ? Rf : Rn).push_back(c);
        }
        std::vector<int> P(Rn);
        P.insert(P.end(), Rf.begin(), Rf.end());
        if (P.empty()) return cudaSuccess;
        const int k = (int)P.size(), k1 = (int)Rn.size();
        const int *id = upload(P);
        if (k1) {
            vec(0, k1, ref(XT, id), ref(XT, id), packed(PX));
            if ((e = op(0, PX, PY, k1))) return e;
            vec(1, k1, ref(C, id), packed(PY), packed(PY));
        }
        if (k > k1) vec(0, k - k1, ref(C, id + k1), ref(C, id + k1), packed(PY, k1));
        norms(k, packed(PY), s.nrm, id);
        std::vector<double> beta;
        if ((e = fetch(s.nrm, beta))) return e;
        std::vector<int> G, Gp;
        for (int p = 0; p < k; ++p) {
            const int c = P[p];
            Slot &z = sl[c];
            const double rr = beta[c] / z.cn;
            if (!fp32) z.rel = rr;
            if (beta[c] <= z.itol * z.cn) {
                z.conv = true;
                z.state = INNER_END;
            } else if (z.it_in >= z.in_max) {
                z.state = INNER_END;
            } else {
                G.push_back(c);
                Gp.push_back(p);
            }
        }
        if (G.empty()) return cudaSuccess;
        const int kg = (int)G.size();
        const int *gid = upload(G), *gp = upload(Gp);
        HM_LAUNCH(h, K_VEC,
                  k_scale<<<nblk((int64_t)n * kg, 256), 256, 0, h->stream>>>(n, kg, s.nrm, gid, ref(PY, gp),
                                                                              ref(Vb, gid)));
        HM_LAUNCH(h, K_SMALL, k_cycle_init<<<nblk(kg * (m + 1), 128), 128, 0, h->stream>>>(kg, m, gid, s));
        for (int c : G) {
            sl[c].j = 0;
            sl[c].first = false;
            sl[c].state = ARNOLDI;
        }
        return cudaGetLastError();
    }

    // one Arnoldi step (CGS2) and Givens update for every slot in a cycle
    cudaError_t arnoldi(const std::vector<int> &Ar)
    {
        cudaError_t e;
        const int k = (int)Ar.size();
        std::vector<int> Jp(k), vin(k), vout(k);
        for (int p = 0; p < k; ++p) {
            const int c = Ar[p], j = sl[c].j;
            Jp[p] = j + 1;
            vin[p] = j * S + c;
            vout[p] = (j + 1) * S + c;
        }
        const int *id = upload(Ar), *J = upload(Jp), *vi = upload(vin), *vo = upload(vout);
        const VRef basis = ref(Vb, id, S), w = packed(PY);
        cudaStream_t st = h->stream;
        vec(0, k, ref(Vb, vi), ref(Vb, vi), packed(PX));
        if ((e = op(0, PX, PY, k))) return e;
        norms(k, w, s.wn, id);   // ||w|| before orthogonalisation (happy-breakdown reference)
        // CGS2: h = V^H w, w -= V h, twice; coefficients accumulated in hj
        HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, k), 256, 0, st>>>(n, basis, J, w, part, nchunk, m + 1));
        HM_LAUNCH(h, K_SMALL,
                  k_dots_final<<<nblk(k * (m + 1), 128), 128, 0, st>>>(k, m + 1, J, nchunk, part, s.hj, m + 1, id));
        HM_LAUNCH(h, K_VEC,
                  k_axpy_basis<<<nblk((int64_t)n * k, 256), 256, 0, st>>>(n, k, basis, J, s.hj, m + 1, id, w));
        HM_LAUNCH(h, K_DOTS, k_dots<<<dim3(nchunk, k), 256, 0, st>>>(n, basis, J, w, part, nchunk, m + 1));
        HM_LAUNCH(h, K_SMALL,
                  k_dots_final<<<nblk(k * (m + 1), 128), 128, 0, st>>>(k, m + 1, J, nchunk, part, h2, m + 1, id));
        HM_LAUNCH(h, K_VEC, k_axpy_basis<<<nblk((int64_t)n * k, 256), 256, 0, st>>>(n, k, basis, J, h2, m + 1, id, w));
        HM_LAUNCH(h, K_SMALL, k_hfold<<<nblk(k * (m + 1), 128), 128, 0, st>>>(k, m + 1, J, id, h2, s.hj, m + 1));
        // h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
        norms(k, w, s.nrm, id);
        HM_LAUNCH(h, K_VEC, k_scale<<<nblk((int64_t)n * k, 256), 256, 0, st>>>(n, k, s.nrm, id, w, ref(Vb, vo)));
        HM_LAUNCH(h, K_SMALL, k_givens<<<nblk(k, 64), 64, 0, st>>>(k, m, id, s));
        std::vector<double> res(S), wpre(S), wn(S);
        cudaMemcpyAsync(res.data(), s.res, sizeof(double) * S, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(wpre.data(), s.wn, sizeof(double) * S, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(wn.data(), s.nrm, sizeof(double) * S, cudaMemcpyDeviceToHost, st);
        if ((e = cudaStreamSynchronize(st))) return e;
        std::vector<int> F;
        for (int c : Ar) {
            Slot &z = sl[c];
            z.it++;
            z.it_in++;
            const bool brk = wn[c] <= 1e-14 * wpre[c];
            if (!fp32) z.rel = res[c] / z.cn;
            if (res[c] <= z.itol * z.cn || brk) {
                z.conv = true;
                z.state = INNER_END;
                F.push_back(c);
            } else if (z.it_in >= z.in_max) {
                z.state = INNER_END;
                F.push_back(c);
            } else if (z.j + 1 == m) {
                z.state = RESTART;
                F.push_back(c);
            } else
                z.j++;
        }
        if (F.empty()) return cudaSuccess;
        // end of the cycle: x~ += V y
        const int kf = (int)F.size();
        const int *fid = upload(F);
        HM_LAUNCH(h, K_SMALL, k_trisolve<<<nblk(kf, 64), 64, 0, st>>>(kf, m, fid, s));
        HM_LAUNCH(h, K_VEC,
                  k_update_x<<<nblk((int64_t)n * kf, 256), 256, 0, st>>>(n, kf, fid, s.J, ref(Vb, fid, S), s.y, m,
                                                                          ref(XT, fid)));
        return cudaGetLastError();
    }

    // one tick: every occupied slot advances by one step; slots that finished are appended to fin
    int tick(std::vector<int> &fin)
    {
        cudaError_t e = cudaSuccess;
        std::vector<int> L;
        if (!(L = in_state(INNER_END)).empty() && (e = inner_end(L))) return fail(e);
        if (!(L = in_state(OUTER)).empty() && (e = outer(L))) return fail(e);
        if (!(L = in_state(RESTART)).empty() && (e = restart(L))) return fail(e);
        if (!(L = in_state(ARNOLDI)).empty() && (e = arnoldi(L))) return fail(e);
        // slots that reached INNER_END in this tick with FP64 finish now (no further operator)
        if (!fp32 && !(L = in_state(INNER_END)).empty() && (e = inner_end(L))) return fail(e);
        if ((e = cudaStreamSynchronize(h->stream))) return fail(e);
        int herr = 0;
        cudaMemcpy(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (herr & ERR_TIMEOUT) {
            h->err = "device-side wait in a triangular sweep timed out";
            return HM_ETIMEOUT;
        }
        for (int c = 0; c < S; ++c)
            if (sl[c].state == DONE && !sl[c].reported) {
                sl[c].reported = true;
                fin.push_back(c);
            }
        return HM_OK;
    }

    int fail(cudaError_t e)
    {
        h->err = std::string("CUDA error in the GMRES engine: ") + cudaGetErrorString(e);
        return HM_ECUDA;
    }

    int active() const
    {
        int a = 0;
        for (const Slot &z : sl) a += (z.state != FREE && z.state != DONE);
        return a;
    }
};

int gmres_solve(hm_ctx *h, const double2 *dV, int nrhs, int64_t ldv, double tol, int restart, int maxit, double2 *dI,
                int64_t ldi, int *iters, double *relres)
{
    // slots of the engine: the FP32 operator takes 64 columns per sweep launch, the FP64 one 16
    const int width = h->opts.precision == 1 ? 64 : 16;
    Engine E;
    cudaError_t e;
    cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
    if ((e = E.open(h, std::min(nrhs, width), restart))) {
        E.close();
        h->err = std::string("solve workspace: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA;
    }
    const int n = h->plan.n;
    std::vector<int> col(E.S, -1);
    int next = 0, done = 0, status = HM_OK;
    while (done < nrhs && status != HM_ECUDA && status != HM_ETIMEOUT) {
        while (next < nrhs) {
            const int c = E.submit(dV + (size_t)next * ldv, tol, maxit);
            if (c == -2) break;
            if (c < 0) {
                status = E.fail(cudaGetLastError());
                break;
            }
            col[c] = next++;
        }
        if (status == HM_ECUDA) break;
        std::vector<int> fin;
        const int s = E.tick(fin);
        if (s != HM_OK) {
            status = s;
            break;
        }
        for (int c : fin) {
            cudaMemcpyAsync(dI + (size_t)col[c] * ldi, E.XO + (size_t)c * n, sizeof(double2) * n,
                            cudaMemcpyDeviceToDevice, h->stream);
            iters[col[c]] = E.sl[c].it;
            relres[col[c]] = E.sl[c].rel;
            if (E.sl[c].status != HM_OK) status = E.sl[c].status;
            E.sl[c] = Slot();
            ++done;
        }
    }
    if ((e = cudaStreamSynchronize(h->stream)) && status != HM_ECUDA) status = E.fail(e);
    E.close();
    return status;
}

}  // namespace hm

// ---- continuous-batching C-ABI ----------------------------------------------------------------
struct hm_batch_s {
    hm_ctx *h = nullptr;
    hm::Engine E;
};

extern "C" {

int hm_batch_bytes(hm_handle h, int32_t slots, int32_t restart, int64_t *bytes)
{
    if (!h || slots < 1 || slots > 1024 || restart < 1 || !bytes) return HM_EINVAL;
    *bytes = (int64_t)hm::Engine::bytes(h->plan.n ? h->plan.n : h->n, slots, restart);
    return HM_OK;
}

int hm_batch_open(hm_handle h, int32_t slots, int32_t restart, hm_batch *out)
{
    if (!h || !out || slots < 1 || slots > 1024 || restart < 1) return HM_EINVAL;
    *out = nullptr;
    if (!h->setup_done || h->batch_open) {
        h->err = h->batch_open ? "a batch is already open on this handle" : "batch before precond_setup";
        return HM_ESTATE;
    }
    cudaSetDevice(h->dev);
    hm_batch b = new hm_batch_s;
    b->h = h;
    cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
    cudaError_t e = b->E.open(h, slots, restart);
    if (e) {
        b->E.close();
        delete b;
        h->err = std::string("batch workspace: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA;
    }
    h->batch_open = true;
    *out = b;
    return HM_OK;
}

int hm_batch_submit(hm_batch b, const hm_c128 *V, double tol, int32_t maxit, int32_t *slot)
{
    if (!b || !V || !slot || maxit < 0 || !(tol >= 0)) return HM_EINVAL;
    cudaSetDevice(b->h->dev);
    const int c = b->E.submit((const double2 *)V, tol, maxit);
    *slot = c;
    if (c == -2) return HM_EBUSY;
    if (c < 0) return b->E.fail(cudaGetLastError());
    return HM_OK;
}

int hm_batch_step(hm_batch b, int32_t *finished, int32_t *nfinished, int32_t *nactive)
{
    if (!b || !finished || !nfinished) return HM_EINVAL;
    cudaSetDevice(b->h->dev);
    std::vector<int> fin;
    const int s = b->E.tick(fin);
    for (size_t i = 0; i < fin.size(); ++i) finished[i] = fin[i];
    *nfinished = (int32_t)fin.size();
    if (nactive) *nactive = b->E.active();
    return s;
}

int hm_batch_result(hm_batch b, int32_t slot, hm_c128 *I, int32_t *iters, double *relres)
{
    if (!b || slot < 0 || slot >= b->E.S || !I) return HM_EINVAL;
    hm::Slot &z = b->E.sl[slot];
    if (z.state != hm::DONE) {
        b->h->err = "hm_batch_result: the slot holds no finished solve";
        return HM_ESTATE;
    }
    cudaSetDevice(b->h->dev);
    const int n = b->E.n;
    cudaError_t e = cudaMemcpyAsync(I, b->E.XO + (size_t)slot * n, sizeof(double2) * n, cudaMemcpyDefault,
                                    b->h->stream);
    if (!e) e = cudaStreamSynchronize(b->h->stream);
    if (e) return b->E.fail(e);
    if (iters) *iters = z.it;
    if (relres) *relres = z.rel;
    const int st = z.status;
    z = hm::Slot();
    return st;
}

int hm_batch_close(hm_batch b)
{
    if (!b) return HM_EINVAL;
    cudaSetDevice(b->h->dev);
    b->E.close();
    b->h->batch_open = false;
    delete b;
    return HM_OK;
}

}  // extern "C"
