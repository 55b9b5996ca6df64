// The H-matrix the preconditioned solve takes as input, computed on the GPU from the mesh:
// Galerkin EFIE entries of RWG functions (Sec. 2, Eq. 7) for dense blocks, and partially
// pivoted ACA with SVD re-compression (Sec. 2, Eqs. 9-10) for admissible blocks.  This is the
// matrix setup whose time is t_sm in the cost model of Sec. 5.2 (Eq. 46).
//
// Eq. 7 with the time factor e^{+jwt}, G = e^{-jkR}/R, w mu = k eta0 and 1/(w eps) = eta0 / k:
//   Z(m, n) = (j k eta0 / 4 pi) l_m l_n sum_{s,t} +-(1 / A_p A_q) [ <<(r - v_m).(r' - v_n) G>> / 4
//                                                                  - <<G>> / k^2 ],
// f_n = +-(l_n / 2 A) (r - v) on its two triangles (v the free vertex), div f_n = +-l_n / A,
// the sign + when s and t are both T+ or both T-.  With the integrals of a triangle pair
// (p test, q source) I0 = <<G>>, Ir = <<G r>>, Irp = <<G r'>>, Irr = <<G r.r'>>, the first
// inner product is Irr - v_n.Ir - v_m.Irp + v_m.v_n I0.
//
// Quadrature: Radon's 7-point degree-5 rule on both triangles.  A close pair (same triangle,
// or centroids nearer than max(r_abs, c_rel (h_p + h_q) / 2), h the longest edge) uses
// singularity extraction, G = (e^{-jkR} - 1)/R + 1/R: the smooth part by the 7 x 7 rule (limit
// -jk at R = 0), the 1/R and rho/R source integrals in closed form (the potential integrals of
// Wilton et al., IEEE TAP 1984, and Graglia, IEEE TAP 1993) at each test point.
//
// GPU layout: a triangle carries up to three RWG functions and an RWG function two triangles,
// so the entries of a block share their triangle-pair integrals.  Per block, the distinct
// triangles of its rows and of its columns are listed on the host; the kernel first integrates
// every (row triangle, column triangle) pair once (8 complex values, stored value-major so that
// the stores coalesce), then assembles each entry from its four pairs: about a fifth of the
// pair integrations of an entry-by-entry fill on leaf blocks.
//
// ACA (Eqs. 9-10), one CTA per block: first row = local row 0; column pivot = argmax of the
// residual row's moduli over unused columns (lowest index on ties); next row = argmax |u_k|
// over unused rows; a zero residual row moves to the lowest unused row; stop when
// |u_k| |v_k| <= eps ||A_k||_F with the recursive norm update.  A row touches only
// 2 x (column triangles) pairs, so rows and columns are integrated one test point per thread
// (7 threads per pair).  The rank is capped at min(m, n, floor(m n / (m + n)) + 1, 256); a
// block that reaches the cap without meeting the stop rule is filled densely.  Re-compression
// (one CTA per block): U = Q_U R_U and V = Q_V R_V by Gram-Schmidt applied twice, the one-sided
// Jacobi SVD of R_U R_V^T (in shared memory up to rank 64, in global scratch above), truncation
// to the smallest rank whose singular-value tail is <= eps times the Frobenius norm; a block
// whose truncated factors are not smaller than the block (r (m + n) >= m n) is filled densely.
// Dense blocks are cut into tiles of at most 128 x 64 RWG functions, one CTA each.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "cplx.cuh"
#include "hm_internal.h"
#include "jacobi.cuh"

namespace hm {
namespace {

constexpr int NQ = 7;
constexpr int NPV = 8;         // values per triangle pair: I0, Ir (3), Irp (3), Irr
constexpr int ACA_RCAP = 256;  // rank cap of the on-device ACA
constexpr int RC_SMALL = 64;   // ranks re-compressed with their work arrays in shared memory
constexpr int NT = 256;        // threads per CTA
constexpr size_t CHUNK_BYTES = size_t(1) << 30;   // default device scratch per launch
constexpr int NONE = 0x7fffffff;
constexpr int FILL_TR = 128, FILL_TC = 64;   // largest dense tile (RWG rows x columns) of one CTA

__constant__ double c_qw[NQ];

// Radon's degree-5 rule on a triangle: the centroid and two orbits of three points
void radon_rule(double w[NQ], double b[NQ][3])
{
    const double s = std::sqrt(15.0);
    const double a1 = (6.0 - s) / 21.0, a2 = (6.0 + s) / 21.0;
    const double w1 = (155.0 - s) / 1200.0, w2 = (155.0 + s) / 1200.0;
    w[0] = 9.0 / 40.0;
    b[0][0] = b[0][1] = b[0][2] = 1.0 / 3.0;
    for (int i = 0; i < 3; ++i) {
        w[1 + i] = w1;
        w[4 + i] = w2;
        for (int j = 0; j < 3; ++j) {
            b[1 + i][j] = (i == j) ? 1.0 - 2.0 * a1 : a1;
            b[4 + i][j] = (i == j) ? 1.0 - 2.0 * a2 : a2;
        }
    }
}

struct Mesh {
    const double *tv;     // [nt][9] vertices
    const double *tn;     // [nt][3] unit normal
    const double *ta;     // [nt] area
    const double *tc;     // [nt][3] centroid
    const double *th;     // [nt] longest edge
    const double *tq;     // [nt][NQ][3] quadrature points
    const int *btri;      // [nb][2] T+, T-
    const double *bfree;  // [nb][2][3] free vertices
    const double *blen;   // [nb] edge length
    double k, eta0, r_abs, c_rel;
};

// the blocks of one call: RWG rows / columns and their distinct triangles
struct Blocks {
    const int64_t *rptr, *cptr;    // [nblk + 1]
    const int *ridx, *cidx;        // RWG indices
    const int64_t *trptr, *tcptr;  // [nblk + 1]
    const int *tridx, *tcidx;      // distinct triangles of the rows / columns
    const int *rloc, *cloc;        // [2 per row / column RWG] local index of its T+ and T-
};

struct V3 {
    double x, y, z;
};
__device__ __forceinline__ V3 ld3(const double *p) { return V3{p[0], p[1], p[2]}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return V3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b)
{
    return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csc(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

// S0 = int_T 1/|r - r'| ds' and Sv = int_T (r' - rho)/|r - r'| ds' over the flat triangle P
// (unit normal n), rho the projection of r on its plane.  Per edge a -> b with unit tangent l
// and in-plane outward normal u = l x n, h = n.(r - P0): l+- = (b|a - rho).l,
// p0 = (a - rho).u, R0^2 = p0^2 + h^2, R+- = sqrt(l+-^2 + R0^2), f = log((R+ + l+)/(R- + l-))
// (written so that neither factor cancels):
//   S0 = sum p0 f - |h| sum [atan(p0 l+ / (R0^2 + |h| R+)) - atan(p0 l- / (R0^2 + |h| R-))],
//   Sv = sum u (R0^2 f + l+ R+ - l- R-) / 2.
__device__ void potential(const double *P, V3 n, V3 r, double &S0, V3 &Sv)
{
    const double h = dot(n, r - ld3(P)), ah = fabs(h);
    const V3 rho = r - h * n;
    S0 = 0.0;
    Sv = V3{0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
        const V3 a = ld3(P + 3 * i), b = ld3(P + 3 * ((i + 1) % 3));
        const V3 e = b - a;
        const double le = sqrt(dot(e, e));
        const V3 l = (1.0 / le) * e;
        const V3 u = cross(l, n);
        const double lp = dot(b - rho, l), lm = dot(a - rho, l), p0 = dot(a - rho, u);
        const double R02 = p0 * p0 + h * h;
        const double Rp = sqrt(lp * lp + R02), Rm = sqrt(lm * lm + R02);
        double f = 0.0;
        if (R02 > 1e-24 * le * le)   // rho is not on the edge's line
            f = (lp + lm >= 0.0) ? log((Rp + lp) / (Rm + lm)) : log((Rm - lm) / (Rp - lp));
        S0 += p0 * f;
        if (ah > 0.0 && p0 != 0.0) S0 -= ah * (atan(p0 * lp / (R02 + ah * Rp)) - atan(p0 * lm / (R02 + ah * Rm)));
        const double g = 0.5 * (R02 * f + lp * Rp - lm * Rm);
        Sv = V3{Sv.x + g * u.x, Sv.y + g * u.y, Sv.z + g * u.z};
    }
}

__device__ __forceinline__ bool close_pair(const Mesh &M, int p, int q)
{
    const V3 dc = ld3(M.tc + 3 * p) - ld3(M.tc + 3 * q);
    double thr = 0.5 * M.c_rel * (M.th[p] + M.th[q]);
    if (thr < M.r_abs) thr = M.r_abs;
    return p == q || sqrt(dot(dc, dc)) < thr;
}

// test point a of triangle p against source triangle q: o[v] += w_a times the integral over q
// (its area included) of G, G r_a, G r', G r_a.r' (value order I0, Ir, Irp, Irr); the sum over
// a is the pair's integral divided by the test triangle's area
__device__ void point_terms(const Mesh &M, int p, int q, int a, bool close, double2 o[NPV])
{
    const double k = M.k;
    const V3 ra = ld3(M.tq + (p * NQ + a) * 3);
    double2 s0 = make_double2(0.0, 0.0), sv[3] = {s0, s0, s0};
    for (int b = 0; b < NQ; ++b) {
        const V3 rb = ld3(M.tq + (q * NQ + b) * 3);
        const V3 d = ra - rb;
        const double R = sqrt(dot(d, d));
        double2 g;
        if (close) {   // (e^{-jkR} - 1)/R = (-2 sin^2(kR/2) - j sin kR)/R, -jk at R = 0
            if (R < 1e-14) {
                g = make_double2(0.0, -k);
            } else {
                const double sh = sin(0.5 * k * R);
                g = make_double2(-2.0 * sh * sh / R, -sin(k * R) / R);
            }
        } else {
            double sn, cs;
            sincos(k * R, &sn, &cs);
            g = make_double2(cs / R, -sn / R);
        }
        const double2 wg = csc(c_qw[b], g);
        s0 = cadd(s0, wg);
        sv[0] = cadd(sv[0], csc(rb.x, wg));
        sv[1] = cadd(sv[1], csc(rb.y, wg));
        sv[2] = cadd(sv[2], csc(rb.z, wg));
    }
    const double Aq = M.ta[q];
    s0 = csc(Aq, s0);
    for (int j = 0; j < 3; ++j) sv[j] = csc(Aq, sv[j]);
    if (close) {   // the 1/R part in closed form
        const V3 nq = ld3(M.tn + 3 * q);
        double S0;
        V3 Sv;
        potential(M.tv + 9 * q, nq, ra, S0, Sv);
        const V3 rho = ra - dot(nq, ra - ld3(M.tv + 9 * q)) * nq;
        s0.x += S0;
        sv[0].x += Sv.x + rho.x * S0;
        sv[1].x += Sv.y + rho.y * S0;
        sv[2].x += Sv.z + rho.z * S0;
    }
    const double wa = c_qw[a];
    const double rav[3] = {ra.x, ra.y, ra.z};
    o[0] = cadd(o[0], csc(wa, s0));
    double2 dv = make_double2(0.0, 0.0);
    for (int j = 0; j < 3; ++j) {
        o[1 + j] = cadd(o[1 + j], csc(wa * rav[j], s0));
        o[4 + j] = cadd(o[4 + j], csc(wa, sv[j]));
        dv = cadd(dv, csc(rav[j], sv[j]));
    }
    o[7] = cadd(o[7], csc(wa, dv));
}

__device__ void pair_values(const Mesh &M, int p, int q, double2 o[NPV])
{
    for (int v = 0; v < NPV; ++v) o[v] = make_double2(0.0, 0.0);
    const bool close = close_pair(M, p, q);
    for (int a = 0; a < NQ; ++a) point_terms(M, p, q, a, close, o);
}

// Z(m, n) of Eq. 7 from the pair values (point_terms summed over the test points) of
// (T_s of m, T_t of n): pv(s, t, v) returns value v
template <class PV> __device__ double2 assemble(const Mesh &M, int m, int n, PV pv)
{
    double2 zA = make_double2(0.0, 0.0), zP = zA;
    for (int s = 0; s < 2; ++s) {
        const V3 vm = ld3(M.bfree + 6 * m + 3 * s);
        for (int t = 0; t < 2; ++t) {
            const V3 vn = ld3(M.bfree + 6 * n + 3 * t);
            const double sg = (s == t) ? 1.0 : -1.0;
            // pair integral / (A_p A_q) = (pair value, which carries A_q but not A_p) / A_q
            const double inv = 1.0 / M.ta[M.btri[2 * n + t]];
            double2 dt = pv(s, t, 7);
            dt = cadd(dt, csc(-vn.x, pv(s, t, 1)));
            dt = cadd(dt, csc(-vn.y, pv(s, t, 2)));
            dt = cadd(dt, csc(-vn.z, pv(s, t, 3)));
            dt = cadd(dt, csc(-vm.x, pv(s, t, 4)));
            dt = cadd(dt, csc(-vm.y, pv(s, t, 5)));
            dt = cadd(dt, csc(-vm.z, pv(s, t, 6)));
            const double2 i0 = pv(s, t, 0);
            dt = cadd(dt, csc(dot(vm, vn), i0));
            zA = cadd(zA, csc(sg * 0.25 * inv, dt));
            zP = cadd(zP, csc(sg * inv, i0));
        }
    }
    const double k = M.k, c = k * M.eta0 / (4.0 * M_PI) * M.blen[m] * M.blen[n];
    const double2 z = cadd(zA, csc(-1.0 / (k * k), zP));
    return make_double2(-c * z.y, c * z.x);   // j c z
}

// ---------------------------------------------------------------------------------------
// dense tiles: one CTA per tile x of B (at most FILL_TR x FILL_TC RWG functions), its pair
// scratch at pairs + poff[x] (NPV x ntr x ntc, value-major), its entry (i, j) at
// out[ooff[x] + i + j ld[x]] (a column-major piece of its block)
__global__ void __launch_bounds__(NT, 2) k_efie_fill(Mesh M, Blocks B, int ntile, const int64_t *poff, double2 *pairs,
                                                     const int64_t *ooff, const int *ld, double2 *out)
{
    const int b = blockIdx.x;
    if (b >= ntile) return;
    const int m = (int)(B.rptr[b + 1] - B.rptr[b]), n = (int)(B.cptr[b + 1] - B.cptr[b]);
    const int ntr = (int)(B.trptr[b + 1] - B.trptr[b]), ntc = (int)(B.tcptr[b + 1] - B.tcptr[b]);
    const int *Tr = B.tridx + B.trptr[b], *Tc = B.tcidx + B.tcptr[b];
    const int64_t P = (int64_t)ntr * ntc;
    double2 *pb = pairs + poff[b];
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
        double2 o[NPV];
        pair_values(M, Tr[i % ntr], Tc[i / ntr], o);
        for (int v = 0; v < NPV; ++v) pb[v * P + i] = o[v];
    }
    __syncthreads();
    const int *R = B.ridx + B.rptr[b], *C = B.cidx + B.cptr[b];
    const int *rl = B.rloc + 2 * B.rptr[b], *cl = B.cloc + 2 * B.cptr[b];
    double2 *ob = out + ooff[b];
    const int64_t ldo = ld[b];
    for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        const int r0 = rl[2 * i], r1 = rl[2 * i + 1], c0 = cl[2 * j], c1 = cl[2 * j + 1];
        ob[i + j * ldo] = assemble(M, R[i], C[j], [&](int s, int t, int v) {
            return pb[v * P + (int64_t)(s ? r1 : r0) + (int64_t)ntr * (t ? c1 : c0)];
        });
    }
}

// blocks whose rows and columns are the same list (x-th at out + off[x], mm[x] x mm[x]): the
// lower triangle becomes a copy of the upper one, so the block is exactly symmetric
__global__ void k_mirror(int nsym, const int64_t *off, const int *mm, double2 *out)
{
    const int x = blockIdx.x;
    if (x >= nsym) return;
    const int64_t m = mm[x];
    double2 *o = out + off[x];
    for (int64_t e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int64_t i = e % m, j = e / m;
        if (i > j) o[i + j * m] = o[j + i * m];
    }
}

// ---------------------------------------------------------------------------------------
// block reductions (every thread calls them; every thread gets the result)
__device__ double block_sum(double v, double *s_red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    return t;
}

// largest v, ties to the lowest index; (v, i) = (-1, NONE) for none
__device__ void block_argmax(double &v, int &i, double *s_v, int *s_i)
{
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        s_v[threadIdx.x >> 5] = v;
        s_i[threadIdx.x >> 5] = i;
    }
    __syncthreads();
    v = s_v[0];
    i = s_i[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (s_v[w] > v || (s_v[w] == v && s_i[w] < i)) {
            v = s_v[w];
            i = s_i[w];
        }
}

struct AcaWork {
    const int64_t *poff, *uoff, *voff, *foff;   // per block (global index), relative to its chunk
    double2 *pairs, *U, *V;
    unsigned char *flags;
    int *rank;   // per block (global index): ACA rank (-1: cap reached), then the final rank
};

// partial pair values of one residual row (or column): thread x integrates test point x % 7
// of pair j = x / 7, (tp[j % tps], tq[j / tps]); value v of pair j is the sum of its 7
// partials at pw[(v * np + j) * 7 + a]
__device__ void line_pairs(const Mesh &M, int np, const int *tp, int tps, const int *tq, double2 *pw)
{
    for (int x = threadIdx.x; x < np * NQ; x += blockDim.x) {
        const int j = x / NQ, a = x % NQ;
        const int p = tp[j % tps], q = tq[j / tps];
        double2 o[NPV];
        for (int v = 0; v < NPV; ++v) o[v] = make_double2(0.0, 0.0);
        point_terms(M, p, q, a, close_pair(M, p, q), o);
        for (int v = 0; v < NPV; ++v) pw[((int64_t)v * np + j) * NQ + a] = o[v];
    }
}
__device__ __forceinline__ double2 partial_sum(const double2 *pw, int np, int j, int v)
{
    const double2 *s = pw + ((int64_t)v * np + j) * NQ;
    double2 t = s[0];
    for (int a = 1; a < NQ; ++a) t = cadd(t, s[a]);
    return t;
}

__device__ __forceinline__ int aca_cap(int m, int n)
{
    return min(min(min(m, n), (int)((int64_t)m * n / (m + n)) + 1), ACA_RCAP);
}

// partially pivoted ACA of block b0 + blockIdx.x (Eqs. 9-10): U (m x cap), V (n x cap)
__global__ void __launch_bounds__(NT, 2) k_efie_aca(Mesh M, Blocks B, int b0, int nchunk, double eps, AcaWork W)
{
    __shared__ double s_red[NT / 32], s_v[NT / 32];
    __shared__ int s_i[NT / 32];
    __shared__ double2 s_c[ACA_RCAP];
    const int lb = blockIdx.x, b = b0 + lb;
    if (lb >= nchunk) return;
    const int m = (int)(B.rptr[b + 1] - B.rptr[b]), n = (int)(B.cptr[b + 1] - B.cptr[b]);
    const int ntr = (int)(B.trptr[b + 1] - B.trptr[b]), ntc = (int)(B.tcptr[b + 1] - B.tcptr[b]);
    const int *R = B.ridx + B.rptr[b], *C = B.cidx + B.cptr[b];
    const int *Tr = B.tridx + B.trptr[b], *Tc = B.tcidx + B.tcptr[b];
    const int *rl = B.rloc + 2 * B.rptr[b], *cl = B.cloc + 2 * B.cptr[b];
    const int cap = aca_cap(m, n);
    double2 *U = W.U + W.uoff[b], *V = W.V + W.voff[b], *pw = W.pairs + W.poff[b];
    unsigned char *ru = W.flags + W.foff[b], *cu = ru + m;
    for (int i = threadIdx.x; i < m + n; i += blockDim.x) ru[i] = 0;
    __syncthreads();
    int r = 0, istar = 0, result = -1, rows_left = m;
    double nrm2 = 0.0;
    while (r < cap && rows_left > 0) {
        // residual row istar into V[:, r]; pair j = s + 2 c is (T_s of the row, column triangle c)
        const int mi = R[istar];
        const int np = 2 * ntc;
        line_pairs(M, np, M.btri + 2 * mi, 2, Tc, pw);
        if (threadIdx.x < r) s_c[threadIdx.x] = U[istar + (int64_t)threadIdx.x * m];
        __syncthreads();
        double bv = 0.0;
        int bj = NONE;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const int c0 = cl[2 * j], c1 = cl[2 * j + 1];
            double2 z = assemble(M, mi, C[j], [&](int s, int t, int v) {
                return partial_sum(pw, np, s + 2 * (t ? c1 : c0), v);
            });
            for (int l = 0; l < r; ++l) z = cfms(s_c[l], V[j + (int64_t)l * n], z);
            V[j + (int64_t)r * n] = z;
            const double az = hypot(z.x, z.y);
            if (!cu[j] && az > bv) {
                bv = az;
                bj = j;
            }
        }
        block_argmax(bv, bj, s_v, s_i);
        if (threadIdx.x == 0) ru[istar] = 1;
        --rows_left;
        if (bj == NONE || !(bv > 0.0)) {   // zero residual row: the lowest unused row next
            double zv = -1.0;
            int zi = NONE;
            for (int i = threadIdx.x; i < m && zi == NONE; i += blockDim.x)
                if (i != istar && !ru[i]) {
                    zv = 0.0;
                    zi = i;
                }
            block_argmax(zv, zi, s_v, s_i);
            if (zi == NONE) {
                result = r;
                break;
            }
            istar = zi;
            continue;
        }
        // v_r = residual row / pivot
        const double2 piv = V[bj + (int64_t)r * n];
        const double pn = piv.x * piv.x + piv.y * piv.y;
        const double2 pinv = make_double2(piv.x / pn, -piv.y / pn);
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) V[j + (int64_t)r * n] = cmul(V[j + (int64_t)r * n], pinv);
        // residual column bj into U[:, r]; pair j = a + ntr t is (row triangle a, T_t of the column)
        const int nj = C[bj];
        const int np2 = 2 * ntr;
        if (threadIdx.x < r) s_c[threadIdx.x] = V[bj + (int64_t)threadIdx.x * n];
        line_pairs(M, np2, Tr, ntr, M.btri + 2 * nj, pw);
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const int r0 = rl[2 * i], r1 = rl[2 * i + 1];
            double2 z = assemble(M, R[i], nj, [&](int s, int t, int v) {
                return partial_sum(pw, np2, (s ? r1 : r0) + ntr * t, v);
            });
            for (int l = 0; l < r; ++l) z = cfms(U[i + (int64_t)l * m], s_c[l], z);
            U[i + (int64_t)r * m] = z;
        }
        if (threadIdx.x == 0) cu[bj] = 1;
        __syncthreads();
        // ||A_r||_F^2 = ||A_{r-1}||_F^2 + 2 sum_l Re((u_l^H u_r)(v_l^H v_r)) + |u_r|^2 |v_r|^2
        const double2 *ur = U + (int64_t)r * m, *vr = V + (int64_t)r * n;
        double t = 0.0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) t += ur[i].x * ur[i].x + ur[i].y * ur[i].y;
        const double nu2 = block_sum(t, s_red);
        t = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) t += vr[j].x * vr[j].x + vr[j].y * vr[j].y;
        const double nv2 = block_sum(t, s_red);
        const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
        t = 0.0;
        for (int l = wp; l < r; l += blockDim.x >> 5) {
            double2 su = make_double2(0.0, 0.0), sv = su;
            for (int i = lane; i < m; i += 32) su = cjfma(U[i + (int64_t)l * m], ur[i], su);
            for (int j = lane; j < n; j += 32) sv = cjfma(V[j + (int64_t)l * n], vr[j], sv);
            for (int o = 16; o > 0; o >>= 1) {
                su.x += __shfl_xor_sync(0xffffffffu, su.x, o);
                su.y += __shfl_xor_sync(0xffffffffu, su.y, o);
                sv.x += __shfl_xor_sync(0xffffffffu, sv.x, o);
                sv.y += __shfl_xor_sync(0xffffffffu, sv.y, o);
            }
            if (lane == 0) t += su.x * sv.x - su.y * sv.y;
        }
        const double cr = block_sum(t, s_red);
        nrm2 += 2.0 * cr + nu2 * nv2;
        ++r;
        if (sqrt(nu2 * nv2) <= eps * sqrt(fabs(nrm2))) {
            result = r;
            break;
        }
        // next row: argmax |u_r| over unused rows
        double nv = -1.0;
        int ni = NONE;
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            if (!ru[i]) {
                const double a = hypot(ur[i].x, ur[i].y);
                if (a > nv) {
                    nv = a;
                    ni = i;
                }
            }
        block_argmax(nv, ni, s_v, s_i);
        if (ni == NONE) {
            result = r;
            break;
        }
        istar = ni;
    }
    if (result < 0 && rows_left == 0) result = r;
    if (threadIdx.x == 0) W.rank[b] = result;
}

// Gram-Schmidt applied twice to the columns of X (rows x cols, ld rows): Q overwrites X;
// put(i, c, R_ic) receives R (i <= c)
template <class Put>
__device__ void cgs2(double2 *X, int rows, int cols, double2 *s_h, double2 *s_rc, double *s_red, Put put)
{
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = 0; c < cols; ++c) {
        double2 *x = X + (int64_t)c * rows;
        if (threadIdx.x < c) s_rc[threadIdx.x] = make_double2(0.0, 0.0);
        for (int pass = 0; pass < 2; ++pass) {
            __syncthreads();
            for (int l = wp; l < c; l += nw) {
                double2 h = make_double2(0.0, 0.0);
                const double2 *q = X + (int64_t)l * rows;
                for (int i = lane; i < rows; i += 32) h = cjfma(q[i], x[i], h);
                for (int o = 16; o > 0; o >>= 1) {
                    h.x += __shfl_xor_sync(0xffffffffu, h.x, o);
                    h.y += __shfl_xor_sync(0xffffffffu, h.y, o);
                }
                if (lane == 0) s_h[l] = h;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < rows; i += blockDim.x) {
                double2 z = x[i];
                for (int l = 0; l < c; ++l) z = cfms(X[i + (int64_t)l * rows], s_h[l], z);
                x[i] = z;
            }
            if (threadIdx.x < c) s_rc[threadIdx.x] = cadd(s_rc[threadIdx.x], s_h[threadIdx.x]);
        }
        __syncthreads();
        double t = 0.0;
        for (int i = threadIdx.x; i < rows; i += blockDim.x) t += x[i].x * x[i].x + x[i].y * x[i].y;
        const double nrm = sqrt(block_sum(t, s_red));
        if (nrm > 0.0)
            for (int i = threadIdx.x; i < rows; i += blockDim.x) x[i] = csc(1.0 / nrm, x[i]);
        if (threadIdx.x < c) put(threadIdx.x, c, s_rc[threadIdx.x]);
        if (threadIdx.x == 0) put(c, c, make_double2(nrm, 0.0));
    }
    __syncthreads();
}

// re-compression of the ACA factors (rank r) of block b: the truncated factors go to the
// block's slots in Uo (m x r') and Vo (n x r'), the rank r' (or -1: store dense) to W.rank.
// SA, SV: LD x LD work arrays (shared memory for LD = 64, global scratch for the larger ranks)
template <int LD>
__device__ void recompress(int b, int r, int m, int n, double eps, AcaWork &W, double2 *Uo, double2 *Vo, double2 *SA,
                           double2 *SV)
{
    __shared__ double2 s_h[LD], s_rc[LD], s_dv[LD];
    __shared__ double s_red[NT / 32], sig[LD];
    __shared__ int ord[LD], s_rot, s_rank;
    double2 *U = W.U + W.uoff[b], *V = W.V + W.voff[b];
    cgs2(U, m, r, s_h, s_rc, s_red, [&](int i, int c, double2 x) { SV[c * LD + i] = x; });
    cgs2(V, n, r, s_h, s_rc, s_red, [&](int i, int c, double2 x) {
        if (i == c) s_dv[i] = x;
        else SV[i * LD + c] = x;   // R_V(i, c) as R_V^T(c, i), c > i: the strict lower part
    });
    // C(i, j) = sum_{l >= max(i, j)} R_U(i, l) R_V(j, l)
    double f2 = 0.0;
    for (int x = threadIdx.x; x < r * r; x += blockDim.x) {
        const int i = x % r, j = x / r;
        double2 z = make_double2(0.0, 0.0);
        for (int l = max(i, j); l < r; ++l) z = cfma(SV[l * LD + i], (l == j) ? s_dv[j] : SV[j * LD + l], z);
        SA[j * LD + i] = z;
        f2 += z.x * z.x + z.y * z.y;
    }
    f2 = block_sum(f2, s_red);   // also: every thread is past its reads of SV
    for (int x = threadIdx.x; x < r * r; x += blockDim.x) {
        const int i = x % r, j = x / r;
        SV[j * LD + i] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    jacobi_sweeps<double2, LD>(SA, SV, r, r, JacobiEps<double2>::u() * JacobiEps<double2>::u() * f2, &s_rot);
    column_norms2<double2, LD>(SA, r, r, sig);
    __syncthreads();
    if (threadIdx.x == 0) {
        int rr = truncation_rank<double, LD>(sig, ord, r, eps);
        if ((int64_t)rr * (m + n) >= (int64_t)m * n) rr = -1;
        s_rank = rr;
    }
    __syncthreads();
    const int rr = s_rank;
    if (rr > 0) {   // U' = Q_U a_o, V' = Q_V conj(v_o) over the rr largest columns o
        double2 *uo = Uo + W.uoff[b], *vo = Vo + W.voff[b];
        for (int64_t x = threadIdx.x; x < (int64_t)m * rr; x += blockDim.x) {
            const int i = (int)(x % m), o = ord[x / m];
            double2 z = make_double2(0.0, 0.0);
            for (int c = 0; c < r; ++c) z = cfma(U[i + (int64_t)c * m], SA[o * LD + c], z);
            uo[x] = z;
        }
        for (int64_t x = threadIdx.x; x < (int64_t)n * rr; x += blockDim.x) {
            const int j = (int)(x % n), o = ord[x / n];
            double2 z = make_double2(0.0, 0.0);
            for (int c = 0; c < r; ++c) z = cfma(V[j + (int64_t)c * n], jconj(SV[o * LD + c]), z);
            vo[x] = z;
        }
    }
    if (threadIdx.x == 0) W.rank[b] = rr;
}

// blocks b0 + blockIdx.x of rank 1 .. 64, with their work arrays in shared memory
__global__ void __launch_bounds__(NT) k_aca_recompress(int b0, int nchunk, const int64_t *rptr, const int64_t *cptr,
                                                        double eps, AcaWork W, double2 *Uo, double2 *Vo)
{
    extern __shared__ unsigned char smraw[];
    const int lb = blockIdx.x, b = b0 + lb;
    if (lb >= nchunk) return;
    const int r = W.rank[b];
    // a zero block (rank 0), the cap reached (-1), or a rank for k_aca_recompress_big
    if (r <= 0 || r > RC_SMALL) return;
    const int m = (int)(rptr[b + 1] - rptr[b]), n = (int)(cptr[b + 1] - cptr[b]);
    double2 *SA = (double2 *)smraw;
    recompress<RC_SMALL>(b, r, m, n, eps, W, Uo, Vo, SA, SA + RC_SMALL * RC_SMALL);
}

// blocks list[x] of rank 65 .. ACA_RCAP, each with 2 ACA_RCAP^2 entries of global scratch
__global__ void __launch_bounds__(NT) k_aca_recompress_big(int nlist, const int *list, const int64_t *rptr,
                                                            const int64_t *cptr, double eps, AcaWork W, double2 *Uo,
                                                            double2 *Vo, double2 *scratch)
{
    const int x = blockIdx.x;
    if (x >= nlist) return;
    const int b = list[x], r = W.rank[b];
    const int m = (int)(rptr[b + 1] - rptr[b]), n = (int)(cptr[b + 1] - cptr[b]);
    double2 *SA = scratch + (int64_t)x * 2 * ACA_RCAP * ACA_RCAP;
    recompress<ACA_RCAP>(b, r, m, n, eps, W, Uo, Vo, SA, SA + ACA_RCAP * ACA_RCAP);
}

// compact copy: len[x] entries from src + soff[x] to dst + doff[x], one CTA per run
__global__ void k_gather(int nlist, const int64_t *soff, const int64_t *doff, const int64_t *len, const double2 *src,
                         double2 *dst)
{
    const int x = blockIdx.x;
    if (x >= nlist) return;
    for (int64_t e = threadIdx.x; e < len[x]; e += blockDim.x) dst[doff[x] + e] = src[soff[x] + e];
}

// ---------------------------------------------------------------------------------------
// host side
struct DevBufs {
    std::vector<void *> p;
    ~DevBufs()
    {
        for (void *x : p) cudaFree(x);
    }
    template <class T> cudaError_t alloc(T **d, size_t count)
    {
        void *x = nullptr;
        cudaError_t e = cudaMalloc(&x, sizeof(T) * std::max<size_t>(count, 1));
        if (e) return e;
        p.push_back(x);
        *d = (T *)x;
        return cudaSuccess;
    }
    template <class T> cudaError_t up(T **d, const std::vector<T> &v)
    {
        cudaError_t e = alloc(d, v.size());
        if (e || v.empty()) return e;
        return cudaMemcpy(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    }
    // grow-only scratch
    template <class T> cudaError_t grow(T **d, size_t *have, size_t need)
    {
        if (*d && need <= *have) return cudaSuccess;
        if (*d) {
            for (auto &x : p)
                if (x == (void *)*d) x = nullptr;
            cudaFree(*d);
            *d = nullptr;
        }
        cudaError_t e = alloc(d, need);
        *have = e ? 0 : std::max<size_t>(need, 1);
        return e;
    }
};

struct Ctx {
    DevBufs mem;
    Mesh M{};
    Blocks B{};   // the call's blocks on the device (the ACA works on them)
    int nblk = 0, nt = 0;
    const int32_t *tri = nullptr;                   // host, the caller's (valid during the call)
    std::vector<int64_t> rptr, cptr, trptr, tcptr;  // host copies
    std::vector<int> ridx, cidx;
    std::vector<unsigned char> sym;                 // per block: mirror the upper triangle
};

int check_mesh(int nv, const double *V, int nt, const int32_t *T, int nb, const int32_t *tri, const int32_t *fv,
               double k)
{
    if (nv < 3 || nt < 1 || nb < 1 || !V || !T || !tri || !fv || !(k > 0)) return HM_EINVAL;
    for (int t = 0; t < 3 * nt; ++t)
        if (T[t] < 0 || T[t] >= nv) return HM_EINVAL;
    for (int b = 0; b < 2 * nb; ++b)
        if (tri[b] < 0 || tri[b] >= nt || fv[b] < 0 || fv[b] >= nv) return HM_EINVAL;
    return HM_OK;
}

int check_blocks(int nb, int nblk, const int64_t *rptr, const int32_t *ridx, const int64_t *cptr,
                 const int32_t *cidx)
{
    if (nblk < 0 || (nblk > 0 && (!rptr || !ridx || !cptr || !cidx))) return HM_EINVAL;
    if (nblk == 0) return HM_OK;
    if (rptr[0] != 0 || cptr[0] != 0) return HM_EINVAL;
    for (int b = 0; b < nblk; ++b)
        if (rptr[b + 1] <= rptr[b] || cptr[b + 1] <= cptr[b]) return HM_EINVAL;
    for (int64_t i = 0; i < rptr[nblk]; ++i)
        if (ridx[i] < 0 || ridx[i] >= nb) return HM_EINVAL;
    for (int64_t i = 0; i < cptr[nblk]; ++i)
        if (cidx[i] < 0 || cidx[i] >= nb) return HM_EINVAL;
    return HM_OK;
}

// one side (rows or columns) of every block: its distinct triangles and each RWG's local
// indices of its T+ and T-
void side_lists(int nt, int nblk, const int64_t *ptr, const int32_t *idx, const int32_t *tri,
                std::vector<int64_t> &tptr, std::vector<int> &tidx, std::vector<int> &loc)
{
    std::vector<int> stamp(nt, -1), where(nt, 0);
    tptr.assign(nblk + 1, 0);
    tidx.clear();
    loc.assign(2 * (size_t)ptr[nblk], 0);
    for (int b = 0; b < nblk; ++b) {
        int cnt = 0;
        for (int64_t i = ptr[b]; i < ptr[b + 1]; ++i)
            for (int s = 0; s < 2; ++s) {
                const int t = tri[2 * idx[i] + s];
                if (stamp[t] != b) {
                    stamp[t] = b;
                    where[t] = cnt++;
                    tidx.push_back(t);
                }
                loc[2 * i + s] = where[t];
            }
        tptr[b + 1] = tptr[b] + cnt;
    }
}

template <class T> cudaError_t upload(DevBufs &mem, const T **dst, const std::vector<T> &v)
{
    T *d = nullptr;
    cudaError_t e = mem.up(&d, v);
    *dst = d;
    return e;
}

// a set of blocks (RWG row and column lists) on the device with their distinct triangles
cudaError_t upload_blocks(DevBufs &mem, int nt, const int32_t *tri, const std::vector<int64_t> &rptr,
                          const std::vector<int> &ridx, const std::vector<int64_t> &cptr,
                          const std::vector<int> &cidx, Blocks &B, std::vector<int64_t> &trptr,
                          std::vector<int64_t> &tcptr)
{
    const int nblk = (int)rptr.size() - 1;
    std::vector<int> tridx, tcidx, rloc, cloc;
    side_lists(nt, nblk, rptr.data(), ridx.data(), tri, trptr, tridx, rloc);
    side_lists(nt, nblk, cptr.data(), cidx.data(), tri, tcptr, tcidx, cloc);
    cudaError_t e;
    if ((e = upload(mem, &B.rptr, rptr)) || (e = upload(mem, &B.cptr, cptr)) || (e = upload(mem, &B.trptr, trptr)) ||
        (e = upload(mem, &B.tcptr, tcptr)) || (e = upload(mem, &B.ridx, ridx)) || (e = upload(mem, &B.cidx, cidx)) ||
        (e = upload(mem, &B.tridx, tridx)) || (e = upload(mem, &B.tcidx, tcidx)) || (e = upload(mem, &B.rloc, rloc)) ||
        (e = upload(mem, &B.cloc, cloc)))
        return e;
    return cudaSuccess;
}

cudaError_t ctx_init(Ctx &X, const double *V, int nt, const int32_t *T, int nb, const int32_t *tri,
                     const int32_t *fv, double k, double eta0, double r_abs, double c_rel, int nblk,
                     const int64_t *rptr, const int32_t *ridx, const int64_t *cptr, const int32_t *cidx,
                     bool mirror)
{
    double w[NQ], bq[NQ][3];
    radon_rule(w, bq);
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(c_qw, w, sizeof(w)))) return e;
    std::vector<double> tv(9 * (size_t)nt), tn(3 * (size_t)nt), ta(nt), tc(3 * (size_t)nt), th(nt),
        tq(3 * NQ * (size_t)nt), bfree(6 * (size_t)nb), blen(nb);
    for (int t = 0; t < nt; ++t) {
        double *P = &tv[9 * (size_t)t];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) P[3 * i + j] = V[3 * T[3 * t + i] + j];
        double e1[3], e2[3], e3[3];
        for (int j = 0; j < 3; ++j) e1[j] = P[3 + j] - P[j], e2[j] = P[6 + j] - P[j], e3[j] = P[6 + j] - P[3 + j];
        const double nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                              e1[0] * e2[1] - e1[1] * e2[0]};
        const double an = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        auto len = [](const double *x) { return std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]); };
        ta[t] = 0.5 * an;
        th[t] = std::max(len(e1), std::max(len(e2), len(e3)));
        for (int j = 0; j < 3; ++j) {
            tn[3 * t + j] = nn[j] / an;
            tc[3 * t + j] = (P[j] + P[3 + j] + P[6 + j]) / 3.0;
        }
        for (int q = 0; q < NQ; ++q)
            for (int j = 0; j < 3; ++j)
                tq[(t * NQ + q) * 3 + j] = bq[q][0] * P[j] + bq[q][1] * P[3 + j] + bq[q][2] * P[6 + j];
    }
    std::vector<int> btri(2 * (size_t)nb);
    for (int n = 0; n < nb; ++n) {
        btri[2 * n] = tri[2 * n];
        btri[2 * n + 1] = tri[2 * n + 1];
        for (int s = 0; s < 2; ++s)
            for (int j = 0; j < 3; ++j) bfree[6 * n + 3 * s + j] = V[3 * fv[2 * n + s] + j];
        // the edge: the two vertices of T+ other than its free vertex
        const int32_t *tt = T + 3 * tri[2 * n];
        double ev[2][3] = {{0, 0, 0}, {0, 0, 0}};
        int c = 0;
        for (int i = 0; i < 3; ++i)
            if (tt[i] != fv[2 * n] && c < 2) {
                for (int j = 0; j < 3; ++j) ev[c][j] = V[3 * tt[i] + j];
                ++c;
            }
        double d2 = 0;
        for (int j = 0; j < 3; ++j) d2 += (ev[1][j] - ev[0][j]) * (ev[1][j] - ev[0][j]);
        blen[n] = std::sqrt(d2);
    }
    Mesh &M = X.M;
    M.k = k;
    M.eta0 = eta0;
    M.r_abs = r_abs;
    M.c_rel = c_rel;
    if ((e = upload(X.mem, &M.tv, tv)) || (e = upload(X.mem, &M.tn, tn)) || (e = upload(X.mem, &M.ta, ta)) ||
        (e = upload(X.mem, &M.tc, tc)) || (e = upload(X.mem, &M.th, th)) || (e = upload(X.mem, &M.tq, tq)) ||
        (e = upload(X.mem, &M.bfree, bfree)) || (e = upload(X.mem, &M.blen, blen)) ||
        (e = upload(X.mem, &M.btri, btri)))
        return e;
    X.nblk = nblk;
    X.nt = nt;
    X.tri = tri;
    X.rptr.assign(rptr, rptr + nblk + 1);
    X.cptr.assign(cptr, cptr + nblk + 1);
    X.ridx.assign(ridx, ridx + rptr[nblk]);
    X.cidx.assign(cidx, cidx + cptr[nblk]);
    X.sym.assign(nblk, 0);
    for (int b = 0; b < nblk && mirror; ++b)
        X.sym[b] = rptr[b + 1] - rptr[b] == cptr[b + 1] - cptr[b] &&
                   std::equal(ridx + rptr[b], ridx + rptr[b + 1], cidx + cptr[b]);
    return upload_blocks(X.mem, nt, tri, X.rptr, X.ridx, X.cptr, X.cidx, X.B, X.trptr, X.tcptr);
}

// dense blocks `list` of X into host memory, block list[x] at host + hoff[x].  A block is
// cut into tiles of at most FILL_TR x FILL_TC RWG functions (one CTA each), so that a large
// block is spread over the SMs; the tiles of a chunk of blocks get their own triangle lists.
cudaError_t fill_dense(Ctx &X, const std::vector<int> &list, const std::vector<int64_t> &hoff, hm_c128 *host,
                       size_t chunk_bytes)
{
    cudaError_t e;
    double2 *d_pairs = nullptr, *d_out = nullptr;
    size_t h_pairs = 0, h_out = 0;
    size_t x0 = 0;
    while (x0 < list.size()) {
        std::vector<int64_t> trp(1, 0), tcp(1, 0), ooff, pofs, soff;
        std::vector<int> tr, tc, lds, sm;
        size_t bytes = 0, x1 = x0;
        int64_t out_len = 0;
        while (x1 < list.size()) {
            const int b = list[x1];
            const int64_t m = X.rptr[b + 1] - X.rptr[b], n = X.cptr[b + 1] - X.cptr[b];
            // pair scratch estimated from the block's own distinct triangles (its tiles share a few)
            const int64_t P = (X.trptr[b + 1] - X.trptr[b]) * (X.tcptr[b + 1] - X.tcptr[b]);
            const size_t nbytes = sizeof(double2) * (size_t)(NPV * P * 3 / 2 + m * n);
            if (x1 > x0 && bytes + nbytes > chunk_bytes) break;
            const int *R = X.ridx.data() + X.rptr[b], *C = X.cidx.data() + X.cptr[b];
            if (X.sym[b]) {
                soff.push_back(out_len);
                sm.push_back((int)m);
            }
            for (int64_t c0 = 0; c0 < n; c0 += FILL_TC)
                for (int64_t r0 = 0; r0 < m; r0 += FILL_TR) {
                    const int64_t r1 = std::min(m, r0 + FILL_TR), c1 = std::min(n, c0 + FILL_TC);
                    tr.insert(tr.end(), R + r0, R + r1);
                    tc.insert(tc.end(), C + c0, C + c1);
                    trp.push_back((int64_t)tr.size());
                    tcp.push_back((int64_t)tc.size());
                    ooff.push_back(out_len + r0 + c0 * m);
                    lds.push_back((int)m);
                }
            pofs.push_back(out_len);
            out_len += m * n;
            bytes += nbytes;
            ++x1;
        }
        DevBufs tmem;   // the chunk's tiles
        Blocks TB{};
        std::vector<int64_t> ttrp, ttcp;
        if ((e = upload_blocks(tmem, X.nt, X.tri, trp, tr, tcp, tc, TB, ttrp, ttcp))) return e;
        const int ntile = (int)ooff.size();
        std::vector<int64_t> po(ntile + 1, 0);
        for (int t = 0; t < ntile; ++t) po[t + 1] = po[t] + NPV * (ttrp[t + 1] - ttrp[t]) * (ttcp[t + 1] - ttcp[t]);
        const int64_t *d_po, *d_oo, *d_so;
        const int *d_ld, *d_sm;
        if ((e = X.mem.grow(&d_pairs, &h_pairs, (size_t)po.back())) || (e = X.mem.grow(&d_out, &h_out, (size_t)out_len)) ||
            (e = upload(tmem, &d_po, po)) || (e = upload(tmem, &d_oo, ooff)) || (e = upload(tmem, &d_ld, lds)) ||
            (e = upload(tmem, &d_so, soff)) || (e = upload(tmem, &d_sm, sm)))
            return e;
        k_efie_fill<<<ntile, NT>>>(X.M, TB, ntile, d_po, d_pairs, d_oo, d_ld, d_out);
        if (!soff.empty()) k_mirror<<<(unsigned)soff.size(), NT>>>((int)soff.size(), d_so, d_sm, d_out);
        if ((e = cudaGetLastError()) || (e = cudaDeviceSynchronize())) return e;
        // copy out, one copy per run of blocks adjacent in the host layout
        const size_t nl = x1 - x0;
        size_t y = 0;
        auto block_end = [&](size_t q) {   // end of block x0 + q in the chunk's output
            const int b = list[x0 + q];
            return pofs[q] + (X.rptr[b + 1] - X.rptr[b]) * (X.cptr[b + 1] - X.cptr[b]);
        };
        while (y < nl) {
            size_t z = y + 1;
            while (z < nl && hoff[x0 + z] == hoff[x0 + y] + (pofs[z] - pofs[y])) ++z;
            if ((e = cudaMemcpy(host + hoff[x0 + y], d_out + pofs[y], sizeof(double2) * (block_end(z - 1) - pofs[y]),
                                cudaMemcpyDeviceToHost)))
                return e;
            y = z;
        }
        x0 = x1;
    }
    return cudaSuccess;
}

int status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return HM_OK;
    std::fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA;
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" int hm_efie_fill(int32_t nv, const double *V, int32_t nt, const int32_t *T, int32_t nb,
                            const int32_t *tri, const int32_t *free_v, double k, double eta0, double r_abs,
                            double c_rel, int32_t nblk, const int64_t *rptr, const int32_t *ridx,
                            const int64_t *cptr, const int32_t *cidx, int32_t mirror, const int64_t *off,
                            hm_c128 *out, int64_t scratch_bytes, int32_t device)
{
    int c;
    if ((c = check_mesh(nv, V, nt, T, nb, tri, free_v, k)) || (c = check_blocks(nb, nblk, rptr, ridx, cptr, cidx)))
        return c;
    if ((mirror != 0 && mirror != 1) || scratch_bytes < 0) return HM_EINVAL;
    if (nblk == 0) return HM_OK;
    if (!off || !out || off[0] != 0) return HM_EINVAL;
    for (int b = 0; b < nblk; ++b)
        if (off[b + 1] - off[b] != (rptr[b + 1] - rptr[b]) * (cptr[b + 1] - cptr[b])) return HM_EINVAL;
    cudaError_t e;
    if ((e = cudaSetDevice(device))) return status(e, "hm_efie_fill");
    Ctx X;
    if ((e = ctx_init(X, V, nt, T, nb, tri, free_v, k, eta0, r_abs, c_rel, nblk, rptr, ridx, cptr, cidx,
                      mirror != 0)))
        return status(e, "hm_efie_fill");
    std::vector<int> list(nblk);
    for (int b = 0; b < nblk; ++b) list[b] = b;
    const size_t chunk_bytes = scratch_bytes ? (size_t)scratch_bytes : CHUNK_BYTES;
    return status(fill_dense(X, list, std::vector<int64_t>(off, off + nblk), out, chunk_bytes), "hm_efie_fill");
}

extern "C" int hm_efie_far(int32_t nv, const double *V, int32_t nt, const int32_t *T, int32_t nb, const int32_t *tri,
                           const int32_t *free_v, double k, double eta0, double r_abs, double c_rel, int32_t nblk,
                           const int64_t *rptr, const int32_t *ridx, const int64_t *cptr, const int32_t *cidx,
                           double eps, int32_t *rank, int64_t *uoff, int64_t *voff, int64_t cap_u, hm_c128 *U,
                           int64_t cap_v, hm_c128 *Vf, int64_t *need, int64_t scratch_bytes, int32_t device)
{
    int c;
    if ((c = check_mesh(nv, V, nt, T, nb, tri, free_v, k)) || (c = check_blocks(nb, nblk, rptr, ridx, cptr, cidx)))
        return c;
    if (!(eps > 0) || !(eps < 1) || cap_u < 0 || cap_v < 0 || !need || scratch_bytes < 0) return HM_EINVAL;
    const size_t chunk_bytes = scratch_bytes ? (size_t)scratch_bytes : CHUNK_BYTES;
    need[0] = need[1] = 0;
    if (nblk == 0) return HM_OK;
    if (!rank || !uoff || !voff || (cap_u > 0 && !U) || (cap_v > 0 && !Vf)) return HM_EINVAL;
    cudaError_t e;
    if ((e = cudaSetDevice(device))) return status(e, "hm_efie_far");
    Ctx X;
    if ((e = ctx_init(X, V, nt, T, nb, tri, free_v, k, eta0, r_abs, c_rel, nblk, rptr, ridx, cptr, cidx, false)))
        return status(e, "hm_efie_far");
    const size_t smem = sizeof(double2) * 2 * RC_SMALL * RC_SMALL;
    if ((e = cudaFuncSetAttribute(k_aca_recompress, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return status(e, "hm_efie_far");
    // work slots per block, relative to the block's chunk: pair partials, U and V (cap columns),
    // the used-row / used-column flags
    std::vector<int64_t> wp(nblk), wu(nblk), wv(nblk), wf(nblk);
    std::vector<int> chunk(1, 0);
    std::vector<size_t> cneed_p, cneed_u, cneed_v, cneed_f;
    {
        int64_t sp = 0, su = 0, sv = 0, sf = 0;
        size_t bytes = 0;
        for (int b = 0; b < nblk; ++b) {
            const int64_t m = X.rptr[b + 1] - X.rptr[b], n = X.cptr[b + 1] - X.cptr[b];
            const int64_t nt2 = std::max(X.trptr[b + 1] - X.trptr[b], X.tcptr[b + 1] - X.tcptr[b]);
            const int64_t cp = std::min<int64_t>(std::min(std::min(m, n), m * n / (m + n) + 1), ACA_RCAP);
            const int64_t np = (int64_t)NPV * NQ * 2 * nt2;
            const size_t nbytes = sizeof(double2) * (size_t)(np + 2 * cp * (m + n)) + (size_t)(m + n);
            if (b > chunk.back() && bytes + nbytes > chunk_bytes) {
                chunk.push_back(b);
                cneed_p.push_back(sp), cneed_u.push_back(su), cneed_v.push_back(sv), cneed_f.push_back(sf);
                sp = su = sv = sf = 0;
                bytes = 0;
            }
            wp[b] = sp, wu[b] = su, wv[b] = sv, wf[b] = sf;
            sp += np, su += cp * m, sv += cp * n, sf += m + n;
            bytes += nbytes;
        }
        chunk.push_back(nblk);
        cneed_p.push_back(sp), cneed_u.push_back(su), cneed_v.push_back(sv), cneed_f.push_back(sf);
    }
    AcaWork W{};
    if ((e = upload(X.mem, &W.poff, wp)) || (e = upload(X.mem, &W.uoff, wu)) || (e = upload(X.mem, &W.voff, wv)) ||
        (e = upload(X.mem, &W.foff, wf)) || (e = X.mem.alloc(&W.rank, nblk)))
        return status(e, "hm_efie_far");
    double2 *Uo = nullptr, *Vo = nullptr, *d_cu = nullptr, *d_cv = nullptr, *d_big = nullptr;
    int64_t *d_so = nullptr, *d_do = nullptr, *d_len = nullptr;
    int *d_blist = nullptr;
    size_t hp = 0, hu = 0, hv = 0, hf = 0, huo = 0, hvo = 0, hcu = 0, hcv = 0, hso = 0, hdo = 0, hlen = 0, hbig = 0,
           hbl = 0;
    constexpr int BIG_BATCH = 128;   // blocks of rank > 64 re-compressed per launch (2 MiB scratch each)
    int64_t tot_u = 0, tot_v = 0;
    std::vector<int> dense;
    std::vector<int64_t> dense_off;
    for (size_t ci = 0; ci + 1 < chunk.size(); ++ci) {
        const int b0 = chunk[ci], b1 = chunk[ci + 1], nc = b1 - b0;
        if ((e = X.mem.grow(&W.pairs, &hp, cneed_p[ci])) || (e = X.mem.grow(&W.U, &hu, cneed_u[ci])) ||
            (e = X.mem.grow(&W.V, &hv, cneed_v[ci])) || (e = X.mem.grow(&W.flags, &hf, cneed_f[ci])) ||
            (e = X.mem.grow(&Uo, &huo, cneed_u[ci])) || (e = X.mem.grow(&Vo, &hvo, cneed_v[ci])))
            return status(e, "hm_efie_far");
        k_efie_aca<<<nc, NT>>>(X.M, X.B, b0, nc, eps, W);
        if ((e = cudaGetLastError()) || (e = cudaDeviceSynchronize()) ||
            (e = cudaMemcpy(rank + b0, W.rank + b0, sizeof(int) * nc, cudaMemcpyDeviceToHost)))
            return status(e, "hm_efie_far");
        std::vector<int> big;   // ACA ranks above what the shared-memory re-compression holds
        for (int b = b0; b < b1; ++b)
            if (rank[b] > RC_SMALL) big.push_back(b);
        k_aca_recompress<<<nc, NT, smem>>>(b0, nc, X.B.rptr, X.B.cptr, eps, W, Uo, Vo);
        for (size_t x0 = 0; x0 < big.size(); x0 += BIG_BATCH) {
            const int nbl = (int)std::min<size_t>(BIG_BATCH, big.size() - x0);
            if ((e = X.mem.grow(&d_big, &hbig, (size_t)nbl * 2 * ACA_RCAP * ACA_RCAP)) ||
                (e = X.mem.grow(&d_blist, &hbl, (size_t)nbl)) ||
                (e = cudaMemcpy(d_blist, big.data() + x0, sizeof(int) * nbl, cudaMemcpyHostToDevice)))
                return status(e, "hm_efie_far");
            k_aca_recompress_big<<<nbl, NT>>>(nbl, d_blist, X.B.rptr, X.B.cptr, eps, W, Uo, Vo, d_big);
            if ((e = cudaGetLastError()) || (e = cudaDeviceSynchronize())) return status(e, "hm_efie_far");
        }
        if ((e = cudaGetLastError()) || (e = cudaDeviceSynchronize()) ||
            (e = cudaMemcpy(rank + b0, W.rank + b0, sizeof(int) * nc, cudaMemcpyDeviceToHost)))
            return status(e, "hm_efie_far");
        // block order: the factors (m r then n r entries) or the dense block (m n, rank -1)
        std::vector<int64_t> su, sv, du, dv, lu, lv;
        std::vector<int> cdense;
        std::vector<int64_t> cdoff;
        const int64_t cu0 = tot_u, cv0 = tot_v;
        for (int b = b0; b < b1; ++b) {
            const int64_t m = X.rptr[b + 1] - X.rptr[b], n = X.cptr[b + 1] - X.cptr[b];
            uoff[b] = tot_u;
            voff[b] = tot_v;
            if (rank[b] < 0) {
                cdense.push_back(b);
                cdoff.push_back(tot_u);
                tot_u += m * n;
            } else if (rank[b] > 0) {
                su.push_back(wu[b]), du.push_back(tot_u - cu0), lu.push_back(m * rank[b]);
                sv.push_back(wv[b]), dv.push_back(tot_v - cv0), lv.push_back(n * rank[b]);
                tot_u += m * rank[b];
                tot_v += n * rank[b];
            }
        }
        if (tot_u > cap_u || tot_v > cap_v) continue;   // only the ranks and the sizes from here on
        dense.insert(dense.end(), cdense.begin(), cdense.end());
        dense_off.insert(dense_off.end(), cdoff.begin(), cdoff.end());
        if (su.empty()) continue;
        const int nl = (int)su.size();
        if ((e = X.mem.grow(&d_cu, &hcu, (size_t)(tot_u - cu0))) ||
            (e = X.mem.grow(&d_cv, &hcv, (size_t)(tot_v - cv0))) || (e = X.mem.grow(&d_so, &hso, nl)) ||
            (e = X.mem.grow(&d_do, &hdo, nl)) || (e = X.mem.grow(&d_len, &hlen, nl)))
            return status(e, "hm_efie_far");
        auto gather = [&](const std::vector<int64_t> &s, const std::vector<int64_t> &d, const std::vector<int64_t> &l,
                          const double2 *src, double2 *dst) -> cudaError_t {
            cudaError_t e2;
            if ((e2 = cudaMemcpy(d_so, s.data(), sizeof(int64_t) * nl, cudaMemcpyHostToDevice)) ||
                (e2 = cudaMemcpy(d_do, d.data(), sizeof(int64_t) * nl, cudaMemcpyHostToDevice)) ||
                (e2 = cudaMemcpy(d_len, l.data(), sizeof(int64_t) * nl, cudaMemcpyHostToDevice)))
                return e2;
            k_gather<<<nl, 128>>>(nl, d_so, d_do, d_len, src, dst);
            if ((e2 = cudaGetLastError())) return e2;
            return cudaDeviceSynchronize();
        };
        if ((e = gather(su, du, lu, Uo, d_cu)) || (e = gather(sv, dv, lv, Vo, d_cv))) return status(e, "hm_efie_far");
        // dense blocks leave gaps in U (filled below): copy the runs of factors between them
        size_t y = 0;
        while (y < du.size()) {
            size_t z = y + 1;
            while (z < du.size() && du[z] == du[z - 1] + lu[z - 1]) ++z;
            const int64_t len = du[z - 1] + lu[z - 1] - du[y];
            if ((e = cudaMemcpy(U + cu0 + du[y], d_cu + du[y], sizeof(double2) * len, cudaMemcpyDeviceToHost)))
                return status(e, "hm_efie_far");
            y = z;
        }
        if (tot_v > cv0 &&
            (e = cudaMemcpy(Vf + cv0, d_cv, sizeof(double2) * (tot_v - cv0), cudaMemcpyDeviceToHost)))
            return status(e, "hm_efie_far");
    }
    need[0] = tot_u;
    need[1] = tot_v;
    if (tot_u > cap_u || tot_v > cap_v) return HM_ENOMEM;
    if (!dense.empty() && (e = fill_dense(X, dense, dense_off, U, chunk_bytes))) return status(e, "hm_efie_far");
    return HM_OK;
}
