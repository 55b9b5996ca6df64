// One-sided (Hestenes) Jacobi SVD of a small complex matrix held by one CTA (in shared memory,
// or in global memory for the larger ACA cores),
// and the truncation rank of Sec. 3.4 / Eq. 10 (smallest r whose singular-value tail has
// Frobenius norm <= tol times the total).  Used by the fill-in compression and by the
// re-compression of ACA factors; a one-warp form serves the many small fill-in blocks.
//
// A (nr x nc, nr >= nc, column c at A + c * LD) is rotated in place until its columns are
// mutually orthogonal; V (nc x nc, same stride, the identity on entry) accumulates the
// rotations, so that A_in V = A_out and A_in = A_out V^H.  Column pairs are rotated in
// round-robin order (each round pairs every column once; the warps take the pairs of a round
// in parallel), each rotation the complex Jacobi rotation that makes the two columns
// orthogonal.  With u the unit roundoff, a pair is skipped once its coupling |a_p^H a_q| is
// below sqrt(nr) u |a_p| |a_q| (orthogonal to working precision) or below floor2 (both columns
// at the rounding level of the matrix); sweeps repeat until no pair needs a rotation.
#pragma once
#include "cplx.cuh"

namespace hm {

template <class T> struct JacobiEps;
template <> struct JacobiEps<double2> { static __device__ double u() { return 1.1102230246251565e-16; } };
template <> struct JacobiEps<float2> { static __device__ float u() { return 5.9604645e-8f; } };

__device__ __forceinline__ double2 jconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 jconj(float2 a) { return make_float2(a.x, -a.y); }

// every thread of the CTA calls it; blockDim.x a multiple of 32
template <class TC, int LD>
__device__ void jacobi_sweeps(TC *A, TC *V, int nr, int nc, typename Real<TC>::type floor2, int *s_rot)
{
    typedef typename Real<TC>::type R;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const R ctol = sqrt(R(nr)) * JacobiEps<TC>::u();
    const int np = (nc + 1) & ~1;   // players of the round robin (one dummy when nc is odd)
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (threadIdx.x == 0) *s_rot = 0;
        __syncthreads();
        for (int t = 0; t < np - 1; ++t) {
            for (int pi = wp; pi < np / 2; pi += nw) {
                int p, q;
                if (pi == 0) {
                    p = t;
                    q = np - 1;
                } else {
                    p = (t + pi) % (np - 1);
                    q = (t - pi + np - 1) % (np - 1);
                }
                if (p >= nc || q >= nc) continue;
                TC *ap = A + p * LD, *aq = A + q * LD;
                R al = 0, be = 0;
                TC ga = czero(TC());
                for (int r = lane; r < nr; r += 32) {
                    const TC x = ap[r], y = aq[r];
                    al += x.x * x.x + x.y * x.y;
                    be += y.x * y.x + y.y * y.y;
                    ga.x += x.x * y.x + x.y * y.y;   // conj(x) y
                    ga.y += x.x * y.y - x.y * y.x;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
                    ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
                }
                const R g = sqrt(ga.x * ga.x + ga.y * ga.y);
                if (!(g > ctol * sqrt(al * be)) || !(g > floor2)) continue;
                const R zeta = (be - al) / (2 * g);
                const R tt = (zeta >= 0 ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
                const R cs = R(1) / sqrt(R(1) + tt * tt), sn = cs * tt;
                TC ph;   // conj(gamma) / |gamma|
                ph.x = ga.x / g;
                ph.y = -ga.y / g;
                for (int r = lane; r < nr; r += 32) {
                    const TC x = ap[r];
                    const TC y = cmul(ph, aq[r]);
                    ap[r].x = cs * x.x - sn * y.x;
                    ap[r].y = cs * x.y - sn * y.y;
                    aq[r].x = sn * x.x + cs * y.x;
                    aq[r].y = sn * x.y + cs * y.y;
                }
                TC *vp = V + p * LD, *vq = V + q * LD;
                for (int r = lane; r < nc; r += 32) {
                    const TC x = vp[r];
                    const TC y = cmul(ph, vq[r]);
                    vp[r].x = cs * x.x - sn * y.x;
                    vp[r].y = cs * x.y - sn * y.y;
                    vq[r].x = sn * x.x + cs * y.x;
                    vq[r].y = sn * x.y + cs * y.y;
                }
                if (lane == 0) *s_rot = 1;
            }
            __syncthreads();
        }
        if (!*s_rot) break;
        __syncthreads();
    }
}

// The same sweeps by one warp, each column pair of a round on its own lane (nc <= 64, so a
// round has at most 32 pairs), or, when a round has at most 16 pairs, on two lanes that take
// the even and the odd rows and add their partial inner products with one shuffle: no CTA
// barrier (only __syncwarp between rounds).  A has leading dimension lda, V ldv (runtime).
// Pairs, rotations, the skip rule and the sweep limit are those of jacobi_sweeps; both lanes
// of a pair hold the same sums (addition commutes), so they take the same decision.
template <class TC>
__device__ void jacobi_sweeps_warp(TC *A, int lda, TC *V, int ldv, int nr, int nc, typename Real<TC>::type floor2)
{
    typedef typename Real<TC>::type R;
    const int lane = threadIdx.x & 31;
    const R ctol = sqrt(R(nr)) * JacobiEps<TC>::u();
    const int np = (nc + 1) & ~1;
    const bool split = np / 2 <= 16;
    const int pl = split ? (lane & 15) : lane;   // pair of the round
    const int r0 = split ? (lane >> 4) : 0, rs = split ? 2 : 1;
    for (int sweep = 0; sweep < 40; ++sweep) {
        bool rot = false;
        for (int t = 0; t < np - 1; ++t) {
            int p = t, q = np - 1;
            if (pl > 0) {
                p = t + pl;
                if (p >= np - 1) p -= np - 1;
                q = t - pl + np - 1;
                if (q >= np - 1) q -= np - 1;
            }
            const bool act = pl < np / 2 && p < nc && q < nc;
            TC *ap = A + p * lda, *aq = A + q * lda;
            R al = 0, be = 0;
            TC ga = czero(TC());
            if (act) {
#pragma unroll 4
                for (int r = r0; r < nr; r += rs) {
                    const TC x = ap[r], y = aq[r];
                    al += x.x * x.x + x.y * x.y;
                    be += y.x * y.x + y.y * y.y;
                    ga.x += x.x * y.x + x.y * y.y;   // conj(x) y
                    ga.y += x.x * y.y - x.y * y.x;
                }
            }
            if (split) {
                al += __shfl_xor_sync(0xffffffffu, al, 16);
                be += __shfl_xor_sync(0xffffffffu, be, 16);
                ga.x += __shfl_xor_sync(0xffffffffu, ga.x, 16);
                ga.y += __shfl_xor_sync(0xffffffffu, ga.y, 16);
            }
            const R g = sqrt(ga.x * ga.x + ga.y * ga.y);
            if (act && g > ctol * sqrt(al * be) && g > floor2) {
                const R zeta = (be - al) / (2 * g);
                const R tt = (zeta >= 0 ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
                const R cs = R(1) / sqrt(R(1) + tt * tt), sn = cs * tt;
                TC ph;   // conj(gamma) / |gamma|
                ph.x = ga.x / g;
                ph.y = -ga.y / g;
#pragma unroll 4
                for (int r = r0; r < nr; r += rs) {
                    const TC x = ap[r];
                    const TC y = cmul(ph, aq[r]);
                    ap[r].x = cs * x.x - sn * y.x;
                    ap[r].y = cs * x.y - sn * y.y;
                    aq[r].x = sn * x.x + cs * y.x;
                    aq[r].y = sn * x.y + cs * y.y;
                }
                TC *vp = V + p * ldv, *vq = V + q * ldv;
#pragma unroll 4
                for (int r = r0; r < nc; r += rs) {
                    const TC x = vp[r];
                    const TC y = cmul(ph, vq[r]);
                    vp[r].x = cs * x.x - sn * y.x;
                    vp[r].y = cs * x.y - sn * y.y;
                    vq[r].x = sn * x.x + cs * y.x;
                    vq[r].y = sn * x.y + cs * y.y;
                }
                rot = true;
            }
            __syncwarp();
        }
        if (!__any_sync(0xffffffffu, rot)) break;
    }
}

// sig[c] <- ||a_c||^2; every thread calls it
template <class TC, int LD>
__device__ void column_norms2(const TC *A, int nr, int nc, typename Real<TC>::type *sig)
{
    typedef typename Real<TC>::type R;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = wp; c < nc; c += nw) {
        R s2 = 0;
        for (int r = lane; r < nr; r += 32) s2 += A[c * LD + r].x * A[c * LD + r].x + A[c * LD + r].y * A[c * LD + r].y;
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) sig[c] = s2;
    }
}

// one thread: ord <- columns by descending sig (stable); returns the smallest r with
// sqrt(sum_{i >= r} sigma_i^2) <= tol sqrt(sum sigma_i^2) (suffix sums from the smallest up,
// so that no cancellation enters the tail); nc <= MAXN
template <class R, int MAXN = 64> __device__ int truncation_rank(const R *sig, int *ord, int nc, double tol)
{
    for (int c = 0; c < nc; ++c) ord[c] = c;
    for (int a = 1; a < nc; ++a) {
        const int v = ord[a];
        int b = a - 1;
        while (b >= 0 && sig[ord[b]] < sig[v]) {
            ord[b + 1] = ord[b];
            --b;
        }
        ord[b + 1] = v;
    }
    double suf[MAXN + 1];
    suf[nc] = 0.0;
    for (int i = nc - 1; i >= 0; --i) suf[i] = suf[i + 1] + (double)sig[ord[i]];
    const double thr = tol * sqrt(suf[0]);
    for (int i = 0; i <= nc; ++i)
        if (sqrt(suf[i]) <= thr) return i;
    return nc;
}

}  // namespace hm
