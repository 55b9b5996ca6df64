/*
 * RWG / EFIE Galerkin matrix entries (paper Sec. 2, Eq. 7) and partially pivoted ACA
 * (Sec. 2, Eqs. 9-10).  This is the seeded input generator of the solver: it produces
 * the near-field blocks and far-field low-rank factors that the preconditioned solve
 * consumes.  It contains none of the preconditioner or Krylov arithmetic.
 *
 * Conventions: time factor e^{+j w t}, Green's function G = e^{-jkR}/R, lambda = 1,
 * k = 2*pi (passed in), eta0 passed in.  With w*mu = k*eta0 and 1/(w*eps) = eta0/k,
 * Eq. 7 becomes
 *     Z(m,n) = (j k eta0 / 4 pi) [ <f_m, G f_n> - k^-2 <div f_m, G div f_n> ].
 *
 * Quadrature: the 7-point degree-5 rule of Radon on both triangles of every pair.
 * Close pairs (centroid distance below max(r_abs, c_rel*(size_p+size_q)/2)) use
 * singularity extraction: G = (e^{-jkR}-1)/R + 1/R; the smooth part by the 7x7 rule
 * (limit -jk at R = 0), the 1/R and rho/R source integrals in closed form (the
 * potential integrals of Wilton et al. 1984 / Graglia 1993, written out below) and the
 * test integral by the 7-point rule.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no ISA-specific flags).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define NQ 7

typedef struct {
    int nt, nb;
    double k, eta0, r_abs, c_rel;
    double *tv;    /* [nt][3][3] vertices */
    double *tn;    /* [nt][3] unit normal (from vertex order) */
    double *ta;    /* [nt] area */
    double *tc;    /* [nt][3] centroid */
    double *ts;    /* [nt] longest edge */
    double *tq;    /* [nt][NQ][3] quadrature points */
    int32_t *btri; /* [nb][2] */
    double *bfree; /* [nb][2][3] */
    double *blen;  /* [nb] */
} efie_ctx;

static double QW[NQ];
static double QB[NQ][3];

static void init_rule(void)
{
    /* Radon's 7-point rule, exact to degree 5 on a triangle (weights sum to one). */
    double s15 = sqrt(15.0);
    double a = (6.0 - s15) / 21.0, b = (6.0 + s15) / 21.0;
    double wa = (155.0 - s15) / 1200.0, wb = (155.0 + s15) / 1200.0;
    double bc[NQ][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                        {1 - 2 * a, a, a}, {a, 1 - 2 * a, a}, {a, a, 1 - 2 * a},
                        {1 - 2 * b, b, b}, {b, 1 - 2 * b, b}, {b, b, 1 - 2 * b}};
    double w[NQ] = {9.0 / 40.0, wa, wa, wa, wb, wb, wb};
    for (int i = 0; i < NQ; ++i) {
        QW[i] = w[i];
        for (int j = 0; j < 3; ++j) QB[i][j] = bc[i][j];
    }
}

static inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void sub3(const double *a, const double *b, double *c) { c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2]; }
static inline void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double norm3(const double *a) { return sqrt(dot3(a, a)); }

void efie_rule(double *w, double *bary)
{
    init_rule();
    for (int i = 0; i < NQ; ++i) {
        w[i] = QW[i];
        for (int j = 0; j < 3; ++j) bary[3 * i + j] = QB[i][j];
    }
}

void *efie_create(int nv, const double *V, int nt, const int32_t *T, int nb, const int32_t *btri,
                  const int32_t *bfree, double k, double eta0, double r_abs, double c_rel)
{
    (void)nv;
    init_rule();
    efie_ctx *c = (efie_ctx *)calloc(1, sizeof(efie_ctx));
    c->nt = nt; c->nb = nb; c->k = k; c->eta0 = eta0; c->r_abs = r_abs; c->c_rel = c_rel;
    c->tv = malloc(sizeof(double) * 9 * nt);
    c->tn = malloc(sizeof(double) * 3 * nt);
    c->ta = malloc(sizeof(double) * nt);
    c->tc = malloc(sizeof(double) * 3 * nt);
    c->ts = malloc(sizeof(double) * nt);
    c->tq = malloc(sizeof(double) * 3 * NQ * nt);
    for (int t = 0; t < nt; ++t) {
        double *P = c->tv + 9 * t;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) P[3 * i + j] = V[3 * T[3 * t + i] + j];
        double e1[3], e2[3], e3[3], nn[3];
        sub3(P + 3, P, e1); sub3(P + 6, P, e2); sub3(P + 6, P + 3, e3);
        cross3(e1, e2, nn);
        double an = norm3(nn);
        c->ta[t] = 0.5 * an;
        for (int j = 0; j < 3; ++j) {
            c->tn[3 * t + j] = nn[j] / an;
            c->tc[3 * t + j] = (P[j] + P[3 + j] + P[6 + j]) / 3.0;
        }
        double s = norm3(e1);
        if (norm3(e2) > s) s = norm3(e2);
        if (norm3(e3) > s) s = norm3(e3);
        c->ts[t] = s;
        for (int q = 0; q < NQ; ++q)
            for (int j = 0; j < 3; ++j)
                c->tq[(t * NQ + q) * 3 + j] = QB[q][0] * P[j] + QB[q][1] * P[3 + j] + QB[q][2] * P[6 + j];
    }
    c->btri = malloc(sizeof(int32_t) * 2 * nb);
    c->bfree = malloc(sizeof(double) * 6 * nb);
    c->blen = malloc(sizeof(double) * nb);
    for (int n = 0; n < nb; ++n) {
        c->btri[2 * n] = btri[2 * n];
        c->btri[2 * n + 1] = btri[2 * n + 1];
        for (int s = 0; s < 2; ++s)
            for (int j = 0; j < 3; ++j) c->bfree[6 * n + 3 * s + j] = V[3 * bfree[2 * n + s] + j];
        /* edge length: the two non-free vertices of T+ */
        const int32_t *tt = T + 3 * btri[2 * n];
        double ev[2][3];
        int m = 0;
        for (int i = 0; i < 3; ++i)
            if (tt[i] != bfree[2 * n]) {
                for (int j = 0; j < 3; ++j) ev[m][j] = V[3 * tt[i] + j];
                ++m;
            }
        double d[3];
        sub3(ev[1], ev[0], d);
        c->blen[n] = norm3(d);
    }
    return c;
}

void efie_destroy(void *p)
{
    efie_ctx *c = (efie_ctx *)p;
    if (!c) return;
    free(c->tv); free(c->tn); free(c->ta); free(c->tc); free(c->ts); free(c->tq);
    free(c->btri); free(c->bfree); free(c->blen);
    free(c);
}

/* log((R+ + l+)/(R- + l-)) written so that neither factor cancels. */
static inline double edge_log(double lp, double lm, double Rp, double Rm)
{
    if (lp + lm >= 0.0) return log((Rp + lp) / (Rm + lm));
    return log((Rm - lm) / (Rp - lp));
}

/*
 * Closed-form source integrals over the flat triangle with vertices P[0..2] (normal n):
 *   S0 = \int 1/|r - r'| ds',   Sv = \int (r' - rho)/|r - r'| ds',
 * rho = projection of r onto the triangle plane.  For each edge i (from a to b), with
 * unit tangent l, outward in-plane normal u = l x n, d = n.(r - P0):
 *   l+- = (b|a - rho).l, P0 = (a - rho).u, R0^2 = P0^2 + d^2, R+- = sqrt(l+-^2 + R0^2),
 *   S0 = sum_i P0 log((R+ + l+)/(R- + l-))
 *        - |d| sum_i [atan(P0 l+/(R0^2 + |d| R+)) - atan(P0 l-/(R0^2 + |d| R-))],
 *   Sv = 1/2 sum_i u_i [R0^2 log((R+ + l+)/(R- + l-)) + l+ R+ - l- R-].
 */
void efie_potint(const double *P, const double *n, const double *r, double *S0, double *Sv)
{
    double d = n[0] * (r[0] - P[0]) + n[1] * (r[1] - P[1]) + n[2] * (r[2] - P[2]);
    double ad = fabs(d);
    double rho[3] = {r[0] - d * n[0], r[1] - d * n[1], r[2] - d * n[2]};
    double s0 = 0.0, sv[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
        const double *a = P + 3 * i;
        const double *b = P + 3 * ((i + 1) % 3);
        double e[3], l[3], u[3], am[3], bm[3];
        sub3(b, a, e);
        double le = norm3(e);
        for (int j = 0; j < 3; ++j) l[j] = e[j] / le;
        cross3(l, n, u);
        sub3(a, rho, am);
        sub3(b, rho, bm);
        double lp = dot3(bm, l), lm = dot3(am, l);
        double P0 = dot3(am, u);
        double R02 = P0 * P0 + d * d;
        double Rp = sqrt(lp * lp + R02), Rm = sqrt(lm * lm + R02);
        double f2 = 0.0;
        double scale = le;
        if (R02 > 1e-24 * scale * scale) f2 = edge_log(lp, lm, Rp, Rm);
        s0 += P0 * f2;
        if (ad > 0.0 && fabs(P0) > 0.0)
            s0 -= ad * (atan(P0 * lp / (R02 + ad * Rp)) - atan(P0 * lm / (R02 + ad * Rm)));
        double g = R02 * f2 + lp * Rp - lm * Rm;
        for (int j = 0; j < 3; ++j) sv[j] += 0.5 * u[j] * g;
    }
    *S0 = s0;
    for (int j = 0; j < 3; ++j) Sv[j] = sv[j];
}

/* Smooth kernel (e^{-jkR} - 1)/R with the R -> 0 limit -jk, cos-1 written as -2 sin^2. */
static inline cplx gsmooth(double k, double R)
{
    if (R < 1e-14) return -I * k;
    double kr = k * R;
    double s = sin(0.5 * kr);
    return (-2.0 * s * s - I * sin(kr)) / R;
}

/*
 * Triangle pair integrals with the areas included:
 *   I0 = \int_p \int_q G,  Ir = \int\int G r,  Irp = \int\int G r',  Irr = \int\int G r.r'
 */
static void pair_integrals(const efie_ctx *c, int p, int q, cplx *I0, cplx Ir[3], cplx Irp[3], cplx *Irr)
{
    const double *qp = c->tq + (size_t)p * NQ * 3;
    const double *qq = c->tq + (size_t)q * NQ * 3;
    double k = c->k;
    double dc[3];
    sub3(c->tc + 3 * p, c->tc + 3 * q, dc);
    double dist = norm3(dc);
    double thr = 0.5 * c->c_rel * (c->ts[p] + c->ts[q]);
    if (thr < c->r_abs) thr = c->r_abs;
    int close = (p == q) || (dist < thr);
    cplx i0 = 0, irr = 0, ir[3] = {0, 0, 0}, irp[3] = {0, 0, 0};
    double Ap = c->ta[p], Aq = c->ta[q];
    for (int a = 0; a < NQ; ++a) {
        const double *ra = qp + 3 * a;
        cplx in0 = 0, inv[3] = {0, 0, 0};
        for (int b = 0; b < NQ; ++b) {
            const double *rb = qq + 3 * b;
            double dd[3];
            sub3(ra, rb, dd);
            double R = norm3(dd);
            cplx g;
            if (close) {
                g = gsmooth(k, R);
            } else {
                double kr = k * R;
                g = (cos(kr) - I * sin(kr)) / R;
            }
            cplx wg = QW[b] * g;
            in0 += wg;
            inv[0] += wg * rb[0];
            inv[1] += wg * rb[1];
            inv[2] += wg * rb[2];
        }
        in0 *= Aq;
        inv[0] *= Aq; inv[1] *= Aq; inv[2] *= Aq;
        if (close) {
            double S0, Sv[3];
            const double *nq = c->tn + 3 * q;
            efie_potint(c->tv + 9 * q, nq, ra, &S0, Sv);
            double d = dot3(nq, ra) - dot3(nq, c->tv + 9 * q);
            double rho[3] = {ra[0] - d * nq[0], ra[1] - d * nq[1], ra[2] - d * nq[2]};
            in0 += S0;
            for (int j = 0; j < 3; ++j) inv[j] += Sv[j] + rho[j] * S0;
        }
        double wa = QW[a];
        i0 += wa * in0;
        for (int j = 0; j < 3; ++j) {
            ir[j] += wa * ra[j] * in0;
            irp[j] += wa * inv[j];
        }
        irr += wa * (ra[0] * inv[0] + ra[1] * inv[1] + ra[2] * inv[2]);
    }
    *I0 = Ap * i0;
    *Irr = Ap * irr;
    for (int j = 0; j < 3; ++j) {
        Ir[j] = Ap * ir[j];
        Irp[j] = Ap * irp[j];
    }
}

/* Z(m, n) of Eq. 7 for RWG functions m (test) and n (source). */
static cplx entry(const efie_ctx *c, int m, int n)
{
    cplx zA = 0, zP = 0;
    for (int s = 0; s < 2; ++s) {
        int p = c->btri[2 * m + s];
        const double *vm = c->bfree + 6 * m + 3 * s;
        double sm = s == 0 ? 1.0 : -1.0;
        for (int t = 0; t < 2; ++t) {
            int q = c->btri[2 * n + t];
            const double *vn = c->bfree + 6 * n + 3 * t;
            double sn = t == 0 ? 1.0 : -1.0;
            cplx I0, Ir[3], Irp[3], Irr;
            pair_integrals(c, p, q, &I0, Ir, Irp, &Irr);
            double inv = 1.0 / (c->ta[p] * c->ta[q]);
            cplx dotterm = Irr - (vn[0] * Ir[0] + vn[1] * Ir[1] + vn[2] * Ir[2])
                           - (vm[0] * Irp[0] + vm[1] * Irp[1] + vm[2] * Irp[2]) + dot3(vm, vn) * I0;
            zA += sm * sn * 0.25 * inv * dotterm;
            zP += sm * sn * inv * I0;
        }
    }
    double lm = c->blen[m], ln = c->blen[n];
    double k = c->k;
    return (I * k * c->eta0 / (4.0 * M_PI)) * lm * ln * (zA - zP / (k * k));
}

/*
 * Dense blocks: block b has rows ridx[rptr[b]..rptr[b+1]) and columns
 * cidx[cptr[b]..cptr[b+1]); it is written column-major at out + off[b] (complex).
 */
void efie_fill_blocks(void *ctx, int nblk, const int64_t *rptr, const int32_t *ridx, const int64_t *cptr,
                      const int32_t *cidx, const int64_t *off, double *out)
{
    efie_ctx *c = (efie_ctx *)ctx;
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < nblk; ++b) {
        int64_t m = rptr[b + 1] - rptr[b], n = cptr[b + 1] - cptr[b];
        const int32_t *R = ridx + rptr[b];
        const int32_t *C = cidx + cptr[b];
        cplx *ob = o + off[b];
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < m; ++i) ob[i + j * m] = entry(c, R[i], C[j]);
    }
}

/*
 * Partially pivoted ACA of one block (rows R, cols C).  Returns the rank r and sets
 * *Uo (m x r) and *Vo (n x r), column-major, block ~= U V^T (malloc'd, caller frees
 * with efie_free); returns -1 (no factors) if maxr steps did not satisfy the stop rule.
 *
 * Pivoting: first row = local row 0; column pivot = argmax |residual row| over unused
 * columns (lowest index on ties); next row = argmax |u_k| over unused rows.  A zero
 * residual row marks that row used and moves to the next unused row.  Stop when
 * |u_k||v_k| <= eps ||A_k||_F with the usual recursive norm update.
 */
static int aca_one(const efie_ctx *c, int m, const int32_t *R, int n, const int32_t *C, double eps, int maxr,
                   cplx **Uo, cplx **Vo)
{
    char *urow = calloc(m, 1), *ucol = calloc(n, 1);
    cplx *row = malloc(sizeof(cplx) * n);
    int cap = 16;
    cplx *U = malloc(sizeof(cplx) * (size_t)m * cap), *V = malloc(sizeof(cplx) * (size_t)n * cap);
    double nrm2 = 0.0;
    int r = 0, istar = 0, result = -1;
    int rows_left = m;
    while (r < maxr && rows_left > 0) {
        for (int j = 0; j < n; ++j) {
            cplx z = entry(c, R[istar], C[j]);
            for (int l = 0; l < r; ++l) z -= U[istar + (size_t)l * m] * V[j + (size_t)l * n];
            row[j] = z;
        }
        urow[istar] = 1;
        --rows_left;
        int jstar = -1;
        double best = 0.0;
        for (int j = 0; j < n; ++j)
            if (!ucol[j] && cabs(row[j]) > best) {
                best = cabs(row[j]);
                jstar = j;
            }
        if (jstar < 0 || best == 0.0) {
            int nx = -1;
            for (int i = 0; i < m; ++i)
                if (!urow[i]) { nx = i; break; }
            if (nx < 0) { result = r; break; }
            istar = nx;
            continue;
        }
        if (r == cap) {
            cap *= 2;
            U = realloc(U, sizeof(cplx) * (size_t)m * cap);
            V = realloc(V, sizeof(cplx) * (size_t)n * cap);
        }
        cplx piv = row[jstar];
        cplx *v = V + (size_t)r * n;
        cplx *u = U + (size_t)r * m;
        for (int j = 0; j < n; ++j) v[j] = row[j] / piv;
        for (int i = 0; i < m; ++i) {
            cplx z = entry(c, R[i], C[jstar]);
            for (int l = 0; l < r; ++l) z -= U[i + (size_t)l * m] * V[jstar + (size_t)l * n];
            u[i] = z;
        }
        ucol[jstar] = 1;
        double nu2 = 0, nv2 = 0;
        for (int i = 0; i < m; ++i) nu2 += creal(u[i] * conj(u[i]));
        for (int j = 0; j < n; ++j) nv2 += creal(v[j] * conj(v[j]));
        double cross = 0.0;
        for (int l = 0; l < r; ++l) {
            cplx su = 0, sv = 0;
            for (int i = 0; i < m; ++i) su += conj(U[i + (size_t)l * m]) * u[i];
            for (int j = 0; j < n; ++j) sv += conj(V[j + (size_t)l * n]) * v[j];
            cross += creal(su * sv);
        }
        nrm2 += 2.0 * cross + nu2 * nv2;
        ++r;
        if (sqrt(nu2 * nv2) <= eps * sqrt(fabs(nrm2))) { result = r; break; }
        int nx = -1;
        best = -1.0;
        for (int i = 0; i < m; ++i)
            if (!urow[i] && cabs(u[i]) > best) {
                best = cabs(u[i]);
                nx = i;
            }
        if (nx < 0) { result = r; break; }
        istar = nx;
    }
    if (result < 0 && rows_left == 0) result = r;
    free(urow); free(ucol); free(row);
    if (result < 0) {
        free(U); free(V);
        *Uo = *Vo = NULL;
    } else {
        *Uo = U;
        *Vo = V;
    }
    return result;
}

/*
 * Batched ACA over nblk far blocks; block b gets rank[b] (or -1) and malloc'd factors
 * uptr[b] (m x r), vptr[b] (n x r), released with efie_free.
 */
void efie_aca_blocks(void *ctx, int nblk, const int64_t *rptr, const int32_t *ridx, const int64_t *cptr,
                     const int32_t *cidx, double eps, const int32_t *maxr, void **uptr, void **vptr, int32_t *rank)
{
    efie_ctx *c = (efie_ctx *)ctx;
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < nblk; ++b) {
        int m = (int)(rptr[b + 1] - rptr[b]), n = (int)(cptr[b + 1] - cptr[b]);
        cplx *U, *V;
        rank[b] = aca_one(c, m, ridx + rptr[b], n, cidx + cptr[b], eps, maxr[b], &U, &V);
        uptr[b] = U;
        vptr[b] = V;
    }
}

void efie_free(void *p) { free(p); }
