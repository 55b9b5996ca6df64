/*
 * hmsolve — GPU (sm_103a) solver for ACA-compressed H-matrix RWG/EFIE systems Z I = V
 * with the symmetric near-field Schur-complement preconditioner of arXiv 2111.13483.
 *
 * Problem statement (Sec. 3.1, Eq. 11): Z = Z_N + Z_F, Z_N the dense near-field leaf
 * blocks, Z_F the far-field low-rank blocks (Sec. 2, Eqs. 9-10).  The library reorders
 * the leaf blocks (Sec. 3.3, Algorithm 1, reverse Cuthill-McKee), eliminates the near
 * field block by block with symmetric Schur complements (Sec. 3.1-3.2, Eqs. 12-21),
 * optionally compresses the fill-in coefficient blocks (Sec. 3.4), and solves the
 * block-diagonally preconditioned transformed system (Eqs. 22-28) with restarted GMRES
 * (Sec. 5).
 *
 * Conventions for every call:
 *   - complex numbers are hm_c128 (interleaved re, im, 16 bytes), matrices column-major;
 *   - all indices are 0-based; "cluster order" is the order of the leaves of the
 *     cluster tree, each leaf a contiguous range of positions;
 *   - every call returns an HM_* status and never aborts; hm_last_error() explains the
 *     last failure on a handle;
 *   - host pointers passed in are read during the call only (the library deep-copies);
 *     output buffers are caller-allocated;
 *   - a handle is used from one host thread at a time and orders all its GPU work on
 *     its stream (hm_opts.stream, or a stream it creates).
 */
#ifndef HMSOLVE_H
#define HMSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hm_ctx *hm_handle;
typedef struct {
    double re, im;
} hm_c128;

enum {
    HM_OK = 0,
    HM_EINVAL = -1,     /* bad argument or inconsistent description */
    HM_ENOMEM = -2,     /* device allocation failed or hbm_budget exceeded */
    HM_ESINGULAR = -3,  /* a pivot block D_k is numerically singular (Sec. 3.1, Eq. 14) */
    HM_ENOCONV = -4,    /* maxit reached; the best iterate, iters and relres are written */
    HM_ETIMEOUT = -5,   /* a device-side bounded wait expired (no hang; context usable) */
    HM_ECUDA = -6,      /* CUDA runtime error */
    HM_ESTATE = -7,     /* call out of order (e.g. solve before precond_setup) */
    HM_EBUSY = -8       /* hm_batch_submit: every slot is occupied */
};

/*
 * H-matrix description (Sec. 2 Eqs. 8-10, Sec. 3.1 Eq. 11).  All arrays host memory.
 *   n, n_leaves   unknowns and leaf clusters;
 *   perm[n]       original RWG index of cluster-order position i;
 *   leaf_ptr[n_leaves+1]  leaf l covers positions [leaf_ptr[l], leaf_ptr[l+1]), 1..64 each;
 *   near pairs b < n_near: leaves near_t[b] <= near_s[b]; block Z(t-rows, s-cols) is
 *       stored column-major at near_data + near_off[b] (n_t x n_s entries); the (s, t)
 *       block is its transpose (Z is complex symmetric, Sec. 3.2).  Every (t, t) pair must
 *       be present and each unordered pair at most once;
 *   far blocks b < n_far: cluster-order ranges rows [far_r0, far_r1), cols [far_c0,
 *       far_c1) with far_r1 <= far_c0 (upper half; the mirrored block is the transpose);
 *       far_rank[b] = r >= 0: block = U V^T with U (m x r) at far_U + far_uoff[b] and
 *       V (n x r) at far_V + far_voff[b]; far_rank[b] = -1: dense m x n block at
 *       far_U + far_uoff[b].  Near and far blocks together must cover every entry once.
 *   near_len, far_U_len, far_V_len: lengths (entries) of the three data arrays.
 */
typedef struct {
    int32_t n, n_leaves;
    const int32_t *perm;
    const int32_t *leaf_ptr;
    int32_t n_near;
    const int32_t *near_t, *near_s;
    const int64_t *near_off;
    const hm_c128 *near_data;
    int64_t near_len;
    int32_t n_far;
    const int32_t *far_r0, *far_r1, *far_c0, *far_c1;
    const int32_t *far_rank;
    const int64_t *far_uoff, *far_voff;
    const hm_c128 *far_U, *far_V;
    int64_t far_U_len, far_V_len;
} hm_desc;

/*
 *   ordering   0 = keep the cluster order, 1 = reverse Cuthill-McKee, 2 = Sloan (the
 *              Algorithm 1 orderings compared in Sec. 3.3, Tables 3-4; see hm_plan_order_method);
 *   fill_tol   Sec. 3.4 compression tolerance for fill-in coefficient blocks, 0 = off;
 *   precision  0 = complex FP64 throughout; 1 = complex FP32 operator/preconditioner
 *              inside an FP64 refinement loop on Z (FP64 pivots, Arnoldi, residual);
 *   device     CUDA device ordinal;
 *   hbm_budget bytes the handle may allocate on the device, 0 = no limit;
 *   stream     cudaStream_t to order work on, NULL = the library creates one;
 *   preconditioner  0 = the symmetric near-field Schur complement (Sec. 3, Eq. 28);
 *              1 = block Jacobi, M = the near-field diagonal blocks Z_kk (the block diagonal
 *              preconditioner of Sec. 1, a comparison): GMRES on M^{-1} Z x = M^{-1} b with
 *              the same engine, no coefficients, blocks in the ordering's order; precision 0
 *              only (HM_EINVAL otherwise);
 *              2 = null field, the one-sided comparison of Sec. 3 and Sec. 5.2 as read here:
 *              the elimination of Sec. 3.1 restricted to the near-field pattern (S_k = the
 *              later near-field neighbours of k; an update whose target block is not a
 *              near-field pair is dropped), M = L D L^T, and GMRES on M^{-1} Z x = M^{-1} b
 *              with M^{-1} = L^{-T} D^{-1} L^{-1} applied from the left (x~ = x); no fill-in
 *              blocks, so fill_tol has nothing to compress; precision 0 only (HM_EINVAL
 *              otherwise);
 *   compress_in_setup  with fill_tol > 0: 0 = the fill-in coefficient blocks are truncated once
 *              the elimination is complete and only the sweeps use the truncations; 1 = each is
 *              truncated as soon as its elimination step forms it, so that the Schur updates of
 *              that step (and every later block) use it (the abstract has the fill-in blocks
 *              compressed while the preconditioner is computed; Sec. 3.4 is silent on the point).
 */
typedef struct {
    int32_t ordering;
    double fill_tol;
    int32_t precision;
    int32_t device;
    size_t hbm_budget;
    void *stream;
    int32_t preconditioner;
    int32_t compress_in_setup;
} hm_opts;

typedef struct {
    int32_t n, n_blocks;
    int64_t near_entries;     /* stored near-field entries (t <= s blocks) */
    int64_t far_entries;      /* stored far-field entries, sum r (m + n) + dense m n */
    int64_t fill_blocks;      /* sum_k |S_k| coefficient blocks (Sec. 3.3 fill) */
    int64_t coef_entries;     /* coefficient entries as stored: dense n_k n_j + r (n_k + n_j) */
    int64_t coef_entries_dense; /* same without compression */
    int64_t diag_entries;     /* sum_k n_k^2 */
    int32_t bandwidth;        /* block bandwidth of the near-field graph in solve order */
    double setup_ms;          /* device time of the last precond_setup */
    double setup_gflop;       /* algorithmic flops of setup (8 real flops per complex MAC) */
    size_t device_bytes;      /* bytes currently allocated on the device by the handle */
} hm_stats;

/* Fills *o with the defaults: RCM, fill_tol 0, FP64, device 0, no budget, own stream, Schur. */
int hm_default_opts(hm_opts *o);

/*
 * Validates *d, copies the near blocks, far factors and index maps to the device and
 * plans the solve order (Algorithm 1 steps 1-5) and the symbolic fill of the scaling
 * coefficients.  On success *out receives a new handle.  HM_EINVAL on a malformed
 * description, HM_ENOMEM when allocation fails or exceeds opts->hbm_budget.
 */
int hmat_create(const hm_desc *d, const hm_opts *opts, hm_handle *out);

/*
 * Symmetric near-field Schur elimination (Sec. 3.1-3.2): for each block k in solve
 * order D_k = A_kk, W_kj = D_k^{-1} A_kj (the negated right coefficients, Eq. 14; the
 * left ones are their transposes), A_ij -= A_ik W_kj for i >= j later neighbours
 * (Eq. 19); then the Sec. 3.4 compression of fill-in W blocks when fill_tol > 0, and
 * D_k^{-1} for the Eq. 28 preconditioner.  Every call recomputes the factors from the
 * resident near-field blocks (same result each time).  HM_ESINGULAR names the block in
 * hm_last_error.
 */
int precond_setup(hm_handle h);

/*
 * Solves Z I = V for nrhs right-hand sides given in the ORIGINAL RWG order, host
 * memory: V column j at V + j*ldv, I column j at I + j*ldi (ldv, ldi >= n).  GMRES(restart)
 * on Eq. 28 until the preconditioned relative residual is <= tol (FP64 mode) or, in
 * mixed mode, until ||V - Z I|| / ||V|| <= tol.  iters[j] = Arnoldi steps taken for
 * column j (inner steps in mixed mode), relres[j] = final relative residual of the
 * criterion above.  Each column has its own Krylov space; up to 64 columns (mixed mode)
 * or 16 (FP64) are in flight at a time, sharing each operator launch, and a finished
 * column's place is taken by the next (the hm_batch engine below).  A column's result
 * does not depend on the others.  HM_ENOCONV if some column did not converge within
 * maxit (its best iterate is still written).  In mixed mode the inner solves run to
 * min(0.5, max(1e-7, 0.6 tol ||V|| / ||V - Z I||, 0.1 rho)), rho = the factor by which the
 * last refinement pass reduced ||V - Z I|| (fill_tol before the first pass), and at most 40
 * refinement passes are made.
 */
int solve(hm_handle h, const hm_c128 *V, int32_t nrhs, int64_t ldv, double tol, int32_t restart,
          int32_t maxit, hm_c128 *I, int64_t ldi, int32_t *iters, double *relres);

/* As solve(), with V and I in device memory (e.g. torch tensors), ordered on the handle's
 * stream.  iters and relres are host arrays. */
int solve_device(hm_handle h, const void *dV, int32_t nrhs, int64_t ldv, double tol, int32_t restart,
                 int32_t maxit, void *dI, int64_t ldi, int32_t *iters, double *relres);

int hmat_stats(hm_handle h, hm_stats *s);
const char *hm_last_error(hm_handle h);
void hmat_destroy(hm_handle h);

/* ---- inspection entry points (parity tests and diagnostics) ---------------------- */

/* Solve order: order[p] = leaf (cluster order) placed at block position p.  n_leaves entries. */
int hm_get_order(hm_handle h, int32_t *order);

/* Symbolic fill S_k of Sec. 3.3: ptr[n_blocks+1] and idx[ptr[n_blocks]] (sorted block
 * positions > k).  Pass idx = NULL to query ptr only. */
int hm_get_fill(hm_handle h, int32_t *ptr, int32_t *idx);

/*
 * Copies factor blocks to host memory after precond_setup, in solve order:
 *   what 0: D_k        (n_k x n_k)  the scaled near-field block of Eq. 21;
 *   what 1: D_k^{-1}   (n_k x n_k);
 *   what 2: W_k        (n_k x sum_{j in S_k} n_j) the coefficient row of block k as the
 *                      sweeps apply it, blocks in S_k order: with fill_tol > 0 the fill-in
 *                      blocks are their Sec. 3.4 truncations (low-rank blocks expanded);
 *   what 3: same as 2.
 * out must hold the stated number of entries.
 */
int hm_get_block(hm_handle h, int32_t what, int32_t k, hm_c128 *out);

/* Sec. 3.4 ranks of the last precond_setup, one per entry of the S_k lists (hm_get_fill
 * order): r >= 0 = fill-in block kept at rank r, -1 = dense (near-pattern block, no
 * compression requested, or a truncation that would not save storage). */
int hm_get_fill_ranks(hm_handle h, int32_t *rank);

/*
 * Applies one operator to nrhs device vectors (solve order, column-major, ld = n):
 *   op 0: y = A x   with A = D^{-1}[D + L^{-1} Z_F L^{-T}]  (Eq. 28, paper form); for the
 *         comparison preconditioners A = M^{-1} Z (block Jacobi: M^{-1} = D^{-1}, ops 1 and
 *         2 copy; null field: M^{-1} = L^{-T} D^{-1} L^{-1});
 *   op 1: y = L^{-1} x     (Eq. 23, the left scalings);
 *   op 2: y = L^{-T} x     (Eq. 24, the right scalings);
 *   op 3: y = Z_F x        (far field, Eq. 11);
 *   op 4: y = D^{-1} x     (Eq. 28 preconditioner solve);
 *   op 5: y = Z x          (near + far, ORIGINAL order; the refinement residual operator);
 *   ops 8-12: ops 0-4 with the complex-FP32 factors and arithmetic of the mixed-precision
 *       inner solve (x and y stay complex FP64); precision 1 handles only (else HM_ESTATE).
 * x and y must not overlap.
 */
int hm_apply(hm_handle h, int32_t op, const void *dx, void *dy, int32_t nrhs);

/* Solution-order index map: new2orig[p] = original RWG index at solve-order position p. */
int hm_get_index_map(hm_handle h, int32_t *new2orig);

/*
 * Kernel accounting.  Every launch is counted by kernel class:
 *   0 near scatter, 1 pivot inverse, 2 coefficient panel, 3 Schur update, 4 forward sweep,
 *   5 backward sweep, 6 far phase 1, 7 far phase 2, 8 block diagonal, 9 permutations,
 *   10 near product, 11 dot products, 12 vector updates, 13 small GMRES kernels,
 *   14 fill-in compression.
 * hm_profile(mode): 1 = also time each launch with CUDA events on the handle's stream,
 * 0 = stop timing, 2 = zero all counters.  hm_get_profile returns, for one class, the
 * launches counted, the launches timed and their summed device time in ms.
 */
int hm_profile(hm_handle h, int32_t mode);
int hm_get_profile(hm_handle h, int32_t cls, int64_t *launches, int64_t *timed, double *ms);
/* Right-hand-side columns processed by class cls since the last reset, summed over its calls
 * (counted for the sweeps, classes 4-5, and the far-field product, classes 6-7; else 0). */
int hm_get_profile_cols(hm_handle h, int32_t cls, int64_t *cols);

/*
 * Far-field product y = Z_F x (as hm_apply op 3) that allocates no device memory; the paper
 * has no counterpart, it exists for callers that must not call cudaMalloc / cudaFree at
 * the point of the call (cudaFree synchronises the whole device, which a serving loop with
 * several busy streams cannot afford; a process whose device memory sits in another
 * allocator's pool may see cudaMalloc fail).  x, y: nrhs device vectors in solve order,
 * column-major, ld = n, not overlapping.  Scratch is one static 16 MiB device array
 * (1,048,576 complex doubles) held by every GPU that loads the library until exit; a call
 * needing more than n*nrhs + 2*sum(rank)*nrhs entries of it returns HM_EINVAL.  The first
 * call on a device looks up the array's device address.  The address is cached per device for the life of the process and belongs to the device's
 * primary context as the first call found it: after cudaDeviceReset the library must be
 * unloaded and loaded again before this call is used.  All calls share the array, so calls that overlap on the GPU race and must be serialised.
 * Synchronises the handle's stream before returning.
 */
int hm_far_apply_noalloc(hm_handle h, const void *dx, void *dy, int32_t nrhs);

/*
 * Schedule of the block-triangular sweeps (Eqs. 23, 24): the right-hand-side columns of a
 * launch are split into `groups` (1, 2 or 4) independent chains, and `kind` selects how a
 * chain is computed: 1 = one CTA per block row; 2 = one CTA per two consecutive block rows;
 * 3 = one chain CTA walks all block rows adding the dependencies of the last four rows
 * from shared memory, while one helper CTA per block row adds all older dependencies;
 * 4 = one CTA per block row with the block products on the tensor cores (complex-FP32
 * sweeps of a precision 1 handle: TF32 operands split into a rounded part and a remainder,
 * FP32 accumulation; the FP64 sweeps take kind 1 for it); 5 and 6 = one CTA per block row in
 * thread-block clusters of 8 and 16 CTAs (16 where the device fits them, else 8) that take
 * consecutive block rows, a row reading the results of earlier rows of its cluster from their
 * shared memory (complex-FP32 sweeps; the FP64 sweeps take kind 1 for them).  Kinds 1-3, 5
 * and 6 give bitwise the same result, and kind 4 gives bitwise the same result for every
 * number of groups.  (0, 0) -- the default -- lets the library time kind 1 with 1, 2 and 4
 * groups and each tile on its first calls of each width and keep the fastest.
 * Kinds 2 and 3 apply to groups of at most 16 columns (kind 1 otherwise).  With compressed
 * fill-in blocks (fill_tol > 0) kinds 2-4 take kind 1.  `tile` (kind 1) selects the
 * register tile of each thread -- rows x columns x tiles per thread -- for groups of 5-16
 * columns: 0 = 2 x 2 x 1, 1 = 1 x 2 x 2, 2 = 1 x 1 x 4; for 17-64 columns: 0 = 2 x 4 x 2,
 * 1 = 2 x 2 x 4, 2 = 1 x 4 x 4 (1 x 1 x 1 up to 4 columns); every tile adds an output's terms
 * in the same order, so all give bitwise the same result.  HM_EINVAL for other values.
 */
int hm_set_sweep_schedule(hm_handle h, int32_t groups, int32_t kind, int32_t tile);

/*
 * Test hook for the bounded device-side waits of the sweeps (Eqs. 23, 24; the paper has no
 * counterpart).  After this call every triangular sweep on the handle leaves block row
 * `block` (solve order) out -- it is never computed or published -- and any single wait of a
 * sweep on another block gives up after `wait_ns` nanoseconds (0 = the default bound of 2 s),
 * so the operator or solve that contains the sweep returns HM_ETIMEOUT instead of hanging and
 * the handle stays usable.  hm_test_hold(h, -1, 0) restores normal operation.  Synchronises
 * the handle's stream first.  HM_EINVAL for block outside -1 .. n_blocks-1 or wait_ns < 0.
 */
int hm_test_hold(hm_handle h, int32_t block, int64_t wait_ns);

/*
 * One complex-FP32 block product C = A B, computed by the tensor-core micro-kernel that the
 * complex-FP32 sweeps use for their block products (Eqs. 23, 24: y_i -= W_ki^T y_k and
 * x_k -= W_kj y_j): tcgen05 MMAs on TF32 operands, each FP32 value split into a rounded TF32
 * part and a TF32 remainder (three products per step, the remainder-times-remainder term
 * dropped), accumulated in FP32 in tensor memory.  A is m x k, B is k x ncols, C is m x ncols,
 * column-major, complex FP32 (interleaved re, im floats), device memory; 1 <= m <= 64,
 * 1 <= ncols <= 64, k >= 0 (k = 0 writes zeros).  One CTA on `stream` (NULL = the legacy
 * default stream); synchronises the stream before returning.  A column of C depends only on
 * A and that column of B: it is bitwise the same for any ncols.  HM_EINVAL on bad sizes or
 * leading dimensions (lda >= m, ldb >= k, ldc >= m), HM_ECUDA on a CUDA error.
 */
int hm_tc_cgemm(int32_t m, int32_t k, int32_t ncols, const void *dA, int64_t lda, const void *dB, int64_t ldb,
                void *dC, int64_t ldc, void *stream);

/*
 * How the complex-FP32 far-field product (Z_F u of Sec. 2, Eq. 11, inside the operator of a
 * precision 1 handle) computes its block products: kind 1 = register-tiled FMAs on the CUDA
 * cores, kind 2 = the tensor-core micro-kernel of hm_tc_cgemm; 0 = the default (1: at 64
 * columns on the 30,720-unknown sphere kind 2 took 3.22 against 3.47 ms, at one column 2.07
 * against 0.80 ms, and the choice must not depend on the width).  Both
 * sum every output's terms in a fixed order, each its own; the FP64 far field always runs on
 * the CUDA cores.  HM_EINVAL for other values.
 */
int hm_set_far_schedule(hm_handle h, int32_t kind);

/*
 * How the complex-FP32 Schur updates of a precision 1 handle's precond_setup (Sec. 3.1, Eq. 19:
 * A_ij -= A_ik W_kj for i >= j in S_k, the dense contraction of the elimination) are computed:
 * kind 1 = register-tiled FMAs on the CUDA cores, one CTA per row block and group of column
 * blocks; kind 2 = the tensor-core micro-kernel of hm_tc_cgemm (TF32 operands split into a
 * rounded part and a remainder, FP32 accumulation), one CTA per row block and 64 columns of the
 * panel W_k; 0 = the default (1: on the 30,720-unknown sphere kind 2 took 275 against 252 ms of
 * updates per setup -- its operands are loaded, split and drained by the threads, and the
 * products of ~28-unknown blocks are too short to hide that).  Both sum every output's terms in
 * a fixed order; the FP64 setup always runs on the CUDA cores.  Takes effect at the next
 * precond_setup.  HM_EINVAL for other values.
 */
int hm_set_update_schedule(hm_handle h, int32_t kind);

/*
 * How many CTAs invert each pivot block D_k in precond_setup (Sec. 3.1, Eq. 14: the FP64
 * Gauss-Jordan inverse with partial pivoting that every coefficient panel of step k needs):
 * 1 = one CTA; 2, 4 or 8 = a thread-block cluster of that many CTAs on as many SMs, each
 * eliminating a share of the columns, the pivot column passed through distributed shared
 * memory with one cluster barrier per pivot (same arithmetic per entry: the inverses are bitwise
 * those of one CTA); 0 = the default (8: on the 30,720-unknown sphere the 1,112 inversions of a
 * setup took 200, 162, 123 and 109 ms with 1, 2, 4 and 8 CTAs -- each column step still costs
 * a cluster barrier and the pivot search).  Both precisions; the block-Jacobi setup always
 * uses one CTA per block.  Takes effect at the next precond_setup.  HM_EINVAL for other values.
 */
int hm_set_pivot_schedule(hm_handle h, int32_t ctas);

/* ---- continuous batching (serving) ---------------------------------------------------- */

/*
 * A slot engine over one handle: each of `slots` slots holds one right-hand side and runs
 * its own solve of Z I = V (Eq. 11) through the preconditioned system (Eq. 28) with
 * GMRES(restart) -- FP64, or the mixed-precision refinement loop when the handle's
 * precision is 1 -- exactly as solve() does.  hm_batch_step advances every occupied slot
 * by one GMRES step (one operator application; all slots that need the same operator in a
 * step share one multi-column launch); a slot whose solve has ended is reported, its
 * result is read with hm_batch_result, which frees the slot for the next submission.
 * Requests can therefore join while others are in flight.  A column's result is bitwise
 * the same as solve() on that column alone.  The paper has no serving loop: this layer
 * only schedules its solve.
 *
 * One batch per handle at a time; the handle's stream carries all of its work and a batch
 * is used from one host thread.  The workspace (hm_batch_bytes) is taken from the
 * handle's hbm_budget at open (HM_ENOMEM if it does not fit) and returned at close.
 */
typedef struct hm_batch_s *hm_batch;

/* Device bytes hm_batch_open(h, slots, restart) takes (beyond the operator's own scratch). */
int hm_batch_bytes(hm_handle h, int32_t slots, int32_t restart, int64_t *bytes);
/* 1 <= slots <= 1024, restart >= 1.  HM_ESTATE before precond_setup or with a batch open. */
int hm_batch_open(hm_handle h, int32_t slots, int32_t restart, hm_batch *out);
/*
 * Copies V (n entries, ORIGINAL order; host or device memory) into a free slot, which
 * starts at the next step; *slot = its index.  tol and maxit as in solve().  HM_EBUSY
 * (*slot = -2) when no slot is free.
 */
int hm_batch_submit(hm_batch b, const hm_c128 *V, double tol, int32_t maxit, int32_t *slot);
/*
 * One step of every occupied slot.  finished[] (room for `slots` entries) receives the
 * slots whose solve ended in this step, *nfinished their count, *nactive (may be NULL) the
 * slots still running.  Returns HM_OK, HM_ETIMEOUT or HM_ECUDA (then the batch should be
 * closed).  Synchronises the handle's stream.
 */
int hm_batch_step(hm_batch b, int32_t *finished, int32_t *nfinished, int32_t *nactive);
/*
 * Copies the finished slot's solution I (n entries, ORIGINAL order) to host or device
 * memory and frees the slot.  Returns the solve's status (HM_OK or HM_ENOCONV, with
 * iters/relres as in solve()), or HM_ESTATE when the slot holds no finished solve.
 */
int hm_batch_result(hm_batch b, int32_t slot, hm_c128 *I, int32_t *iters, double *relres);
/* Frees the workspace; unread results are dropped. */
int hm_batch_close(hm_batch b);

/* ---- host-only planning (no device work, no handle) -------------------------------- */

/*
 * Algorithm 1 (Sec. 3.3) steps 1-4 on a leaf graph with n_leaves nodes and n_pairs edges
 * (t[b], s[b]) (self loops and repeats ignored): reverse Cuthill-McKee, components in order
 * of their lowest node, George-Liu pseudo-peripheral start from the minimum-(degree,
 * index) node, neighbours by ascending (degree, index), the whole sequence reversed.
 * order[p] = node placed at position p (n_leaves entries).  HM_EINVAL on bad input.
 */
int hm_plan_order(int32_t n_leaves, int32_t n_pairs, const int32_t *t, const int32_t *s, int32_t *order);

/*
 * Algorithm 1 step 3 with a chosen reordering (Sec. 3.3 compares several, Tables 3-4):
 * method 0 = identity, 1 = reverse Cuthill-McKee as hm_plan_order, 2 = Sloan's profile and
 * wavefront reduction: per component (in order of its lowest node) a start node s and an end
 * node e from rooted level structures (s = the minimum-(degree, index) node; the last level's
 * nodes in ascending (degree, index), one per degree: one whose structure is deeper than s's
 * and narrower than all tried replaces s and the search restarts, one only narrower becomes
 * e), priorities 2 dist(i, e) - (deg(i) + 1), then the queued node of highest priority (lowest
 * index on ties) is numbered next, with the priority updates of Sloan's algorithm (numbering a
 * preactive node raises its neighbours by 1; a node turning active gains 1 and so does each of
 * its neighbours not yet numbered).  Not reversed.  Same arguments and errors as hm_plan_order
 * (HM_EINVAL also for another method).
 */
int hm_plan_order_method(int32_t method, int32_t n_leaves, int32_t n_pairs, const int32_t *t, const int32_t *s,
                         int32_t *order);

/*
 * Symbolic fill of the scaling coefficients (Sec. 3.3, Figs. 3b-7b): for blocks numbered
 * 0..n_blocks-1 with near pairs (i[b], j[b]), S_k = later neighbours of k once the
 * neighbours of every earlier block have been coupled.  ptr[n_blocks+1] always written;
 * idx (sorted S_k lists) written when non-NULL and ptr[n_blocks] <= idx_cap.
 */
int hm_plan_fill(int32_t n_blocks, int32_t n_pairs, const int32_t *i, const int32_t *j, int32_t *ptr,
                 int32_t *idx, int64_t idx_cap);

/*
 * hm_plan_fill with a choice of lists: closure 1 = the symbolic fill (as hm_plan_fill);
 * closure 0 = no fill, S_k = the later near-field neighbours of k only (the lists of the
 * null-field comparison, hm_opts.preconditioner = 2).  Same outputs and errors as
 * hm_plan_fill; HM_EINVAL for other closure values.
 */
int hm_plan_fill_closure(int32_t closure, int32_t n_blocks, int32_t n_pairs, const int32_t *i, const int32_t *j,
                         int32_t *ptr, int32_t *idx, int64_t idx_cap);

/*
 * The library's plan of the far-field product Z_F u (the U (V^T u) products of Sec. 2, Eq. 11,
 * over the admissible blocks of Eq. 8) for the far blocks of an H-matrix description, in
 * cluster order: the same checks as hmat_create on n, leaf_ptr and the far arrays (fields of
 * hm_desc; far_U / far_V are not needed), no device work.  `what` selects one table, written
 * as int64 rows into out:
 *   0  seg_ptr, n_leaves + 1 entries: the phase-2 segments of leaf l are seg_ptr[l] ..
 *      seg_ptr[l+1] - 1;
 *   1  segments, 6 per segment (foff, yrow, fi, fk, len, src): for the leaf's rows a + i,
 *      y[a + i] += sum_{k < len} F[foff + i*fi + k*fk] * Y[yrow + k], with F = far_V when
 *      src & 1 else far_U, and Y = the rank vectors t (src >> 1 == 0), s (1) or u itself (2);
 *   2  part_ptr, n_leaves * parts + 1 entries: part p of leaf l (one CTA) covers segments
 *      part_ptr[l*parts + p] .. part_ptr[l*parts + p + 1] - 1;
 *   3  phase-1 tasks, 4 per task (lo, hi, first item, end item): items contract over the
 *      cluster-order range [lo, hi);
 *   4  phase-1 items, 5 per item (off, ld, rank, row, isv): for l < rank,
 *      (isv ? t : s)[row + l] = sum_{lo <= i < hi} (isv ? far_V : far_U)[off + l*ld + i - lo] * u[i].
 * *count: in, the capacity of out in int64 entries; out, the entries of the table (always
 * written).  out == NULL only queries the count.  HM_EINVAL on bad input or a too small out.
 */
int hm_plan_far(int32_t n, int32_t n_leaves, const int32_t *leaf_ptr, int32_t n_far, const int32_t *far_r0,
                const int32_t *far_r1, const int32_t *far_c0, const int32_t *far_c1, const int32_t *far_rank,
                const int64_t *far_uoff, const int64_t *far_voff, int32_t what, int64_t *out, int64_t *count);

/*
 * The inputs of the solve computed on the device from the mesh (Sec. 2): Galerkin EFIE
 * entries of RWG functions (Eq. 7) and ACA factors of admissible blocks (Eqs. 9-10).  No
 * handle; each call uploads the mesh, runs its kernels on the legacy default stream of
 * `device` and returns when the outputs are in host memory.  All pointers are host pointers,
 * caller-owned, read (or written) during the call only.
 *
 * Mesh: nv vertices V (nv x 3 doubles), nt triangles T (nt x 3 vertex indices), nb RWG
 * functions; tri (nb x 2) the T+ and T- triangle of each, free_v (nb x 2) the vertex of T+
 * and of T- opposite the common edge (the edge length is taken from T+).  Entries use
 * G = e^{-jkR}/R with wavenumber k and impedance eta0 (time factor e^{+jwt}):
 *   Z(m, n) = (j k eta0 / 4 pi) [ <f_m, G f_n> - k^-2 <div f_m, G div f_n> ],
 * Radon's 7-point rule on both triangles; triangle pairs with centroid distance below
 * max(r_abs, c_rel (h_p + h_q) / 2) (h the longest edge) or p == q use singularity extraction
 * with the closed-form 1/R and rho/R integrals.  Blocks: block b has the RWG rows
 * ridx[rptr[b] .. rptr[b+1]-1] and columns cidx[cptr[b] .. cptr[b+1]-1] (rptr[0] = cptr[0]
 * = 0, every block at least 1 x 1, indices in 0 .. nb-1).
 *
 * Blocks are processed in chunks whose device scratch stays within scratch_bytes (0 = 1 GiB;
 * a single block larger than that gets a chunk of its own); the results do not depend on it.
 *
 * Errors: HM_EINVAL on any bad argument (indices out of range, empty blocks, inconsistent
 * offsets, k <= 0, eps outside (0, 1), scratch_bytes < 0); HM_ENOMEM if a device allocation
 * fails; HM_ECUDA on another CUDA error (message on stderr).
 */

/*
 * Dense blocks: block b is written column-major (m_b x n_b, hm_c128) at out + off[b];
 * off has nblk + 1 entries with off[0] = 0 and off[b+1] - off[b] = m_b n_b.  mirror = 1: a
 * block whose row list equals its column list is made exactly symmetric, its lower triangle a
 * copy of its upper one (the symmetric storage of Sec. 3.2); mirror = 0: every entry computed.
 */
int hm_efie_fill(int32_t nv, const double *V, int32_t nt, const int32_t *T, int32_t nb, const int32_t *tri,
                 const int32_t *free_v, double k, double eta0, double r_abs, double c_rel, int32_t nblk,
                 const int64_t *rptr, const int32_t *ridx, const int64_t *cptr, const int32_t *cidx, int32_t mirror,
                 const int64_t *off, hm_c128 *out, int64_t scratch_bytes, int32_t device);

/*
 * Admissible blocks in the layout hm_desc takes for its far field: partially pivoted ACA
 * (first row 0, column pivot = argmax of the residual row's moduli over unused columns, ties to
 * the lowest index, next row = argmax |u_k| over unused rows, a zero residual row moving to
 * the lowest unused row, stop when |u_k| |v_k| <= eps ||A_k||_F), then re-compression (QR of
 * both factors, SVD of the small core, the smallest rank with a Frobenius tail <= eps times the
 * whole).  Per block: rank[b] = r >= 0 with U (m_b x r) at U + uoff[b] and V (n_b x r) at
 * Vf + voff[b], block = U V^T; or rank[b] = -1 with the dense block (m_b x n_b) at U + uoff[b]
 * -- when the ACA rank reached min(m_b, n_b, floor(m_b n_b / (m_b + n_b)) + 1, 256) without the
 * stop rule, or when r (m_b + n_b) >= m_b n_b.  Column-major; blocks follow each other in
 * block order in U and in Vf.  need[0], need[1] (always written) are the entries of U and Vf
 * the layout takes; if they exceed cap_u or cap_v the call still writes rank and returns
 * HM_ENOMEM (U, Vf, uoff, voff then undefined).
 */
int hm_efie_far(int32_t nv, const double *V, int32_t nt, const int32_t *T, int32_t nb, const int32_t *tri,
                const int32_t *free_v, double k, double eta0, double r_abs, double c_rel, int32_t nblk,
                const int64_t *rptr, const int32_t *ridx, const int64_t *cptr, const int32_t *cidx, double eps,
                int32_t *rank, int64_t *uoff, int64_t *voff, int64_t cap_u, hm_c128 *U, int64_t cap_v, hm_c128 *Vf,
                int64_t *need, int64_t scratch_bytes, int32_t device);

#ifdef __cplusplus
}
#endif
#endif
