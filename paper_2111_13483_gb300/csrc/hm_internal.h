// Internal declarations of the hmsolve library (host planner, device kernels, C-ABI).
#pragma once
#include <atomic>

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hmsolve.h"

namespace hm {

// ---- device memory accounted against the handle's HBM budget -------------------------
struct Arena {
    size_t used = 0, budget = 0;
    std::vector<void *> ptrs;
    std::vector<size_t> sizes;
    cudaError_t alloc(void **p, size_t bytes);
    void release(void *p, size_t bytes);
    void release_all();
};

template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
};

// ---- per-kernel-class launch counts and (opt-in) CUDA-event timings ------------------
enum KClass {
    K_SCATTER = 0, K_PIVOT, K_PANEL, K_UPDATE, K_SWEEP_FWD, K_SWEEP_BWD, K_FAR1, K_FAR2, K_DIAG, K_PERMUTE,
    K_NEAR, K_DOTS, K_VEC, K_SMALL, K_COMPRESS, K_NCLASS
};

struct Prof {
    bool on = false;
    int64_t count[K_NCLASS] = {};
    double ms[K_NCLASS] = {};
    int64_t timed[K_NCLASS] = {};
    int64_t cols[K_NCLASS] = {};   // right-hand-side columns processed (sweeps, far field)
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    cudaEvent_t cur_start = nullptr;
    void begin(cudaStream_t st);
    void end(cudaStream_t st, int cls);
    void flush();          // synchronises on the pending events and accumulates ms
    void reset();
    void destroy();
};

// ---- host plan: solve order, symbolic fill, storage layout ---------------------------
constexpr int SWEEP_SR = 2;   // blocks per super-row of the sweeps
constexpr int SWEEP_T = 4;    // recent dependencies handled by the chain CTA

struct Plan {
    int nb = 0, n = 0;
    std::vector<int> order;      // block p -> leaf
    std::vector<int> pos;        // leaf -> block p
    std::vector<int> size;       // n_p
    std::vector<int> boff;       // first unknown of block p in solve order (nb+1)
    std::vector<int> new2orig;   // solve-order position -> original RWG index
    std::vector<int> new2cl;     // solve-order position -> cluster-order position
    std::vector<int> cl2new;     // cluster-order position -> solve-order position
    // S_k (sorted block positions > k) in CSR; srow[e] = row offset of block S_k[a] inside
    // the stacked column k (rows = sum over S_k of n_j), M[k] = that total.
    std::vector<int> sptr, sidx, srow, M;
    // stacked columns of the A workspace / W panels: entry offsets (same for both)
    std::vector<int64_t> coff;   // column k: M_k x n_k (A) and n_k x M_k (W panel)
    std::vector<int64_t> doff;   // diagonal block k: n_k x n_k
    int64_t coef_entries = 0, diag_entries = 0;
    // forward sweep gathers: row i <- blocks W_ki, k < i; rptr/ridx = k, rcol = column
    // offset of block i inside panel k
    std::vector<int> rptr, ridx, rcol;
    std::vector<int> rent;       // the S-list entry e of each forward gather entry (block (k, j))
    std::vector<int64_t> pboff;  // per S-list entry e: offset of block (k, S_k[e]) in the W panels
                                 // (one more entry: the panels' total)
    // fill-in blocks (Sec. 3.4): entries e of sidx whose pair (k, S_k[e]) is not a near pair
    std::vector<int> fill_e;     // entry index into sidx
    std::vector<int> fill_k;     // its block row k
    std::vector<int> fill_ptr;   // row k's fill-in blocks are fill_e[fill_ptr[k] .. fill_ptr[k+1])
    // super-rows of SWEEP_SR consecutive blocks in sweep order (index 0 forward, 1 backward):
    // xptr/xdep = the union of the members' dependency blocks outside the super-row, in the
    // order the sweep adds them; xoff[e * SWEEP_SR + s] = column of member s's coefficient
    // block in the dependency's panel (forward) or of the dependency's block in member s's
    // panel (backward), -1 if the pair has none; xint[(r * SWEEP_SR + s) * SWEEP_SR + s2] =
    // the same for member s as the dependency of member s2 (s < s2)
    std::vector<int> xptr[2], xdep[2], xoff[2], xint[2];
    // recent dependencies of each block for the chain-and-helpers sweeps (index 0 forward,
    // 1 backward): rec[d][b * SWEEP_T + j] = the j-th dependency within SWEEP_T positions of b
    // in walk order (-1 past the last), reccol the panel column as in ridx/rcol, sidx/srow
    std::vector<int> rec[2], reccol[2];
    int bandwidth = 0;
    double setup_flops = 0;
    int max_S = 0, max_M = 0;
    int64_t n_updates = 0;
};

// One contraction segment of a leaf's far-field rows (phase 2 of the far product):
// F(i, k) = Fbase[foff + i * fi + k * fk] (Fbase = U, or V when src & 1), and
// Y(k, r) = Ybase[(yrow + k) * nrhs + r] (Ybase = t, s, u for src >> 1 = 0, 1, 2), k < len.
struct FarSegD {
    int64_t foff, yrow;
    int fi, fk, len, src;
};

constexpr int FAR_PARTS = 8;

// far-field incidence lists (cluster order): per leaf l, entries (b << 2 | kind), kind
// 0 = low-rank row side, 1 = low-rank column side, 2 = dense row side, 3 = dense column side
struct FarPlan {
    int nf = 0;
    int64_t entries = 0;
    std::vector<int> lptr, lent;
    int64_t tlen = 0;                 // sum of ranks
    std::vector<int64_t> toff;        // per block: offset of its rank vectors
    std::vector<int> item_blk;        // rank item e (toff[b] <= e < toff[b+1]) -> block b
    // rank-vector tasks: factor columns contracting over one index range [p1_lo, p1_hi),
    // at most 64 per task; items p1_ptr[t]..p1_ptr[t+1]: factor V (isv) or U at p1_off with
    // column stride p1_ld, p1_rank columns, output rows p1_row.. of t (isv) or s
    std::vector<int> p1_lo, p1_hi, p1_ptr, p1_ld, p1_rank, p1_row, p1_isv;
    std::vector<int64_t> p1_off;
    // phase-2 segments per leaf: seg_ptr[l]..seg_ptr[l+1] in the order of the leaf's list
    // (len <= 32 each); seg_kcum[q] = sum of len over the segments before q
    std::vector<int> seg_ptr, seg_kcum;
    std::vector<FarSegD> segs;
    // each leaf's segments in FAR_PARTS consecutive parts of about equal contraction length:
    // part (l, p) covers segments part_ptr[l*FAR_PARTS + p] .. part_ptr[l*FAR_PARTS + p + 1]
    std::vector<int> part_ptr;
    // near-field incidence lists (cluster order) for Z_N products: per leaf l, entries
    // (b << 1 | side), side 0 = l is the row leaf t, 1 = l is the column leaf s (t != s)
    std::vector<int> nptr, nent;
};

// Online choice of the schedule of a sweep launch -- the number of independent column
// groups and the blocks per CTA (1, or a super-row of SWEEP_SR) -- per precision, direction
// and width class: candidates are timed on real calls (every candidate computes the same
// result) and the fastest per column is kept.
constexpr int SWEEP_GMAX = 4;
struct SweepTune {
    int ncand = 0, trial = 0, best = 0;   // candidate code: groups | kind << 4 | tile shape << 8
    int cand[16] = {}, width[16] = {};
    cudaEvent_t ev[32] = {};
};

}  // namespace hm

// ---- the handle -------------------------------------------------------------------------
struct hm_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    hm_opts opts{};
    std::string err;
    hm::Arena arena;
    hm::Prof prof;

    // host copies of the description (index data only)
    int n = 0, nl = 0;
    std::vector<int> perm, leaf_ptr, near_t, near_s;
    std::vector<int64_t> near_off;
    std::vector<int> far_r0, far_r1, far_c0, far_c1, far_rank;
    std::vector<int64_t> far_uoff, far_voff;
    int64_t near_len = 0, farU_len = 0, farV_len = 0;

    hm::Plan plan;
    hm::FarPlan fplan;

    // device: inputs
    double2 *d_near = nullptr, *d_farU = nullptr, *d_farV = nullptr;
    int *d_near_t = nullptr, *d_near_s = nullptr;
    int64_t *d_near_off = nullptr;
    int *d_far_r0 = nullptr, *d_far_r1 = nullptr, *d_far_c0 = nullptr, *d_far_c1 = nullptr, *d_far_rank = nullptr;
    int64_t *d_far_uoff = nullptr, *d_far_voff = nullptr, *d_far_toff = nullptr;
    int *d_flptr = nullptr, *d_flent = nullptr, *d_nptr = nullptr, *d_nent = nullptr, *d_far_item = nullptr;
    int *d_p1_lo = nullptr, *d_p1_hi = nullptr, *d_p1_ptr = nullptr, *d_p1_ld = nullptr, *d_p1_rank = nullptr,
        *d_p1_row = nullptr, *d_p1_isv = nullptr;
    int64_t *d_p1_off = nullptr;
    int *d_seg_ptr = nullptr, *d_seg_kcum = nullptr, *d_part_ptr = nullptr;
    hm::FarSegD *d_segs = nullptr;
    int *d_leaf_ptr = nullptr, *d_perm = nullptr;
    int *d_new2cl = nullptr, *d_cl2new = nullptr, *d_new2orig = nullptr, *d_pos = nullptr;
    // device: plan
    int *d_size = nullptr, *d_boff = nullptr, *d_sptr = nullptr, *d_sidx = nullptr, *d_srow = nullptr, *d_M = nullptr;
    int64_t *d_coff = nullptr, *d_doff = nullptr;
    int *d_rptr = nullptr, *d_ridx = nullptr, *d_rcol = nullptr;
    int *d_xptr[2] = {nullptr, nullptr}, *d_xdep[2] = {nullptr, nullptr}, *d_xoff[2] = {nullptr, nullptr},
        *d_xint[2] = {nullptr, nullptr}, *d_rec[2] = {nullptr, nullptr}, *d_reccol[2] = {nullptr, nullptr};
    // device: setup outputs / workspace
    double2 *d_A = nullptr;      // stacked columns workspace (scratch during setup; FP64 setup)
    float2 *d_A32 = nullptr;     // the same for the mixed-precision setup
    double2 *d_Ad = nullptr;     // diagonal blocks workspace -> D_k after setup
    double2 *d_W = nullptr;      // coefficient panels W_k (uncompressed)
    double2 *d_Dinv = nullptr;   // D_k^{-1}
    // the coefficient store the sweeps read: per S-list entry e, block (k, S_k[e]) at
    // Wc + cboff[e], dense (crank[e] = -1, n_k x n_j column-major) or, for a Sec. 3.4
    // compressed fill-in block of rank r, its factors P (n_k x r) then Q (n_j x r), W_kj ~ P Q^T.
    // Without compressed blocks Wc is the panel array itself (cboff = pboff).
    double2 *d_Wc = nullptr;
    float2 *d_Wc32 = nullptr;
    int64_t wc_len = 0;          // entries of Wc when it is its own allocation (0: it aliases W)
    bool lowrank = false;        // some block is stored as factors
    int64_t *d_cboff = nullptr, *d_pboff = nullptr;
    int *d_crank = nullptr, *d_rent = nullptr;
    std::vector<int64_t> cboff;
    std::vector<int> crank;
    bool setup_done = false;
    double setup_ms = 0;
    // fill-in compression (Sec. 3.4): block lists and the ranks of the last setup (-1 dense)
    int *d_fill_e = nullptr, *d_fill_k = nullptr, *d_fill_rank = nullptr;
    std::vector<int> fill_ranks;
    // device: solve workspace
    int *d_flags = nullptr, *d_ticket = nullptr, *d_err = nullptr;
    int epoch = 0;
    double2 *d_t = nullptr, *d_s = nullptr;  // far rank vectors (per rhs column)
    int t_cols = 0;
    double2 *d_work = nullptr;               // operator scratch vectors
    void *d_farpart = nullptr;               // far-field partial sums (FAR_PARTS x n x nrhs)
    size_t farpart_bytes = 0;
    int work_cols = 0;
    // complex-FP32 factors of the mixed-precision setup (D_k, W, D_k^{-1}; D_k^{-1} is also
    // kept in FP64 in d_Dinv) and FP32 copies of the far factors for the inner operator
    float2 *d_W32 = nullptr, *d_Ad32 = nullptr, *d_Dinv32 = nullptr, *d_farU32 = nullptr, *d_farV32 = nullptr;
    float2 *d_t32 = nullptr, *d_s32 = nullptr, *d_work32 = nullptr;
    uint4 *d_ytag = nullptr;   // tagged sweep results (complex FP32 sweeps), n x 64
    int t32_cols = 0;
    bool batch_open = false;   // an hm_batch holds this handle
    hm::SweepTune sweep_tune[2][2][5];   // [FP32][forward][width class]
    int sweep_fixed = 0;                 // a schedule code set by hm_set_sweep_schedule, 0 = tuned
    int far_kind = 1;                    // complex-FP32 far field: 1 CUDA cores, 2 tensor cores
    int update_kind = 1;                 // complex-FP32 Schur updates: 1 CUDA cores, 2 tensor cores
    int pivot_cl = 8;                    // CTAs per pivot inversion (1 = one CTA; 2, 4, 8 = a cluster)
    // fill-in compression packing (compress.cu): CTA b takes the blocks first[b] .. first[b+1]
    std::vector<int> cw_first;
    int *d_cw = nullptr;                 // first, then the block order, then the shared-memory offsets
    size_t cw_smem = 0;
    int *d_ucum = nullptr;               // per S-list entry: tensor-core update tasks of the step before it
    std::vector<int> utot;               // per step: tensor-core update tasks
};

// Launch wrapper: counts every launch by kernel class and, when profiling is on, brackets
// it with CUDA events on the handle's stream.
#define HM_LAUNCH(hp, cls, ...)                 \
    do {                                        \
        (hp)->prof.begin((hp)->stream);         \
        __VA_ARGS__;                            \
        (hp)->prof.end((hp)->stream, (cls));    \
    } while (0)

namespace hm {
constexpr int ERR_TIMEOUT = 0x40000000;   // d_err bit: a bounded device-side wait expired
// words of the handle's error block d_err (ERR_WORDS ints): the error code, the block row the
// sweeps leave out (test hook, -1 = none) and the bound on one device-side wait (uint64 ns)
constexpr int ERR_CODE = 0, ERR_HOLD = 1, ERR_BOUND = 2, ERR_WORDS = 4;
constexpr unsigned long long WAIT_NS_DEFAULT = 2000000000ull;

// A kernel's attributes (its dynamic shared-memory limit, cluster sizes) belong to one device:
// a process with handles on several GPUs must set them on each.  A call site keeps one of these
// and sets its attributes when need() says the current device has not had them yet.
struct DeviceOnce {
    std::atomic<unsigned long long> mask{0};   // device ordinals 0..63 done
    static int device()
    {
        int d = 0;
        cudaGetDevice(&d);
        return d;
    }
    bool need() const
    {
        const int d = device();
        return d < 0 || d >= 64 || !((mask.load() >> d) & 1ull);
    }
    void done()
    {
        const int d = device();
        if (d >= 0 && d < 64) mask.fetch_or(1ull << d);
    }
};

// planner.cpp
int validate_and_copy(hm_ctx *h, const hm_desc *d);
void plan_order(hm_ctx *h);
void plan_far(hm_ctx *h);
std::vector<int> rcm_order(int nl, const std::vector<int> &t, const std::vector<int> &s);
std::vector<int> sloan_order(int nl, const std::vector<int> &t, const std::vector<int> &s);
void symbolic_fill(int nl, const std::vector<int> &pi, const std::vector<int> &pj, std::vector<int> &sptr,
                   std::vector<int> &sidx, bool closure = true);

// kernels (setup.cu / solve.cu): return cudaError_t of the launches
cudaError_t setup_run(hm_ctx *h, int *bad_block);
cudaError_t block_jacobi_setup(hm_ctx *h, int *bad_block);
cudaError_t compress_run(hm_ctx *h);
cudaError_t pack_run(hm_ctx *h);
template <class TC> cudaError_t compress_step(hm_ctx *h, int k, TC *W);
cudaError_t op_apply(hm_ctx *h, int op, const double2 *x, double2 *y, int nrhs);
cudaError_t op_apply32(hm_ctx *h, int op, const double2 *x, double2 *y, int nrhs);
cudaError_t make_fp32_copies(hm_ctx *h);
cudaError_t to_solve_order(hm_ctx *h, const double2 *src, int64_t lds, double2 *dst, int nrhs);
cudaError_t to_orig_order(hm_ctx *h, const double2 *src, double2 *dst, int64_t ldd, int nrhs);
cudaError_t z_apply_orig(hm_ctx *h, const double2 *x, double2 *y, int nrhs);
template <class T>
cudaError_t far_product(hm_ctx *h, const T *U, const T *V, T *t, T *s, const T *ucl, T *y, int nrhs);
cudaError_t ensure_solve_workspace(hm_ctx *h, int nrhs);
void sweep_tune_release(hm_ctx *h);
int gmres_solve(hm_ctx *h, const double2 *dV, int nrhs, int64_t ldv, double tol, int restart, int maxit,
                double2 *dI, int64_t ldi, int *iters, double *relres);
}  // namespace hm
