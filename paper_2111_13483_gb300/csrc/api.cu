// C-ABI entry points of hmsolve (declared in include/hmsolve.h).  Argument checks, device
// uploads, error mapping; the arithmetic is in setup.cu and solve.cu.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "hm_internal.h"

namespace hm {

cudaError_t Arena::alloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    if (budget && used + bytes > budget) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        used += bytes;
        ptrs.push_back(*p);
        sizes.push_back(bytes);
    } else
        cudaGetLastError();
    return e;
}

void Arena::release(void *p, size_t)
{
    if (!p) return;
    for (size_t i = 0; i < ptrs.size(); ++i)
        if (ptrs[i] == p) {
            cudaFree(p);
            used -= sizes[i];
            ptrs.erase(ptrs.begin() + i);
            sizes.erase(sizes.begin() + i);
            return;
        }
}

void Arena::release_all()
{
    for (void *p : ptrs) cudaFree(p);
    ptrs.clear();
    sizes.clear();
    used = 0;
}

void Prof::begin(cudaStream_t st)
{
    if (!on) return;
    if (pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        pool.push_back(e);
    }
    cur_start = pool.back();
    pool.pop_back();
    cudaEventRecord(cur_start, st);
}

void Prof::end(cudaStream_t st, int cls)
{
    count[cls]++;
    if (!on || !cur_start) return;
    cudaEvent_t e1;
    if (pool.empty()) cudaEventCreate(&e1);
    else {
        e1 = pool.back();
        pool.pop_back();
    }
    cudaEventRecord(e1, st);
    pending.push_back({cls, {cur_start, e1}});
    cur_start = nullptr;
    if (pending.size() > 4096) flush();
}

void Prof::flush()
{
    for (auto &p : pending) {
        cudaEventSynchronize(p.second.second);
        float ms = 0;
        cudaEventElapsedTime(&ms, p.second.first, p.second.second);
        this->ms[p.first] += ms;
        timed[p.first]++;
        pool.push_back(p.second.first);
        pool.push_back(p.second.second);
    }
    pending.clear();
}

void Prof::reset()
{
    flush();
    for (int c = 0; c < K_NCLASS; ++c) count[c] = 0, ms[c] = 0, timed[c] = 0, cols[c] = 0;
}

void Prof::destroy()
{
    flush();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
}

template <class T>
static cudaError_t upload(hm_ctx *h, T **dst, const T *src, size_t count)
{
    cudaError_t e = h->arena.alloc((void **)dst, sizeof(T) * (count ? count : 1));
    if (e) return e;
    if (count) e = cudaMemcpyAsync(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, h->stream);
    return e;
}

template <class T>
static cudaError_t upload(hm_ctx *h, T **dst, const std::vector<T> &v)
{
    return upload(h, dst, v.data(), v.size());
}

static int cuda_fail(hm_ctx *h, cudaError_t e, const char *where)
{
    h->err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA;
}

}  // namespace hm

using namespace hm;

extern "C" {

int hm_default_opts(hm_opts *o)
{
    if (!o) return HM_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->ordering = 1;
    o->fill_tol = 0.0;
    o->precision = 0;
    o->device = 0;
    o->hbm_budget = 0;
    o->stream = nullptr;
    return HM_OK;
}

int hmat_create(const hm_desc *d, const hm_opts *opts, hm_handle *out)
{
    if (!out) return HM_EINVAL;
    *out = nullptr;
    hm_ctx *h = new (std::nothrow) hm_ctx();
    if (!h) return HM_ENOMEM;
    if (opts) h->opts = *opts;
    else hm_default_opts(&h->opts);
    int st;
    if (h->opts.ordering < 0 || h->opts.ordering > 2 || h->opts.fill_tol < 0 || h->opts.precision < 0 ||
        h->opts.precision > 1 || h->opts.preconditioner < 0 || h->opts.preconditioner > 2 ||
        h->opts.compress_in_setup < 0 || h->opts.compress_in_setup > 1 ||
        (h->opts.preconditioner != 0 && h->opts.precision != 0)) {
        delete h;
        return HM_EINVAL;
    }
    if ((st = validate_and_copy(h, d)) != HM_OK) {
        // keep the message reachable: a failed create returns no handle, so print it
        std::fprintf(stderr, "hmat_create: %s\n", h->err.c_str());
        delete h;
        return st;
    }
    cudaError_t e;
    int ndev = 0;
    if ((e = cudaGetDeviceCount(&ndev)) || h->opts.device < 0 || h->opts.device >= ndev) {
        std::fprintf(stderr, "hmat_create: no CUDA device %d\n", h->opts.device);
        cudaGetLastError();
        delete h;
        return HM_ECUDA;
    }
    h->dev = h->opts.device;
    cudaSetDevice(h->dev);
    h->arena.budget = h->opts.hbm_budget;
    if (h->opts.stream)
        h->stream = (cudaStream_t)h->opts.stream;
    else {
        if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking))) {
            delete h;
            return HM_ECUDA;
        }
        h->own_stream = true;
    }
    plan_order(h);
    plan_far(h);
    Plan &P = h->plan;
    FarPlan &F = h->fplan;
    if ((e = upload(h, &h->d_near, (const double2 *)d->near_data, (size_t)d->near_len)) ||
        (e = upload(h, &h->d_farU, (const double2 *)d->far_U, (size_t)d->far_U_len)) ||
        (e = upload(h, &h->d_farV, (const double2 *)d->far_V, (size_t)(d->far_V ? d->far_V_len : 0))) ||
        (e = upload(h, &h->d_near_t, h->near_t)) || (e = upload(h, &h->d_near_s, h->near_s)) ||
        (e = upload(h, &h->d_near_off, h->near_off)) || (e = upload(h, &h->d_far_r0, h->far_r0)) ||
        (e = upload(h, &h->d_far_r1, h->far_r1)) || (e = upload(h, &h->d_far_c0, h->far_c0)) ||
        (e = upload(h, &h->d_far_c1, h->far_c1)) || (e = upload(h, &h->d_far_rank, h->far_rank)) ||
        (e = upload(h, &h->d_far_uoff, h->far_uoff)) || (e = upload(h, &h->d_far_voff, h->far_voff)) ||
        (e = upload(h, &h->d_far_toff, F.toff)) || (e = upload(h, &h->d_far_item, F.item_blk)) ||
        (e = upload(h, &h->d_p1_lo, F.p1_lo)) || (e = upload(h, &h->d_p1_hi, F.p1_hi)) ||
        (e = upload(h, &h->d_p1_ptr, F.p1_ptr)) || (e = upload(h, &h->d_p1_off, F.p1_off)) ||
        (e = upload(h, &h->d_p1_ld, F.p1_ld)) || (e = upload(h, &h->d_p1_rank, F.p1_rank)) ||
        (e = upload(h, &h->d_p1_row, F.p1_row)) || (e = upload(h, &h->d_p1_isv, F.p1_isv)) ||
        (e = upload(h, &h->d_seg_ptr, F.seg_ptr)) || (e = upload(h, &h->d_segs, F.segs)) ||
        (e = upload(h, &h->d_seg_kcum, F.seg_kcum)) || (e = upload(h, &h->d_part_ptr, F.part_ptr)) ||
        (e = upload(h, &h->d_flptr, F.lptr)) ||
        (e = upload(h, &h->d_flent, F.lent)) || (e = upload(h, &h->d_nptr, F.nptr)) ||
        (e = upload(h, &h->d_nent, F.nent)) || (e = upload(h, &h->d_leaf_ptr, h->leaf_ptr)) ||
        (e = upload(h, &h->d_new2cl, P.new2cl)) || (e = upload(h, &h->d_cl2new, P.cl2new)) ||
        (e = upload(h, &h->d_new2orig, P.new2orig)) || (e = upload(h, &h->d_perm, h->perm)) ||
        (e = upload(h, &h->d_pos, P.pos)) || (e = upload(h, &h->d_size, P.size)) ||
        (e = upload(h, &h->d_boff, P.boff)) || (e = upload(h, &h->d_sptr, P.sptr)) ||
        (e = upload(h, &h->d_sidx, P.sidx)) || (e = upload(h, &h->d_srow, P.srow)) ||
        (e = upload(h, &h->d_M, P.M)) || (e = upload(h, &h->d_coff, P.coff)) || (e = upload(h, &h->d_doff, P.doff)) ||
        (e = upload(h, &h->d_rptr, P.rptr)) || (e = upload(h, &h->d_ridx, P.ridx)) ||
        (e = upload(h, &h->d_rcol, P.rcol)) || (e = upload(h, &h->d_fill_e, P.fill_e)) ||
        (e = upload(h, &h->d_xptr[0], P.xptr[0])) || (e = upload(h, &h->d_xdep[0], P.xdep[0])) ||
        (e = upload(h, &h->d_xoff[0], P.xoff[0])) || (e = upload(h, &h->d_xint[0], P.xint[0])) ||
        (e = upload(h, &h->d_xptr[1], P.xptr[1])) || (e = upload(h, &h->d_xdep[1], P.xdep[1])) ||
        (e = upload(h, &h->d_xoff[1], P.xoff[1])) || (e = upload(h, &h->d_xint[1], P.xint[1])) ||
        (e = upload(h, &h->d_rec[0], P.rec[0])) || (e = upload(h, &h->d_reccol[0], P.reccol[0])) ||
        (e = upload(h, &h->d_rec[1], P.rec[1])) || (e = upload(h, &h->d_reccol[1], P.reccol[1])) ||
        (e = upload(h, &h->d_fill_k, P.fill_k)) || (e = upload(h, &h->d_rent, P.rent)) ||
        (e = upload(h, &h->d_pboff, P.pboff)) || (e = upload(h, &h->d_cboff, P.pboff)) ||
        (e = h->arena.alloc((void **)&h->d_crank, sizeof(int) * std::max<size_t>(P.sidx.size(), 1))) ||
        (e = cudaMemsetAsync(h->d_crank, 0xff, sizeof(int) * std::max<size_t>(P.sidx.size(), 1), h->stream))) {
        int s = cuda_fail(h, e, "hmat_create upload");
        std::fprintf(stderr, "hmat_create: %s\n", h->err.c_str());
        h->arena.release_all();
        if (h->own_stream) cudaStreamDestroy(h->stream);
        delete h;
        return s;
    }
    int err_init[ERR_WORDS] = {0, -1, 0, 0};
    std::memcpy(err_init + ERR_BOUND, &WAIT_NS_DEFAULT, sizeof(WAIT_NS_DEFAULT));
    if ((e = h->arena.alloc((void **)&h->d_err, sizeof(int) * ERR_WORDS)) ||
        (e = h->arena.alloc((void **)&h->d_ticket, sizeof(int))) ||
        (e = cudaMemcpy(h->d_err, err_init, sizeof(err_init), cudaMemcpyHostToDevice)) ||
        (h->opts.precision == 1 && (e = make_fp32_copies(h))) || (e = cudaStreamSynchronize(h->stream))) {
        int s = cuda_fail(h, e, "hmat_create");
        h->arena.release_all();
        if (h->own_stream) cudaStreamDestroy(h->stream);
        delete h;
        return s;
    }
    *out = h;
    return HM_OK;
}

int precond_setup(hm_handle h)
{
    if (!h) return HM_EINVAL;
    cudaSetDevice(h->dev);
    h->setup_done = false;
    Plan &P = h->plan;
    cudaError_t e;
    const bool mixed = h->opts.precision == 1;
    if (h->opts.preconditioner == 1) {   // block Jacobi: D_k = Z_kk and its inverse only
        if (!h->d_Dinv && ((e = h->arena.alloc((void **)&h->d_Dinv, sizeof(double2) * P.diag_entries)) ||
                           (e = h->arena.alloc((void **)&h->d_Ad, sizeof(double2) * P.diag_entries))))
            return cuda_fail(h, e, "precond_setup allocation");
        cudaEvent_t b0, b1;
        cudaEventCreate(&b0);
        cudaEventCreate(&b1);
        cudaEventRecord(b0, h->stream);
        int bad = -1;
        e = block_jacobi_setup(h, &bad);
        cudaEventRecord(b1, h->stream);
        cudaEventSynchronize(b1);
        float ms = 0;
        cudaEventElapsedTime(&ms, b0, b1);
        cudaEventDestroy(b0);
        cudaEventDestroy(b1);
        if (e) return cuda_fail(h, e, "precond_setup");
        if (bad >= 0) {
            h->err = "diagonal block " + std::to_string(bad) + " (solve order; leaf " + std::to_string(P.order[bad]) +
                     ") is numerically singular";
            return HM_ESINGULAR;
        }
        h->setup_ms = ms;
        h->setup_done = true;
        return HM_OK;
    }
    if (!h->d_Dinv) {   // factors: FP64, or FP32 (with D_k^{-1} in both) for the mixed setup
        if ((e = h->arena.alloc((void **)&h->d_Dinv, sizeof(double2) * P.diag_entries)) ||
            (mixed ? ((e = h->arena.alloc((void **)&h->d_W32, sizeof(float2) * P.coef_entries)) ||
                      (e = h->arena.alloc((void **)&h->d_Ad32, sizeof(float2) * P.diag_entries)) ||
                      (e = h->arena.alloc((void **)&h->d_Dinv32, sizeof(float2) * P.diag_entries)))
                   : ((e = h->arena.alloc((void **)&h->d_W, sizeof(double2) * P.coef_entries)) ||
                      (e = h->arena.alloc((void **)&h->d_Ad, sizeof(double2) * P.diag_entries)))))
            return cuda_fail(h, e, "precond_setup allocation");
    }
    if ((e = mixed ? h->arena.alloc((void **)&h->d_A32, sizeof(float2) * P.coef_entries)
                   : h->arena.alloc((void **)&h->d_A, sizeof(double2) * P.coef_entries)))
        return cuda_fail(h, e, "precond_setup workspace");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, h->stream);
    int bad = -1;
    e = setup_run(h, &bad);
    if (!e && bad < 0) e = compress_run(h);
    if (!e && bad < 0) e = pack_run(h);
    cudaEventRecord(e1, h->stream);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->arena.release(h->d_A, 0);
    h->arena.release(h->d_A32, 0);
    h->d_A = nullptr;
    h->d_A32 = nullptr;
    if (e) return cuda_fail(h, e, "precond_setup");
    if (bad >= 0) {
        h->err = "pivot block D_" + std::to_string(bad) + " (solve order; leaf " + std::to_string(P.order[bad]) +
                 ") is numerically singular";
        return HM_ESINGULAR;
    }
    h->setup_ms = ms;
    h->setup_done = true;
    return HM_OK;
}

int solve_device(hm_handle h, const void *dV, int32_t nrhs, int64_t ldv, double tol, int32_t restart, int32_t maxit,
                 void *dI, int64_t ldi, int32_t *iters, double *relres)
{
    if (!h) return HM_EINVAL;
    if (!h->setup_done) {
        h->err = "solve before precond_setup";
        return HM_ESTATE;
    }
    if (nrhs < 0 || (nrhs > 0 && (!dV || !dI || !iters || !relres)) || ldv < h->n || ldi < h->n || restart < 1 ||
        maxit < 0 || !(tol >= 0)) {
        h->err = "solve: bad arguments";
        return HM_EINVAL;
    }
    if (nrhs == 0) return HM_OK;
    cudaSetDevice(h->dev);
    return gmres_solve(h, (const double2 *)dV, nrhs, ldv, tol, restart, maxit, (double2 *)dI, ldi, iters, relres);
}

int solve(hm_handle h, const hm_c128 *V, int32_t nrhs, int64_t ldv, double tol, int32_t restart, int32_t maxit,
          hm_c128 *I, int64_t ldi, int32_t *iters, double *relres)
{
    if (!h) return HM_EINVAL;
    if (!h->setup_done) {
        h->err = "solve before precond_setup";
        return HM_ESTATE;
    }
    if (nrhs < 0 || (nrhs > 0 && (!V || !I || !iters || !relres)) || ldv < h->n || ldi < h->n) {
        h->err = "solve: bad arguments";
        return HM_EINVAL;
    }
    if (nrhs == 0) return HM_OK;
    cudaSetDevice(h->dev);
    double2 *dV = nullptr, *dI = nullptr;
    cudaError_t e;
    const size_t col = sizeof(double2) * (size_t)h->n;
    if ((e = h->arena.alloc((void **)&dV, col * nrhs)) || (e = h->arena.alloc((void **)&dI, col * nrhs))) {
        h->arena.release(dV, 0);
        return cuda_fail(h, e, "solve staging");
    }
    int s = HM_OK;
    if ((e = cudaMemcpy2DAsync(dV, col, V, sizeof(hm_c128) * ldv, col, nrhs, cudaMemcpyHostToDevice, h->stream)))
        s = cuda_fail(h, e, "solve upload");
    if (s == HM_OK) s = solve_device(h, dV, nrhs, h->n, tol, restart, maxit, dI, h->n, iters, relres);
    if (s == HM_OK || s == HM_ENOCONV) {
        if ((e = cudaMemcpy2DAsync(I, sizeof(hm_c128) * ldi, dI, col, col, nrhs, cudaMemcpyDeviceToHost, h->stream)) ||
            (e = cudaStreamSynchronize(h->stream)))
            s = cuda_fail(h, e, "solve download");
    }
    h->arena.release(dV, 0);
    h->arena.release(dI, 0);
    return s;
}

int hmat_stats(hm_handle h, hm_stats *s)
{
    if (!h || !s) return HM_EINVAL;
    std::memset(s, 0, sizeof(*s));
    const Plan &P = h->plan;
    s->n = h->n;
    s->n_blocks = P.nb;
    int64_t ne = 0;
    for (size_t b = 0; b < h->near_t.size(); ++b) {
        int t = h->near_t[b], u = h->near_s[b];
        ne += (int64_t)(h->leaf_ptr[t + 1] - h->leaf_ptr[t]) * (h->leaf_ptr[u + 1] - h->leaf_ptr[u]);
    }
    s->near_entries = ne;
    s->far_entries = h->fplan.entries;
    s->fill_blocks = P.sptr.empty() ? 0 : P.sptr[P.nb];
    s->coef_entries = h->lowrank ? h->wc_len : P.coef_entries;   // what the sweeps read
    s->coef_entries_dense = P.coef_entries;
    s->diag_entries = P.diag_entries;
    s->bandwidth = P.bandwidth;
    s->setup_ms = h->setup_ms;
    s->setup_gflop = P.setup_flops * 1e-9;
    s->device_bytes = h->arena.used;
    return HM_OK;
}

const char *hm_last_error(hm_handle h)
{
    if (!h) return "null handle";
    return h->err.c_str();
}

void hmat_destroy(hm_handle h)
{
    if (!h) return;
    cudaSetDevice(h->dev);
    cudaStreamSynchronize(h->stream);
    h->prof.destroy();
    sweep_tune_release(h);
    h->arena.release_all();
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

int hm_get_order(hm_handle h, int32_t *order)
{
    if (!h || !order) return HM_EINVAL;
    std::memcpy(order, h->plan.order.data(), sizeof(int32_t) * h->plan.nb);
    return HM_OK;
}

int hm_get_index_map(hm_handle h, int32_t *new2orig)
{
    if (!h || !new2orig) return HM_EINVAL;
    std::memcpy(new2orig, h->plan.new2orig.data(), sizeof(int32_t) * h->n);
    return HM_OK;
}

int hm_get_fill(hm_handle h, int32_t *ptr, int32_t *idx)
{
    if (!h || !ptr) return HM_EINVAL;
    std::memcpy(ptr, h->plan.sptr.data(), sizeof(int32_t) * (h->plan.nb + 1));
    if (idx) std::memcpy(idx, h->plan.sidx.data(), sizeof(int32_t) * h->plan.sidx.size());
    return HM_OK;
}

int hm_get_fill_ranks(hm_handle h, int32_t *rank)
{
    if (!h || !rank) return HM_EINVAL;
    const Plan &P = h->plan;
    const int ne = P.sptr.empty() ? 0 : P.sptr[P.nb];
    for (int e = 0; e < ne; ++e) rank[e] = -1;
    for (size_t f = 0; f < h->fill_ranks.size() && f < P.fill_e.size(); ++f) rank[P.fill_e[f]] = h->fill_ranks[f];
    return HM_OK;
}

int hm_get_block(hm_handle h, int32_t what, int32_t k, hm_c128 *out)
{
    if (!h || !out) return HM_EINVAL;
    if (!h->setup_done) {
        h->err = "hm_get_block before precond_setup";
        return HM_ESTATE;
    }
    const Plan &P = h->plan;
    if (k < 0 || k >= P.nb || what < 0 || what > 3) return HM_EINVAL;
    if (h->opts.preconditioner == 1 && what >= 2) {
        h->err = "hm_get_block: the block-Jacobi preconditioner has no coefficient blocks";
        return HM_ESTATE;
    }
    cudaSetDevice(h->dev);
    const bool mixed = h->opts.precision == 1;
    const void *src;
    size_t cnt;
    bool f32 = false;
    int64_t nk = P.size[k];
    if (what == 0) {
        src = mixed ? (const void *)(h->d_Ad32 + P.doff[k]) : (const void *)(h->d_Ad + P.doff[k]);
        f32 = mixed;
        cnt = nk * nk;
    } else if (what == 1) {
        src = h->d_Dinv + P.doff[k];
        cnt = nk * nk;
    } else if (h->lowrank) {   // the row's blocks from the compact store, factors expanded
        const int64_t a = h->cboff[P.sptr[k]], b = h->cboff[P.sptr[k + 1]];
        std::vector<hm_c128> st(b - a);
        cudaError_t e;
        if (mixed) {
            std::vector<float2> tmp(b - a);
            if ((e = cudaMemcpyAsync(tmp.data(), h->d_Wc32 + a, sizeof(float2) * (b - a), cudaMemcpyDeviceToHost,
                                     h->stream)) ||
                (e = cudaStreamSynchronize(h->stream)))
                return cuda_fail(h, e, "hm_get_block");
            for (size_t i = 0; i < tmp.size(); ++i) st[i] = hm_c128{(double)tmp[i].x, (double)tmp[i].y};
        } else if ((e = cudaMemcpyAsync(st.data(), h->d_Wc + a, sizeof(double2) * (b - a), cudaMemcpyDeviceToHost,
                                        h->stream)) ||
                   (e = cudaStreamSynchronize(h->stream)))
            return cuda_fail(h, e, "hm_get_block");
        for (int x = P.sptr[k]; x < P.sptr[k + 1]; ++x) {
            const int64_t nj = P.size[P.sidx[x]], r = h->crank[x];
            const hm_c128 *blk = st.data() + (h->cboff[x] - a);
            hm_c128 *dst = out + (int64_t)P.srow[x] * nk;   // the panel's columns of block x
            for (int64_t c = 0; c < nj; ++c)
                for (int64_t q = 0; q < nk; ++q) {
                    if (r < 0) {
                        dst[q + c * nk] = blk[q + c * nk];
                        continue;
                    }
                    double re = 0, im = 0;   // sum_l P(q, l) Q(c, l)
                    for (int64_t l = 0; l < r; ++l) {
                        const hm_c128 p = blk[q + l * nk], w = blk[nk * r + c + l * nj];
                        re += p.re * w.re - p.im * w.im;
                        im += p.re * w.im + p.im * w.re;
                    }
                    dst[q + c * nk] = hm_c128{re, im};
                }
        }
        return HM_OK;
    } else {
        src = mixed ? (const void *)(h->d_W32 + P.coff[k]) : (const void *)(h->d_W + P.coff[k]);
        f32 = mixed;
        cnt = (size_t)nk * P.M[k];
    }
    cudaError_t e;
    if (!f32) {
        if ((e = cudaMemcpyAsync(out, src, sizeof(double2) * cnt, cudaMemcpyDeviceToHost, h->stream)) ||
            (e = cudaStreamSynchronize(h->stream)))
            return cuda_fail(h, e, "hm_get_block");
        return HM_OK;
    }
    std::vector<float2> tmp(cnt);   // FP32 factors of the mixed setup, widened on the host
    if ((e = cudaMemcpyAsync(tmp.data(), src, sizeof(float2) * cnt, cudaMemcpyDeviceToHost, h->stream)) ||
        (e = cudaStreamSynchronize(h->stream)))
        return cuda_fail(h, e, "hm_get_block");
    for (size_t i = 0; i < cnt; ++i) out[i] = hm_c128{(double)tmp[i].x, (double)tmp[i].y};
    return HM_OK;
}

int hm_set_sweep_schedule(hm_handle h, int32_t groups, int32_t kind, int32_t tile)
{
    if (!h) return HM_EINVAL;
    if (groups == 0 && kind == 0) {
        h->sweep_fixed = 0;
        return HM_OK;
    }
    if ((groups != 1 && groups != 2 && groups != 4) || kind < 1 || kind > 6 || tile < 0 || tile > 2)
        return HM_EINVAL;
    h->sweep_fixed = groups | (kind << 4) | (tile << 8);
    return HM_OK;
}

int hm_test_hold(hm_handle h, int32_t block, int64_t wait_ns)
{
    if (!h || block < -1 || block >= h->plan.nb || wait_ns < 0) return HM_EINVAL;
    cudaSetDevice(h->dev);
    int w[ERR_WORDS] = {0, block, 0, 0};
    const unsigned long long ns = wait_ns ? (unsigned long long)wait_ns : WAIT_NS_DEFAULT;
    std::memcpy(w + ERR_BOUND, &ns, sizeof(ns));
    cudaError_t e;
    // the stream first: no kernel of this handle may be reading the words while they change
    if ((e = cudaStreamSynchronize(h->stream)) ||
        (e = cudaMemcpy(h->d_err + ERR_HOLD, w + ERR_HOLD, sizeof(int) * (ERR_WORDS - ERR_HOLD),
                        cudaMemcpyHostToDevice)))
        return cuda_fail(h, e, "hm_test_hold");
    return HM_OK;
}

int hm_set_far_schedule(hm_handle h, int32_t kind)
{
    if (!h || kind < 0 || kind > 2) return HM_EINVAL;
    h->far_kind = kind == 0 ? 1 : kind;
    return HM_OK;
}

int hm_set_update_schedule(hm_handle h, int32_t kind)
{
    if (!h || kind < 0 || kind > 2) return HM_EINVAL;
    h->update_kind = kind == 0 ? 1 : kind;
    return HM_OK;
}

int hm_set_pivot_schedule(hm_handle h, int32_t ctas)
{
    if (!h || !(ctas == 0 || ctas == 1 || ctas == 2 || ctas == 4 || ctas == 8)) return HM_EINVAL;
    h->pivot_cl = ctas == 0 ? 8 : ctas;
    return HM_OK;
}

int hm_profile(hm_handle h, int32_t mode)
{
    if (!h || mode < 0 || mode > 2) return HM_EINVAL;
    cudaSetDevice(h->dev);
    if (mode == 2) h->prof.reset();
    else {
        h->prof.flush();
        h->prof.on = mode == 1;
    }
    return HM_OK;
}

int hm_get_profile(hm_handle h, int32_t cls, int64_t *launches, int64_t *timed, double *ms)
{
    if (!h || cls < 0 || cls >= K_NCLASS) return HM_EINVAL;
    cudaSetDevice(h->dev);
    h->prof.flush();
    if (launches) *launches = h->prof.count[cls];
    if (timed) *timed = h->prof.timed[cls];
    if (ms) *ms = h->prof.ms[cls];
    return HM_OK;
}

int hm_get_profile_cols(hm_handle h, int32_t cls, int64_t *cols)
{
    if (!h || !cols || cls < 0 || cls >= K_NCLASS) return HM_EINVAL;
    *cols = h->prof.cols[cls];
    return HM_OK;
}

int hm_apply(hm_handle h, int32_t op, const void *dx, void *dy, int32_t nrhs)
{
    if (!h || !dx || !dy || nrhs < 1 || op < 0 || op > 12 || (op > 5 && op < 8)) return HM_EINVAL;
    if (op != 3 && op != 5 && !h->setup_done) {
        h->err = "hm_apply: operator needs precond_setup";
        return HM_ESTATE;
    }
    if (op >= 8 && h->opts.precision != 1) {
        h->err = "hm_apply: the complex-FP32 operators exist for precision 1 handles only";
        return HM_ESTATE;
    }
    if (h->opts.precision == 1 && (op <= 2 || op == 4)) {
        h->err = "hm_apply: a precision 1 handle keeps complex-FP32 factors (ops 8-12)";
        return HM_ESTATE;
    }
    cudaSetDevice(h->dev);
    cudaError_t e;
    if (op == 5) e = hm::z_apply_orig(h, (const double2 *)dx, (double2 *)dy, nrhs);
    else if (op >= 8) e = hm::op_apply32(h, op - 8, (const double2 *)dx, (double2 *)dy, nrhs);
    else e = op_apply(h, op, (const double2 *)dx, (double2 *)dy, nrhs);
    if (!e) e = cudaStreamSynchronize(h->stream);
    if (e) return cuda_fail(h, e, "hm_apply");
    int herr = 0;
    cudaMemcpy(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (herr) {
        h->err = "device-side wait timed out";
        cudaMemset(h->d_err, 0, sizeof(int));
        return HM_ETIMEOUT;
    }
    return HM_OK;
}

}  // extern "C"
