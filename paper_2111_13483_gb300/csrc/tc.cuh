// Complex-FP32 block products on the fifth-generation tensor cores (tcgen05, kind::tf32),
// shared by the complex-FP32 triangular sweeps (ops.cu) and the product entry point of
// tcprod.cu.
//
// Product.  One output block C (m x c complex, m <= 64 rows, c <= 64 columns) accumulates
// sum_q M(row, q) Y(q, col) over a contraction walked in chunks of at most KC.  The complex
// product is one real MMA per k-step: with m8 = m rounded up to 8 and p = c rounded up to 8,
//   A' (128 x K) = [Re M ; Im M]   (rows 0..m8-1 real parts, m8..2 m8-1 imaginary parts),
//   B' (2p x K)  = [Re Y^T ; Im Y^T] (rows 0..p-1 real, p..2p-1 imaginary: B' row = output col),
//   D = A' B'^T  (128 x 2p, FP32, in tensor memory),
// and at the end Re C = D[r][j] - D[m8 + r][p + j], Im C = D[r][p + j] + D[m8 + r][j].
// Rows 2 m8..127 of A' are whatever the shared memory holds there; they only reach rows of D
// that are never read.  Contraction padding (up to a multiple of 8) is zero in both operands.
//
// Precision: every FP32 operand x is split as hi = tf32(x) (round to nearest), lo = tf32(x - hi),
// and each k-step issues lo*hi + hi*lo + hi*hi into the FP32 accumulator (the 3xTF32 scheme of
// Ootomo and Yokota, "Recovering single precision accuracy from Tensor Cores while surpassing
// the FP32 theoretical peak performance", IJHPCA 2022): about FP32 accuracy.  The accumulation
// order is fixed (chunks in walk order, k-steps ascending, the three products in that order), and
// each output column depends only on its own B' rows, so a column's result does not depend on how
// many other columns share the launch.
//
// Shared-memory operands use the K-major, no-swizzle canonical layout: core matrices of 8 rows x
// 16 bytes (4 TF32 values), the core matrices of one 4-wide K group stored consecutively for all
// row groups (stride 128 B), K groups after one another (stride rows * 16 B).  Descriptors: start
// address, leading byte offset = the K-group stride, stride byte offset = 128 B, version 1, no
// swizzle.  A' always spans 128 rows (16 KB per plane at KC = 32), B' spans 2p rows.
#pragma once

#include <cstdint>

#include "cplx.cuh"
#include "hm_internal.h"

namespace hm {
namespace tc {

constexpr int KC = 32;                         // contraction length of one staged chunk
constexpr int AROWS = 128;                     // MMA M
constexpr int A_PLANE = AROWS * KC * 4;        // bytes of one A' plane (hi or lo)
constexpr int B_PLANE = 128 * KC * 4;          // bytes of one B' plane at the widest B' (2p = 128)
constexpr int TMEM_COLS = 128;                 // accumulator columns (2p <= 128)
constexpr int PLANES_BYTES = 2 * A_PLANE + 2 * B_PLANE;   // 64 KB: A'hi, A'lo, B'hi, B'lo
// the drained accumulator (drain) takes up to 128 x 129 floats, a little more than the planes:
// kernels reserve REGION_BYTES from the planes' start
constexpr int REGION_BYTES = 128 * 130 * 4;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row, k) in a K-major canonical operand of `rows` rows (rows a multiple of 8)
__device__ __forceinline__ uint32_t kmaj(int row, int k, int rows)
{
    return (uint32_t)((k >> 2) * (rows * 16) + (row >> 3) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor (tcgen05 format): start >> 4 in bits 0-13, leading byte
// offset >> 4 in bits 16-29, stride byte offset >> 4 in bits 32-45, version 1 at bit 46,
// base offset 0, relative leading offset, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B TF32 (bits
// 7-9 and 10-12 = 2), no negation, both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// hi/lo split of x into two TF32 bit patterns
__device__ __forceinline__ void split(float x, uint32_t &hi, uint32_t &lo)
{
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// whole warp: allocate TMEM_COLS accumulator columns, address written to *dst (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t *dst)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// whole warp (the allocating one)
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *m)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(m)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *m, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}

// D[tmem] (+)= A' B'^T for one k-step of 8
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

// the mbarrier's phase completes once every MMA this thread issued before has finished
__device__ __forceinline__ void commit(uint64_t *m)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(m))
                 : "memory");
}

// whole warp: 8 consecutive accumulator columns of the warp's 32 lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ unsigned long long gtimer_tc()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The per-CTA state of one output block's accumulation.  Shared memory: planes (PLANES_BYTES,
// 1024-byte aligned), the mbarrier and the TMEM address slot.
struct Acc {
    unsigned char *planes;
    uint64_t *mbar;
    uint32_t *tslot;
    uint32_t tmem = 0;
    uint32_t parity = 0;
    bool pending = false;   // MMAs issued and not yet waited for
    bool any = false;       // the accumulator holds a product
    int m8 = 8, p = 8;

    __device__ unsigned char *ahi() const { return planes; }
    __device__ unsigned char *alo() const { return planes + A_PLANE; }
    __device__ unsigned char *bhi() const { return planes + 2 * A_PLANE; }
    __device__ unsigned char *blo() const { return planes + 2 * A_PLANE + B_PLANE; }

    // all threads; warp 0 allocates the accumulator, thread 0 initialises the mbarrier
    __device__ void open(int m, int c)
    {
        m8 = (m + 7) & ~7;
        p = (c + 7) & ~7;
        if (threadIdx.x < 32) tmem_alloc(tslot);
        if (threadIdx.x == 0) mbar_init(mbar);
        fence_before();
        __syncthreads();
        fence_after();
        tmem = *tslot;
    }

    // all threads: wait for the MMAs in flight (bounded; *err gets ERR_TIMEOUT when the bound
    // expires, which only a faulty device could cause)
    __device__ void wait(int *err, unsigned long long bound)
    {
        if (!pending) return;
        if (!mbar_try(mbar, parity)) {
            const unsigned long long t0 = gtimer_tc();
            while (!mbar_try(mbar, parity))
                if (gtimer_tc() - t0 > bound) {
                    if (err) atomicCAS(err, 0, ERR_TIMEOUT);
                    break;
                }
        }
        parity ^= 1u;
        pending = false;
        fence_after();
    }

    // A'(row, k) and A'(m8 + row, k) from one complex coefficient
    __device__ __forceinline__ void put_a(int row, int k, float2 v) const
    {
        uint32_t h, l;
        split(v.x, h, l);
        *(uint32_t *)(ahi() + kmaj(row, k, AROWS)) = h;
        *(uint32_t *)(alo() + kmaj(row, k, AROWS)) = l;
        split(v.y, h, l);
        *(uint32_t *)(ahi() + kmaj(m8 + row, k, AROWS)) = h;
        *(uint32_t *)(alo() + kmaj(m8 + row, k, AROWS)) = l;
    }

    // B'(col, k) and B'(p + col, k) from one complex vector entry Y(k, col)
    __device__ __forceinline__ void put_b(int col, int k, float2 v) const
    {
        uint32_t h, l;
        const int rows = 2 * p;
        split(v.x, h, l);
        *(uint32_t *)(bhi() + kmaj(col, k, rows)) = h;
        *(uint32_t *)(blo() + kmaj(col, k, rows)) = l;
        split(v.y, h, l);
        *(uint32_t *)(bhi() + kmaj(p + col, k, rows)) = h;
        *(uint32_t *)(blo() + kmaj(p + col, k, rows)) = l;
    }

    // zero the contraction padding [klen, klen8) of every used row of A' and B'
    __device__ void zero_pad(int klen) const
    {
        const int k8 = (klen + 7) & ~7, np = k8 - klen, ra = 2 * m8, rb = 2 * p;
        for (int e = threadIdx.x; e < np * (ra + rb); e += blockDim.x) {
            const int k = klen + e % np, r = e / np;
            if (r < ra) {
                *(uint32_t *)(ahi() + kmaj(r, k, AROWS)) = 0u;
                *(uint32_t *)(alo() + kmaj(r, k, AROWS)) = 0u;
            } else {
                *(uint32_t *)(bhi() + kmaj(r - ra, k, rb)) = 0u;
                *(uint32_t *)(blo() + kmaj(r - ra, k, rb)) = 0u;
            }
        }
    }

    // all threads, after writing the planes: make them visible to the tensor cores, then thread 0
    // issues the chunk's MMAs (klen <= KC contraction entries) and commits them to the mbarrier
    __device__ void issue(int klen)
    {
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_after();
            const int rb = 2 * p, steps = (klen + 7) >> 3;
            const uint32_t id = idesc_tf32(AROWS, rb);
            const uint32_t a0 = smem_u32(ahi()), a1 = smem_u32(alo()), b0 = smem_u32(bhi()), b1 = smem_u32(blo());
            const uint32_t alb = AROWS * 16, blb = rb * 16;   // K-group strides
            for (int s = 0; s < steps; ++s) {
                const uint32_t ao = s * 2 * alb, bo = s * 2 * blb;
                mma(tmem, sdesc(a1 + ao, alb, 128), sdesc(b0 + bo, blb, 128), id, any ? 1u : 0u);
                any = true;
                mma(tmem, sdesc(a0 + ao, alb, 128), sdesc(b1 + bo, blb, 128), id, 1u);
                mma(tmem, sdesc(a0 + ao, alb, 128), sdesc(b0 + bo, blb, 128), id, 1u);
            }
            commit(mbar);
        }
        any = any || klen > 0;
        pending = true;
    }

    // all threads, after the last wait: D -> dsm (float, row-major 2 m8 x (2p + 1)); dsm may
    // alias the planes (it needs up to REGION_BYTES).  Returns false (dsm untouched) when no product was accumulated.
    __device__ bool drain(float *dsm) const
    {
        if (!any) return false;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3;
        const int nw = blockDim.x >> 5, halves = nw >= 8 ? 2 : 1, h = warp >> 2;
        const int rb = 2 * p, ld = rb + 1, row = q * 32 + lane;
        if (q * 32 < 2 * m8 && h < halves) {   // warp-uniform
            const int c0 = h * (rb / halves), c1 = c0 + rb / halves;
            for (int c = c0; c < c1; c += 8) {
                float v[8];
                tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
                if (row < 2 * m8)
#pragma unroll
                    for (int i = 0; i < 8; ++i) dsm[row * ld + c + i] = v[i];
            }
        }
        fence_before();
        __syncthreads();
        return true;
    }

    // complex entry (row, col) of the product from the drained matrix
    __device__ __forceinline__ float2 entry(const float *dsm, int row, int col) const
    {
        const int ld = 2 * p + 1;
        return make_float2(dsm[row * ld + col] - dsm[(m8 + row) * ld + p + col],
                           dsm[row * ld + p + col] + dsm[(m8 + row) * ld + col]);
    }

    // all threads: give the accumulator back (after drain, or with no product)
    __device__ void close()
    {
        fence_before();
        __syncthreads();
        if (threadIdx.x < 32) {
            fence_after();
            tmem_dealloc(tmem);
        }
    }
};

// Two-stage variant for streamed products (the far field): the operand planes of chunk c+1 are
// written while the MMAs of chunk c still read the other stage.  Chunks of KC2 contraction
// entries; stage s at planes + s * STAGE2 (A'hi, A'lo, B'hi, B'lo, KC2 entries each), one
// mbarrier per stage.  Same operand layout, split and accumulation order as Acc, so a product
// gives the same result whatever the number of columns.
constexpr int KC2 = 16;
constexpr int A_PLANE2 = AROWS * KC2 * 4;     // 8 KB
constexpr int B_PLANE2 = 128 * KC2 * 4;       // 8 KB
constexpr int STAGE2 = 2 * A_PLANE2 + 2 * B_PLANE2;

struct Acc2 {
    unsigned char *planes;   // 2 * STAGE2 bytes, 1024-byte aligned
    uint64_t *mbar;          // 2 mbarriers
    uint32_t *tslot;
    uint32_t tmem = 0;
    uint32_t parity[2] = {0, 0};
    bool pending[2] = {false, false};
    bool any = false;
    int m8 = 8, p = 8;

    __device__ unsigned char *ahi(int s) const { return planes + s * STAGE2; }
    __device__ unsigned char *alo(int s) const { return planes + s * STAGE2 + A_PLANE2; }
    __device__ unsigned char *bhi(int s) const { return planes + s * STAGE2 + 2 * A_PLANE2; }
    __device__ unsigned char *blo(int s) const { return planes + s * STAGE2 + 2 * A_PLANE2 + B_PLANE2; }

    __device__ void open(int m, int c)
    {
        m8 = (m + 7) & ~7;
        p = (c + 7) & ~7;
        if (threadIdx.x < 32) tmem_alloc(tslot);
        if (threadIdx.x == 0) {
            mbar_init(mbar);
            mbar_init(mbar + 1);
        }
        fence_before();
        __syncthreads();
        fence_after();
        tmem = *tslot;
    }

    // all threads: stage s may be written again once its MMAs have finished
    __device__ void wait(int s, int *err, unsigned long long bound)
    {
        if (!pending[s]) return;
        if (!mbar_try(mbar + s, parity[s])) {
            const unsigned long long t0 = gtimer_tc();
            while (!mbar_try(mbar + s, parity[s]))
                if (gtimer_tc() - t0 > bound) {
                    if (err) atomicCAS(err, 0, ERR_TIMEOUT);
                    break;
                }
        }
        parity[s] ^= 1u;
        pending[s] = false;
        fence_after();
    }

    __device__ __forceinline__ void put_a(int s, int row, int k, float2 v) const
    {
        uint32_t h, l;
        split(v.x, h, l);
        *(uint32_t *)(ahi(s) + kmaj(row, k, AROWS)) = h;
        *(uint32_t *)(alo(s) + kmaj(row, k, AROWS)) = l;
        split(v.y, h, l);
        *(uint32_t *)(ahi(s) + kmaj(m8 + row, k, AROWS)) = h;
        *(uint32_t *)(alo(s) + kmaj(m8 + row, k, AROWS)) = l;
    }

    __device__ __forceinline__ void put_b(int s, int col, int k, float2 v) const
    {
        uint32_t h, l;
        const int rows = 2 * p;
        split(v.x, h, l);
        *(uint32_t *)(bhi(s) + kmaj(col, k, rows)) = h;
        *(uint32_t *)(blo(s) + kmaj(col, k, rows)) = l;
        split(v.y, h, l);
        *(uint32_t *)(bhi(s) + kmaj(p + col, k, rows)) = h;
        *(uint32_t *)(blo(s) + kmaj(p + col, k, rows)) = l;
    }

    __device__ void zero_pad(int s, int klen) const
    {
        const int k8 = (klen + 7) & ~7, np = k8 - klen, ra = 2 * m8, rb = 2 * p;
        for (int e = threadIdx.x; e < np * (ra + rb); e += blockDim.x) {
            const int k = klen + e % np, r = e / np;
            if (r < ra) {
                *(uint32_t *)(ahi(s) + kmaj(r, k, AROWS)) = 0u;
                *(uint32_t *)(alo(s) + kmaj(r, k, AROWS)) = 0u;
            } else {
                *(uint32_t *)(bhi(s) + kmaj(r - ra, k, rb)) = 0u;
                *(uint32_t *)(blo(s) + kmaj(r - ra, k, rb)) = 0u;
            }
        }
    }

    // all threads after writing stage s: thread 0 issues its MMAs, committed to mbar[s]
    __device__ void issue(int s, int klen)
    {
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0 && klen > 0) {
            fence_after();
            const int rb = 2 * p, steps = (klen + 7) >> 3;
            const uint32_t id = idesc_tf32(AROWS, rb);
            const uint32_t a0 = smem_u32(ahi(s)), a1 = smem_u32(alo(s)), b0 = smem_u32(bhi(s)), b1 = smem_u32(blo(s));
            const uint32_t alb = AROWS * 16, blb = rb * 16;
            for (int t = 0; t < steps; ++t) {
                const uint32_t ao = t * 2 * alb, bo = t * 2 * blb;
                mma(tmem, sdesc(a1 + ao, alb, 128), sdesc(b0 + bo, blb, 128), id, any ? 1u : 0u);
                any = true;
                mma(tmem, sdesc(a0 + ao, alb, 128), sdesc(b1 + bo, blb, 128), id, 1u);
                mma(tmem, sdesc(a0 + ao, alb, 128), sdesc(b0 + bo, blb, 128), id, 1u);
            }
            commit(mbar + s);
        }
        any = any || klen > 0;
        pending[s] = pending[s] || klen > 0;
    }

    __device__ bool drain(float *dsm) const
    {
        if (!any) return false;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3;
        const int nw = blockDim.x >> 5, halves = nw >= 8 ? 2 : 1, h = warp >> 2;
        const int rb = 2 * p, ld = rb + 1, row = q * 32 + lane;
        if (q * 32 < 2 * m8 && h < halves) {
            const int c0 = h * (rb / halves), c1 = c0 + rb / halves;
            for (int c = c0; c < c1; c += 8) {
                float v[8];
                tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
                if (row < 2 * m8)
#pragma unroll
                    for (int i = 0; i < 8; ++i) dsm[row * ld + c + i] = v[i];
            }
        }
        fence_before();
        __syncthreads();
        return true;
    }

    __device__ __forceinline__ float2 entry(const float *dsm, int row, int col) const
    {
        const int ld = 2 * p + 1;
        return make_float2(dsm[row * ld + col] - dsm[(m8 + row) * ld + p + col],
                           dsm[row * ld + p + col] + dsm[(m8 + row) * ld + col]);
    }

    __device__ void close()
    {
        fence_before();
        __syncthreads();
        if (threadIdx.x < 32) {
            fence_after();
            tmem_dealloc(tmem);
        }
    }
};

// shared memory a kernel using Acc needs beyond its own: the region, 1024-byte aligned
constexpr size_t SMEM_BYTES = REGION_BYTES + 1024;

__device__ __forceinline__ unsigned char *align1024(unsigned char *p)
{
    return (unsigned char *)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

}  // namespace tc
}  // namespace hm
