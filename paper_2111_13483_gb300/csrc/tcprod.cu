// hm_tc_cgemm: one complex-FP32 block product C = A B computed by the tensor-core
// micro-kernel of the complex-FP32 sweeps (tc.cuh: tcgen05 MMAs on TF32 operands with the
// 3xTF32 split, FP32 accumulation in tensor memory), exposed so that the micro-kernel can be
// checked on its own against a plain product.
#include <cstdio>

#include "hm_internal.h"
#include "tc.cuh"

namespace hm {
namespace {

__device__ int g_tc_err;   // ERR_TIMEOUT when a bounded wait of the last call expired

constexpr unsigned long long TC_WAIT_NS = 1000000000ull;

// One CTA: C (m x nc) = A (m x kdim) B (kdim x nc), column-major; chunks of KC contraction
// entries staged into the operand planes, one MMA batch per chunk.
__global__ void __launch_bounds__(256) k_tc_cgemm(int m, int kdim, int nc, const float2 *A, int64_t lda,
                                                  const float2 *B, int64_t ldb, float2 *C, int64_t ldc)
{
    extern __shared__ unsigned char tc_sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tslot;
    tc::Acc acc;
    acc.planes = tc::align1024(tc_sm);
    acc.mbar = &mbar;
    acc.tslot = &tslot;
    acc.open(m, nc);
    const int m8 = acc.m8, p = acc.p;
    for (int k0 = 0; k0 < kdim; k0 += tc::KC) {
        const int kl = min(tc::KC, kdim - k0);
        acc.wait(&g_tc_err, TC_WAIT_NS);   // the planes are free once the last chunk's MMAs finished
        for (int e = threadIdx.x; e < m8 * kl; e += blockDim.x) {
            const int row = e % m8, kk = e / m8;
            acc.put_a(row, kk, row < m ? A[row + (int64_t)(k0 + kk) * lda] : make_float2(0.f, 0.f));
        }
        for (int e = threadIdx.x; e < p * kl; e += blockDim.x) {
            const int kk = e % kl, col = e / kl;
            acc.put_b(col, kk, col < nc ? B[(k0 + kk) + (int64_t)col * ldb] : make_float2(0.f, 0.f));
        }
        acc.zero_pad(kl);
        acc.issue(kl);
    }
    acc.wait(&g_tc_err, TC_WAIT_NS);
    float *dsm = (float *)acc.planes;
    const bool any = acc.drain(dsm);
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        const int row = e % m, col = e / m;
        C[row + (int64_t)col * ldc] = any ? acc.entry(dsm, row, col) : make_float2(0.f, 0.f);
    }
    acc.close();
}

}  // namespace
}  // namespace hm

extern "C" int hm_tc_cgemm(int32_t m, int32_t k, int32_t ncols, const void *dA, int64_t lda, const void *dB,
                           int64_t ldb, void *dC, int64_t ldc, void *stream)
{
    if (m < 1 || m > 64 || ncols < 1 || ncols > 64 || k < 0 || !dC || (k > 0 && (!dA || !dB)) || lda < m ||
        ldb < k || ldc < m)
        return HM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    const int zero = 0;
    static hm::DeviceOnce attr;
    if (attr.need()) {
        if ((e = cudaFuncSetAttribute(hm::k_tc_cgemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)hm::tc::SMEM_BYTES)))
            return HM_ECUDA;
        attr.done();
    }
    if ((e = cudaMemcpyToSymbolAsync(hm::g_tc_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st)))
        return HM_ECUDA;
    hm::k_tc_cgemm<<<1, 256, hm::tc::SMEM_BYTES, st>>>(m, k, ncols, (const float2 *)dA, lda, (const float2 *)dB, ldb,
                                                       (float2 *)dC, ldc);
    int herr = 0;
    if ((e = cudaGetLastError()) ||
        (e = cudaMemcpyFromSymbolAsync(&herr, hm::g_tc_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st))) {
        std::fprintf(stderr, "hm_tc_cgemm: %s\n", cudaGetErrorString(e));
        return HM_ECUDA;
    }
    return herr ? HM_ETIMEOUT : HM_OK;
}
