// Surrogate network kernels: tensor-core GEMM launcher (tcgen05) and its C
// entry point.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/amfrw.h"
#include "amfrw_tc.cuh"

namespace amfrw {
namespace tc {

// C[M x N] = A[M x K] * B[N x K]^T with the fused epilogue `epi`; N split in
// column tiles of at most 256.
int gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
         const Epi& epi, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        attr = true;
    }
    const int BN = N <= 256 ? N : 256;
    dim3 grid((M + kBM - 1) / kBM, (N + BN - 1) / BN);
    gemm_bf16_kernel<<<grid, kThreads, kSmemBytes, st>>>(A, lda, B, ldb, M, N, K, BN, epi);
    return (int)cudaGetLastError();
}

}  // namespace tc
}  // namespace amfrw

using namespace amfrw;

extern "C" int amfrw_tc_gemm_bf16(const void* dA, int32_t lda, const void* dB, int32_t ldb, float* dC,
                                  int32_t ldc, int32_t M, int32_t N, int32_t K, void* cuda_stream)
{
    if (!dA || !dB || !dC) return AMFRW_EINVAL;
    if (M < 1 || N < 16 || N % 16 || K < 16 || K % 16 || lda % 8 || ldb % 8 || lda < K || ldb < K || ldc < N)
        return AMFRW_EINVAL;
    if ((N > 256 && N % 256) || ((uintptr_t)dA & 15) || ((uintptr_t)dB & 15)) return AMFRW_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int* d_err = nullptr;
    if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) return AMFRW_ENOMEM;
    cudaMemsetAsync(d_err, 0, sizeof(int), st);
    tc::Epi e{};
    e.mode = 0;
    e.C = dC;
    e.ldc = ldc;
    e.error = d_err;
    int rc = tc::gemm((const __nv_bfloat16*)dA, lda, (const __nv_bfloat16*)dB, ldb, M, N, K, e, st);
    int herr = 0;
    if (rc == 0) rc = (int)cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (rc == 0) rc = (int)cudaStreamSynchronize(st);
    cudaFree(d_err);
    if (rc != 0) return AMFRW_ECUDA;
    return herr ? AMFRW_ETIMEOUT : AMFRW_OK;
}
