// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05, sm_103a)
// for the surrogate network's dense layers.
//
//   C[M x N] = A[M x K] * B[N x K]^T        (both operands K-major, BF16;
//                                             FP32 accumulation in TMEM)
//
// One CTA of 128 threads computes a 128 x BN tile (BN = N <= 256, a multiple
// of 16).  K advances in chunks of 64: all threads stage the A and B chunks
// into shared memory in the canonical no-swizzle K-major layout (8-row x
// 16-byte core matrices; along K 128 bytes apart, along M/N 1024 bytes
// apart), one elected thread issues four tcgen05.mma (K = 16 each) and
// commits them to an mbarrier, everybody waits on it, and the next chunk
// overwrites the tile.  The accumulator lives in TMEM (128 lanes x BN
// columns); the epilogue reads it with tcgen05.ld (warp w owns lanes
// 32w..32w+31, i.e. rows 32w..32w+31 of the tile) and applies a fused
// elementwise operation.  Every mbarrier wait is bounded: on timeout the
// kernel waits (bounded) once more for the outstanding commit, records an
// error, skips the rest and frees its TMEM.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace amfrw {
namespace tc {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kThreads = 128;
constexpr uint32_t kSpinLimit = 1u << 26;  // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K
// direction) and stride (M/N direction) byte offsets, descriptor version 1,
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // version
    // base offset 0, layout type 0 (no swizzle)
    return d;
}

// Instruction descriptor of tcgen05.mma.kind::f16: FP32 accumulator, BF16 A
// and B, both K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

// Wait for the phase with the given parity; false if the bound was hit.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P1;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P1;\n\t}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) of a tile in the no-swizzle K-major core
// matrix layout with kBK columns: core matrix (row/8, k/8) at
// ((row/8) * (kBK/8) + k/8) * 128, row%8 at 16-byte stride.
__device__ __forceinline__ uint32_t tile_off(int row, int k)
{
    return (uint32_t)((((row >> 3) * (kBK >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

constexpr uint32_t kLBO = 128;               // next core matrix along K
constexpr uint32_t kSBO = (kBK / 8) * 128;   // next 8-row group along M/N

// Shared memory of one CTA: A tile, B tile (BN <= 256), mbarrier, TMEM address.
// The tiles are allocated at twice their size so that descriptor offsets can
// never address beyond the block's allocation.
constexpr int kTileA = kBM * kBK * 2;
constexpr int kTileB = 256 * kBK * 2;
constexpr size_t kSmemBytes = 2 * (kTileA + kTileB) + 64;

struct Epi {
    int mode;             // 0: C = acc (FP32); 1: Z = acc + bias, H = gelu(Z) (BF16), Ht
                          // 2: D = acc * gelu'(Zprev) -> BF16 D and Dt
    float* C;             // mode 0: [M x N] FP32, row stride ldc
    int ldc;
    const float* bias;    // mode 1: [N]
    float* Z;             // mode 1: [M x N] FP32 pre-activation (row stride N), may be null
    __nv_bfloat16* H;     // mode 1/2: [M x N] BF16 (row stride N)
    __nv_bfloat16* Ht;    // mode 1/2: [N x M] BF16 transpose (row stride ldt), may be null
    int ldt;
    const float* Zprev;   // mode 2: [M x N] FP32 pre-activation of this layer
    int* error;           // set when a bounded wait gave up
};

__device__ __forceinline__ float gelu(float z)
{
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad(float z)
{
    const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    const float pdf = 0.3989422804014327f * __expf(-0.5f * z * z);
    return cdf + z * pdf;
}

// C-tile = A[m0:m0+128, :] * B[n0:n0+BN, :]^T; grid (M/128, N/BN).
__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_kernel(const __nv_bfloat16* __restrict__ A, int lda, const __nv_bfloat16* __restrict__ B,
                     int ldb, int M, int N, int K, int BN, Epi epi)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + 2 * kTileA;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * (kTileA + kTileB));
    uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(smem + 2 * (kTileA + kTileB) + 16);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int m0 = blockIdx.x * kBM;
    const int n0 = blockIdx.y * BN;
    const uint32_t ncols = BN <= 32 ? 32u : (BN <= 64 ? 64u : (BN <= 128 ? 128u : 256u));

    if (warp == 0) tmem_alloc(smem_u32(taddr_slot), ncols);
    if (tid == 0) {
        mbar_init(smem_u32(mbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *taddr_slot;
    const uint32_t idesc = instr_desc_bf16(kBM, BN);
    uint32_t phase = 0;
    bool ok = true;

    for (int k0 = 0; k0 < K && ok; k0 += kBK) {
        const int kc = (K - k0) < kBK ? (K - k0) : kBK;  // multiple of 16
        // stage A (128 rows) and B (BN rows): 16-byte chunks of 8 elements
        for (int q = tid; q < kBM * (kBK / 8); q += kThreads) {
            const int r = q / (kBK / 8), c8 = (q % (kBK / 8)) * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (c8 < kc && m0 + r < M) v = *reinterpret_cast<const uint4*>(A + (size_t)(m0 + r) * lda + k0 + c8);
            *reinterpret_cast<uint4*>(sA + tile_off(r, c8)) = v;
        }
        for (int q = tid; q < BN * (kBK / 8); q += kThreads) {
            const int r = q / (kBK / 8), c8 = (q % (kBK / 8)) * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (c8 < kc && n0 + r < N) v = *reinterpret_cast<const uint4*>(B + (size_t)(n0 + r) * ldb + k0 + c8);
            *reinterpret_cast<uint4*>(sB + tile_off(r, c8)) = v;
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            for (int kk = 0; kk < kc / 16; ++kk) {
                const uint64_t da = smem_desc(smem_u32(sA) + kk * 2 * kLBO, kLBO, kSBO);
                const uint64_t db = smem_desc(smem_u32(sB) + kk * 2 * kLBO, kLBO, kSBO);
                mma_bf16(tmem, da, db, idesc, (k0 > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(smem_u32(mbar));
        }
        __syncthreads();
        // every thread waits; the block agrees on the outcome so that all
        // threads take the same path afterwards
        ok = __syncthreads_and(mbar_wait(smem_u32(mbar), phase) ? 1 : 0) != 0;
        if (!ok) {
            // The committed MMAs may still be writing the accumulator: wait
            // for that commit once more (also bounded) before TMEM is freed
            // below, so that the dealloc does not release columns an MMA in
            // flight still writes.
            __syncthreads_and(mbar_wait(smem_u32(mbar), phase) ? 1 : 0);
        }
        phase ^= 1u;
        fence_after();
    }
    if (!ok) {
        if (tid == 0) atomicExch(epi.error, 1);
    } else {
        // epilogue: row m0 + 32*warp + lane, columns 8 at a time
        const int row = m0 + warp * 32 + (tid & 31);
        for (int c = 0; c < BN; c += 8) {
            float v[8];
            tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            if (row >= M) continue;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int col = n0 + c + i;
                if (col >= N) break;
                if (epi.mode == 0) {
                    epi.C[(size_t)row * epi.ldc + col] = v[i];
                } else if (epi.mode == 1) {
                    const float z = v[i] + epi.bias[col];
                    if (epi.Z) epi.Z[(size_t)row * N + col] = z;
                    const __nv_bfloat16 h = __float2bfloat16(gelu(z));
                    epi.H[(size_t)row * N + col] = h;
                    if (epi.Ht) epi.Ht[(size_t)col * epi.ldt + row] = h;
                } else {
                    const float d = v[i] * gelu_grad(epi.Zprev[(size_t)row * N + col]);
                    const __nv_bfloat16 h = __float2bfloat16(d);
                    epi.H[(size_t)row * N + col] = h;
                    if (epi.Ht) epi.Ht[(size_t)col * epi.ldt + row] = h;
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace tc
}  // namespace amfrw
