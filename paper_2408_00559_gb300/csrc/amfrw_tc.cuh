// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05, sm_103a)
// for the surrogate network's dense layers.
//
//   C[M x N] = A[M x K] * B[N x K]^T        (both operands K-major, BF16;
//                                             FP32 accumulation in TMEM)
//
// One CTA of 128 threads computes a 128 x BN tile (BN = N <= 256, a multiple
// of 16).  K advances in chunks of 64 through a ring of up to four shared-
// memory stages filled by TMA (cp.async.bulk.tensor, one 16-byte-wide box of
// all the tile's rows per 8 elements of K, so each stage is the no-swizzle
// K-major layout of 8-row x 16-byte core matrices: 128 bytes apart along M/N,
// rows x 16 bytes apart along K).  One elected thread issues the loads of
// every stage up front, then for each chunk waits for its stage's "full"
// mbarrier (the TMA transaction count), issues four tcgen05.mma (K = 16 each)
// and commits them to the stage's "empty" mbarrier; the stage of the previous
// chunk is refilled with the chunk S ahead as soon as that commit completes,
// while the current chunk's MMAs run.  A final commit releases the epilogue:
// every warp reads its 32 TMEM lanes (rows) with tcgen05.ld and applies a
// fused elementwise operation.  Every mbarrier wait is bounded: on timeout
// the kernel records an error, waits (bounded) once more for the loads and
// MMAs it issued, skips the rest and frees its TMEM.
#pragma once
#include <cuda.h>
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

// 32 consecutive FP32 columns of this thread's TMEM lane (one wait for all).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

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

// Shared memory of one CTA: S stages of A (128 rows) and B (BN rows) x 64
// elements of K, then the mbarriers (full and empty per stage, done) and the
// TMEM address.  A stage's operand is 8 boxes of rows x 16 bytes.
constexpr int kMaxStages = 4;
constexpr int kTileA = kBM * kBK * 2;
__host__ __device__ constexpr int stage_bytes(int BN) { return kTileA + BN * kBK * 2; }
__host__ __device__ constexpr int smem_bytes(int BN, int stages) { return stages * stage_bytes(BN) + 8 * (2 * kMaxStages + 1) + 16; }

__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

// One 2-D TMA box (x = element along K, y = row) into shared memory,
// completing on the mbarrier with its byte count.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

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
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M,
                     int N, int K, int BN, int S, Epi epi)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int SB = stage_bytes(BN);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * SB);  // full[kMaxStages], empty[kMaxStages], done
    uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(smem + S * SB + 8 * (2 * kMaxStages + 1));
    __shared__ int s_fail;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int m0 = blockIdx.x * kBM;
    const int n0 = blockIdx.y * BN;
    const uint32_t ncols = BN <= 32 ? 32u : (BN <= 64 ? 64u : (BN <= 128 ? 128u : 256u));
    auto full = [&](int st) { return smem_u32(bars + st); };
    auto empty = [&](int st) { return smem_u32(bars + kMaxStages + st); };
    const uint32_t done = smem_u32(bars + 2 * kMaxStages);

    if (warp == 0) tmem_alloc(smem_u32(taddr_slot), ncols);
    if (tid == 0) {
        s_fail = 0;
        for (int st = 0; st < S; ++st) {
            mbar_init(full(st), 1);
            mbar_init(empty(st), 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *taddr_slot;
    const int nk = (K + kBK - 1) / kBK;

    if (tid == 0) {
        const uint32_t idesc = instr_desc_bf16(kBM, BN);
        const uint32_t lboA = kBM * 16, lboB = (uint32_t)BN * 16;  // next 8 elements of K
        const uint32_t tx = (uint32_t)SB;
        int pend[kMaxStages];  // loads issued and not yet waited for: their chunk, or -1
        auto load = [&](int i, int st) {
            const uint32_t a = smem_u32(smem + st * SB), b = a + kTileA;
            mbar_expect_tx(full(st), tx);
            for (int c = 0; c < kBK / 8; ++c) {
                tma_load_2d(a + c * lboA, &tmA, i * kBK + 8 * c, m0, full(st));
                tma_load_2d(b + c * lboB, &tmB, i * kBK + 8 * c, n0, full(st));
            }
            pend[st] = i;
        };
        for (int st = 0; st < kMaxStages; ++st) pend[st] = -1;
        for (int i = 0; i < S && i < nk; ++i) load(i, i);
        bool ok = true;
        int issued = 0;  // chunks whose MMAs were committed
        for (int i = 0; i < nk && ok; ++i) {
            const int st = i % S;
            const uint32_t ph = (uint32_t)((i / S) & 1);
            ok = mbar_wait(full(st), ph);
            if (!ok) break;
            pend[st] = -1;
            fence_after();
            const int kc = (K - i * kBK) < kBK ? (K - i * kBK) : kBK;  // multiple of 16
            const uint32_t a = smem_u32(smem + st * SB), b = a + kTileA;
            for (int kk = 0; kk < kc / 16; ++kk) {
                const uint64_t da = smem_desc(a + kk * 2 * lboA, lboA, 128);
                const uint64_t db = smem_desc(b + kk * 2 * lboB, lboB, 128);
                mma_bf16(tmem, da, db, idesc, (i > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(empty(st));
            issued = i + 1;
            // refill the previous chunk's stage once its MMAs are done (the
            // current chunk's MMAs keep the tensor pipe busy meanwhile)
            const int prev = i - 1, next = prev + S;
            if (prev >= 0 && next < nk) {
                const int ps = prev % S;
                ok = mbar_wait(empty(ps), (uint32_t)((prev / S) & 1));
                if (ok) load(next, ps);
            }
        }
        // the last commit covers every MMA issued above
        mma_commit(done);
        if (!ok) {
            // wait (bounded) for the loads still in flight, so that none lands
            // in shared memory after the block has gone
            for (int st = 0; st < S; ++st)
                if (pend[st] >= 0) mbar_wait(full(st), (uint32_t)((pend[st] / S) & 1));
            s_fail = 1;
        }
        (void)issued;
    }
    // every thread waits for the last commit; the block agrees on the outcome
    const bool fin = __syncthreads_and(mbar_wait(done, 0) ? 1 : 0) != 0;
    const bool ok = fin && s_fail == 0;
    fence_after();
    if (!ok) {
        if (!fin) __syncthreads_and(mbar_wait(done, 0) ? 1 : 0);  // once more before TMEM is freed
        if (tid == 0) atomicExch(epi.error, 1);
    } else {
        // epilogue: row m0 + 32*warp + lane, columns 8 at a time
        // (8 consecutive columns per thread and step: whole 32-byte sectors
        // for the FP32 outputs, 16-byte rows of the BF16 ones; N and the
        // tile offsets are multiples of 16)
        const int row = m0 + warp * 32 + (tid & 31);
        const bool vec_c = (epi.ldc & 3) == 0 && ((uintptr_t)epi.C & 15) == 0;
        for (int c32 = 0; c32 < BN; c32 += 32) {
          // TMEM columns 32 at a time (8 at a time for a 16-column tile)
          float w[32];
          const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c32;
          if (c32 + 32 <= BN) {
              tmem_ld32(ta, w);
          } else {
              float a8[8], b8[8];
              tmem_ld8(ta, a8);
              tmem_ld8(ta + 8, b8);
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                  w[i] = a8[i];
                  w[8 + i] = b8[i];
              }
          }
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const int c = c32 + 8 * g;
            if (c >= BN) break;
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = w[8 * g + i];
            const int col0 = n0 + c;
            if (row >= M || col0 >= N) continue;
            if (epi.mode == 0) {
                float* dst = epi.C + (size_t)row * epi.ldc + col0;
                if (vec_c) {
                    reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
                    reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) dst[i] = v[i];
                }
                continue;
            }
            __align__(16) __nv_bfloat16 h[8];
            if (epi.mode == 1) {
                float z[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    z[i] = v[i] + epi.bias[col0 + i];
                    h[i] = __float2bfloat16(gelu(z[i]));
                }
                if (epi.Z) {
                    float4* zd = reinterpret_cast<float4*>(epi.Z + (size_t)row * N + col0);
                    zd[0] = make_float4(z[0], z[1], z[2], z[3]);
                    zd[1] = make_float4(z[4], z[5], z[6], z[7]);
                }
            } else {
                const float4* zp = reinterpret_cast<const float4*>(epi.Zprev + (size_t)row * N + col0);
                const float4 za = zp[0], zb = zp[1];
                const float zz[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
#pragma unroll
                for (int i = 0; i < 8; ++i) h[i] = __float2bfloat16(v[i] * gelu_grad(zz[i]));
            }
            *reinterpret_cast<uint4*>(epi.H + (size_t)row * N + col0) = *reinterpret_cast<const uint4*>(h);
            if (epi.Ht) {
#pragma unroll
                for (int i = 0; i < 8; ++i) epi.Ht[(size_t)(col0 + i) * epi.ldt + row] = h[i];
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
