// Surrogate network kernels: tensor-core GEMM launcher (tcgen05) and its C
// entry point.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "../../include/amfrw.h"
#include "amfrw_tc.cuh"

namespace amfrw {
namespace tc {

// cuTensorMapEncodeTiled from the driver, looked up through the runtime (no
// link against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor map of a row-major BF16 matrix [rows x K] with leading dimension ld
// (elements): boxes of 8 elements of K by box_rows rows, no swizzle, zero fill
// outside the matrix.
bool make_map(CUtensorMap* tm, const __nv_bfloat16* base, int rows, int K, int ld, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {8, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C[M x N] = A[M x K] * B[N x K]^T with the fused epilogue `epi`; N split in
// column tiles of at most 256.  A, B: 16-byte aligned, lda and ldb multiples
// of 8 (the tensor maps' row strides are multiples of 16 bytes).
int gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
         const Epi& epi, cudaStream_t st)
{
    const int BN = N <= 256 ? N : 256;
    const int nk = (K + kBK - 1) / kBK;
    // at most two stages of the widest tile (96 KB), so that two CTAs share an
    // SM and one's epilogue overlaps the other's loads and MMAs
    int S = kMaxStages;
    while (S > 1 && (S > nk || smem_bytes(BN, S) > 110 * 1024)) --S;
    const int smem = smem_bytes(BN, S);
    // The dynamic shared-memory limit is a per-device attribute of the
    // kernel: raise it once on every device that launches it (to the most any
    // launch asks for).
    static std::mutex mu;
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!attr[dev]) {
            e = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 1024);
            if (e != cudaSuccess) return (int)e;
            attr[dev] = true;
        }
    }
    CUtensorMap tA, tB;
    if (!make_map(&tA, A, M, K, lda, kBM) || !make_map(&tB, B, N, K, ldb, BN)) return (int)cudaErrorInvalidValue;
    dim3 grid((M + kBM - 1) / kBM, (N + BN - 1) / BN);
    gemm_bf16_kernel<<<grid, kThreads, smem, st>>>(tA, tB, M, N, K, BN, S, epi);
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

// ===========================================================================
// Surrogate network: 8 features -> 256 -> 256 -> 256 -> 1, GELU, BF16 weights
// and activations for the tensor-core GEMMs, FP32 accumulation, FP32 master
// weights trained with Adam; an ensemble of independently seeded members
// whose spread estimates the error.  All arithmetic runs in the kernels below
// and in the tcgen05 GEMM.
// ===========================================================================
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <random>
#include <vector>

namespace amfrw {
namespace sg {

constexpr int kIn = 8;        // features
constexpr int kMaxLattice = 32;  // most distinct training values of a feature treated as a lattice
constexpr int kInPad = 16;    // first-layer K padded to the MMA's K
constexpr int kW = 256;       // hidden width
constexpr int kTrainRows = 1024;
constexpr int kPredRows = 65536;
// FP32 parameter vector of one member
constexpr int oW1 = 0;
constexpr int ob1 = oW1 + kW * kInPad;
constexpr int oW2 = ob1 + kW;
constexpr int ob2 = oW2 + kW * kW;
constexpr int oW3 = ob2 + kW;
constexpr int ob3 = oW3 + kW * kW;
constexpr int ow4 = ob3 + kW;
constexpr int ob4 = ow4 + kW;
constexpr int kParams = ob4 + 1;
// control variate: every monomial of degree <= 3 in the 8 normalised features
constexpr int kPolyTerms = 1 + kIn + kIn * (kIn + 1) / 2 + kIn * (kIn + 1) * (kIn + 2) / 6;

using bf16 = __nv_bfloat16;

// The monomials 1, z_i, z_i z_j (i <= j), z_i z_j z_k (i <= j <= k) of one
// feature row, handed to emit(q, value) in that order; the host (least-squares
// fit) and the device (prediction) share this definition so the two agree
// term by term.
template <class Emit>
__host__ __device__ inline void poly_each(const float* z, Emit emit)
{
    int q = 0;
    emit(q++, 1.0);
    for (int i = 0; i < kIn; ++i) emit(q++, (double)z[i]);
    for (int i = 0; i < kIn; ++i)
        for (int j = i; j < kIn; ++j) emit(q++, (double)z[i] * (double)z[j]);
    for (int i = 0; i < kIn; ++i)
        for (int j = i; j < kIn; ++j)
            for (int k = j; k < kIn; ++k) emit(q++, (double)z[i] * (double)z[j] * (double)z[k]);
}

inline void poly_terms(const float* z, double* m)
{
    poly_each(z, [m](int q, double v) { m[q] = v; });
}

// g_b = poly(z_b) + ymu + ysd * mean_b: the predicted target (log price or
// price) in FP64, from the ensemble mean of the standardised residual.
__global__ void finish_kernel(const float* __restrict__ z, const double* __restrict__ coef,
                              const float* __restrict__ mean, int n, double ymu, double ysd, double* g)
{
    __shared__ double c[kPolyTerms];
    for (int q = threadIdx.x; q < kPolyTerms; q += blockDim.x) c[q] = coef[q];
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    float zb[kIn];
    for (int i = 0; i < kIn; ++i) zb[i] = z[(size_t)b * kIn + i];
    double acc = 0.0;
    poly_each(zb, [&](int q, double v) { acc += c[q] * v; });
    g[b] = acc + ymu + ysd * (double)mean[b];
}

// Batch of rows (gathered through idx, or consecutive from r0) as BF16 input
// X [B x 16] (features then zero padding), its transpose Xt [16 x B], and
// the targets.
__global__ void pack_kernel(const float* __restrict__ feats, const float* __restrict__ targets,
                            const int* __restrict__ idx, int r0, int B, bf16* X, bf16* Xt, float* t)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B * kInPad) return;
    const int b = q / kInPad, c = q % kInPad;
    const int row = idx ? idx[b] : r0 + b;
    const float v = c < kIn ? feats[(size_t)row * kIn + c] : 0.0f;
    const bf16 h = __float2bfloat16(v);
    X[(size_t)b * kInPad + c] = h;
    if (Xt) Xt[(size_t)c * B + b] = h;
    if (c == 0 && t) t[b] = targets[row];
}

// y_b = H3_b . w4 + b4 (one warp per row).
__global__ void out_fwd_kernel(const bf16* __restrict__ H3, const float* __restrict__ P, float* y, int B)
{
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    float s = 0.0f;
    for (int k = lane; k < kW; k += 32) s += __bfloat162float(H3[(size_t)b * kW + k]) * P[ow4 + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[b] = s + P[ob4];
}

// L = 1/2 mean (y - t)^2: dy = (y - t)/B, dZ3 = dy w4 gelu'(Z3) (BF16 and its
// transpose), loss accumulated into *loss.
__global__ void out_bwd_kernel(const float* __restrict__ y, const float* __restrict__ t,
                               const float* __restrict__ P, const float* __restrict__ Z3, int B,
                               bf16* dZ3, bf16* dZ3t, float* dy, float* loss)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B * kW) return;
    const int b = q / kW, k = q % kW;
    const float r = y[b] - t[b];
    const float d = r / (float)B;
    if (k == 0) {
        dy[b] = d;
        atomicAdd(loss, 0.5f * r * r / (float)B);
    }
    const bf16 h = __float2bfloat16(d * P[ow4 + k] * tc::gelu_grad(Z3[(size_t)b * kW + k]));
    dZ3[(size_t)b * kW + k] = h;
    dZ3t[(size_t)k * B + b] = h;
}

// Output-layer gradients: g_w4[k] = sum_b dy_b H3[b][k], g_b4 = sum_b dy_b.
__global__ void out_wgrad_kernel(const bf16* __restrict__ H3, const float* __restrict__ dy, int B, float* G)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > kW) return;
    float s = 0.0f;
    if (k < kW) {
        for (int b = 0; b < B; ++b) s += dy[b] * __bfloat162float(H3[(size_t)b * kW + k]);
        G[ow4 + k] = s;
    } else {
        for (int b = 0; b < B; ++b) s += dy[b];
        G[ob4] = s;
    }
}

// Bias gradients from the transposed layer gradient dZt [N x B]: one warp per row.
__global__ void rowsum_kernel(const bf16* __restrict__ dZt, int N, int B, float* gb)
{
    const int n = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (n >= N) return;
    float s = 0.0f;
    for (int b = lane; b < B; b += 32) s += __bfloat162float(dZt[(size_t)n * B + b]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) gb[n] = s;
}

__global__ void adam_kernel(float* P, const float* __restrict__ G, float* Mo, float* Vo, int n, float lr,
                            float b1, float b2, float eps, float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float m = b1 * Mo[i] + (1.0f - b1) * g;
    const float v = b2 * Vo[i] + (1.0f - b2) * g * g;
    Mo[i] = m;
    Vo[i] = v;
    P[i] -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
}

// BF16 copy of a weight matrix [rows x cols] and optionally its transpose.
__global__ void cast_kernel(const float* __restrict__ W, int rows, int cols, bf16* Wb, bf16* Wtb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int r = i / cols, c = i % cols;
    const bf16 h = __float2bfloat16(W[i]);
    Wb[i] = h;
    if (Wtb) Wtb[(size_t)c * rows + r] = h;
}

// Ensemble mean and sample standard deviation of the members' outputs.
__global__ void ensemble_kernel(const float* __restrict__ ys, int members, int n, float* mean, float* spread)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int m = 0; m < members; ++m) s += ys[(size_t)m * n + i];
    const float mu = s / (float)members;
    float q = 0.0f;
    for (int m = 0; m < members; ++m) {
        const float d = ys[(size_t)m * n + i] - mu;
        q += d * d;
    }
    mean[i] = mu;
    spread[i] = members > 1 ? sqrtf(q / (float)(members - 1)) : 0.0f;
}

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

}  // namespace sg
}  // namespace amfrw

using namespace amfrw::sg;

namespace {

thread_local std::string g_sg_error;

int sg_fail(int st, const std::string& m)
{
    g_sg_error = m;
    return st;
}

#define SG_CUDA(expr)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) return sg_fail(AMFRW_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// The instance family a surrogate serves.  The features vary: alpha (one value
// shared by all rates), sigma, beta, K, T, the decay lambda of the rate
// correlations rho_ik = exp(-lambda |i - k|), and the rate/vol correlations
// phi_i, linear in the rate index between phi_1 and phi_{N-1}.  Every other
// field of amfrw_params is fixed by the family.  With that structure the eight
// features determine an instance, so the price is a function of them.
struct Family {
    int32_t n_rates, payoff, n_steps, level, psi, full_grid, precision, pad;
    double F0[7], Fmax[7], tau[7];
    double V0, Vmax, discount, theta, nu;
};

bool close_(double a, double b) { return std::fabs(a - b) <= 1e-12 * std::max(1.0, std::fabs(b)); }

Family family_of(const amfrw_params& p)
{
    Family f{};
    f.n_rates = p.n_rates;
    f.payoff = p.payoff;
    f.n_steps = p.n_steps;
    f.level = p.level;
    f.psi = p.psi;
    f.full_grid = p.full_grid;
    f.precision = p.precision;
    for (int i = 0; i < p.n_rates; ++i) {
        f.F0[i] = p.F0[i];
        f.Fmax[i] = p.Fmax[i];
        f.tau[i] = p.tau[i];
    }
    f.V0 = p.V0;
    f.Vmax = p.Vmax;
    f.discount = p.discount;
    f.theta = p.theta;
    f.nu = p.nu_amf;
    return f;
}

// (alpha, sigma, beta, K, T, lambda, phi_1, phi_{N-1})
void features_of(const amfrw_params& p, double* f)
{
    const int nr = p.n_rates;
    f[0] = p.alpha[0];
    f[1] = p.sigma;
    f[2] = p.beta;
    f[3] = p.K;
    f[4] = p.T;
    f[5] = nr > 1 && p.rho[1] > 0.0 ? -std::log(p.rho[1]) : 0.0;
    f[6] = p.phi[0];
    f[7] = p.phi[nr - 1];
}

bool in_family(const Family& f, const amfrw_params& p)
{
    if (p.n_rates != f.n_rates || p.payoff != f.payoff || p.n_steps != f.n_steps || p.level != f.level ||
        p.psi != f.psi || p.full_grid != f.full_grid || p.precision != f.precision)
        return false;
    const int nr = p.n_rates;
    if (nr > 1 && !(p.rho[1] > 0.0 && p.rho[1] <= 1.0)) return false;
    double feat[8];
    features_of(p, feat);
    for (int i = 0; i < nr; ++i) {
        if (!close_(p.F0[i], f.F0[i]) || !close_(p.Fmax[i], f.Fmax[i]) || !close_(p.tau[i], f.tau[i]))
            return false;
        if (!close_(p.alpha[i], p.alpha[0])) return false;
        const double lin = nr > 1 ? feat[6] + (double)i / (double)(nr - 1) * (feat[7] - feat[6]) : feat[6];
        if (!close_(p.phi[i], lin)) return false;
        for (int k = 0; k < nr; ++k)
            if (!close_(p.rho[i * nr + k], std::exp(-feat[5] * std::fabs((double)(i - k))))) return false;
    }
    return close_(p.V0, f.V0) && close_(p.Vmax, f.Vmax) && close_(p.discount, f.discount) &&
           close_(p.theta, f.theta) && close_(p.nu_amf, f.nu);
}

// The family's instance with raw features f; the arrays live in `st`.
struct InstanceStore {
    double alpha[7], phi[7], rho[49], tau[7], F0[7], Fmax[7];
};

amfrw_params params_from(const Family& fam, const double* f, InstanceStore& st)
{
    const int nr = fam.n_rates;
    for (int i = 0; i < nr; ++i) {
        st.alpha[i] = f[0];
        st.phi[i] = nr > 1 ? f[6] + (double)i / (double)(nr - 1) * (f[7] - f[6]) : f[6];
        st.tau[i] = fam.tau[i];
        st.F0[i] = fam.F0[i];
        st.Fmax[i] = fam.Fmax[i];
        for (int k = 0; k < nr; ++k) st.rho[i * nr + k] = std::exp(-f[5] * std::fabs((double)(i - k)));
    }
    amfrw_params p{};
    p.n_rates = nr;
    p.payoff = fam.payoff;
    p.n_steps = fam.n_steps;
    p.level = fam.level;
    p.psi = fam.psi;
    p.full_grid = fam.full_grid;
    p.precision = fam.precision;
    p.alpha = st.alpha;
    p.phi = st.phi;
    p.rho = st.rho;
    p.tau = st.tau;
    p.F0 = st.F0;
    p.Fmax = st.Fmax;
    p.sigma = f[1];
    p.beta = f[2];
    p.V0 = fam.V0;
    p.Vmax = fam.Vmax;
    p.K = f[3];
    p.T = f[4];
    p.discount = fam.discount;
    p.theta = fam.theta;
    p.nu_amf = fam.nu;
    return p;
}

}  // namespace

// Work buffers of one forward/backward pass: the packed batch, activations,
// pre-activations and gradients, and the stream the pass runs on.  Prediction
// and gradient checks use one set on the caller's stream; training gives every
// member its own set and stream, so the members' steps run concurrently.
struct SgWork {
    bf16 *X = nullptr, *Xt = nullptr, *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *H1t = nullptr, *H2t = nullptr;
    bf16 *dZ1 = nullptr, *dZ2 = nullptr, *dZ3 = nullptr, *dZ1t = nullptr, *dZ2t = nullptr, *dZ3t = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *y = nullptr, *t = nullptr, *dy = nullptr, *loss = nullptr;
    int* idx = nullptr;  // training: the epoch's permutation of the rows
    cudaStream_t st = nullptr;
    bool own_stream = false;
    void release()
    {
        for (void* q : {(void*)X, (void*)Xt, (void*)H1, (void*)H2, (void*)H3, (void*)H1t, (void*)H2t,
                        (void*)dZ1, (void*)dZ2, (void*)dZ3, (void*)dZ1t, (void*)dZ2t, (void*)dZ3t,
                        (void*)Z1, (void*)Z2, (void*)Z3, (void*)y, (void*)t, (void*)dy, (void*)loss, (void*)idx})
            cudaFree(q);
        if (own_stream && st) cudaStreamDestroy(st);
        *this = SgWork{};
    }
};

struct amfrw_surrogate {
    int members = 0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    std::vector<float*> P, G, Mo, Vo;
    std::vector<bf16*> W1b, W2b, W3b, W2tb, W3tb;
    SgWork w;                  // prediction chunk (kPredRows) and gradient checks (kTrainRows)
    float* ys = nullptr;       // prediction chunk: every member's output
    float *pmean = nullptr, *pspread = nullptr;  // prediction chunk: ensemble mean, spread
    double *pg = nullptr, *dpoly = nullptr;      // prediction chunk: target; control-variate coefficients
    int* err = nullptr;
    double poly[kPolyTerms] = {};
    int adam_t = 0;
    double fmin[kIn], fmax[kIn];
    // features that took at most kMaxLattice distinct values in the training
    // set (a lattice, e.g. strikes): queries must lie on one of them
    int nlat[kIn] = {};
    double lat[kIn][kMaxLattice] = {};
    double ymu = 0.0, ysd = 1.0;    // target scaling: t = (g(price) - ymu) / ysd
    bool log_target = false;        // g = log (all training prices > 0), else identity
    double calib = 0.0, rel_bound = 1e-3;
    bool trained = false, calibrated = false;
    Family fam{};
    ~amfrw_surrogate()
    {
        for (auto v : {&P, &G, &Mo, &Vo})
            for (float* q : *v) cudaFree(q);
        for (auto v : {&W1b, &W2b, &W3b, &W2tb, &W3tb})
            for (bf16* q : *v) cudaFree(q);
        w.release();
        for (void* q : {(void*)ys, (void*)err, (void*)pmean, (void*)pspread, (void*)pg, (void*)dpoly}) cudaFree(q);
    }
};

namespace {

// Buffers of one pass set: forward rows (activations) and training rows
// (transposes, pre-activations, gradients).
int sg_work_alloc(SgWork& w, size_t fwd_rows, size_t train_rows)
{
    const size_t B2 = sizeof(bf16), F4 = sizeof(float);
    SG_CUDA(cudaMalloc(&w.X, B2 * fwd_rows * kInPad));
    SG_CUDA(cudaMalloc(&w.Xt, B2 * train_rows * kInPad));
    for (bf16** q : {&w.H1, &w.H2, &w.H3}) SG_CUDA(cudaMalloc(q, B2 * fwd_rows * kW));
    for (bf16** q : {&w.H1t, &w.H2t, &w.dZ1, &w.dZ2, &w.dZ3, &w.dZ1t, &w.dZ2t, &w.dZ3t})
        SG_CUDA(cudaMalloc(q, B2 * train_rows * kW));
    for (float** q : {&w.Z1, &w.Z2, &w.Z3}) SG_CUDA(cudaMalloc(q, F4 * train_rows * kW));
    SG_CUDA(cudaMalloc(&w.y, F4 * fwd_rows));
    SG_CUDA(cudaMalloc(&w.t, F4 * train_rows));
    SG_CUDA(cudaMalloc(&w.dy, F4 * train_rows));
    SG_CUDA(cudaMalloc(&w.loss, F4));
    return AMFRW_OK;
}

int sg_alloc(amfrw_surrogate* s)
{
    const size_t TR = kTrainRows, PR = kPredRows, PQ = std::max(TR, PR);
    const size_t B2 = sizeof(bf16), F4 = sizeof(float);
    for (int m = 0; m < s->members; ++m) {
        float *p, *g, *mo, *vo;
        bf16 *w1, *w2, *w3, *w2t, *w3t;
        SG_CUDA(cudaMalloc(&p, F4 * kParams));
        SG_CUDA(cudaMalloc(&g, F4 * kParams));
        SG_CUDA(cudaMalloc(&mo, F4 * kParams));
        SG_CUDA(cudaMalloc(&vo, F4 * kParams));
        SG_CUDA(cudaMalloc(&w1, B2 * kW * kInPad));
        SG_CUDA(cudaMalloc(&w2, B2 * kW * kW));
        SG_CUDA(cudaMalloc(&w3, B2 * kW * kW));
        SG_CUDA(cudaMalloc(&w2t, B2 * kW * kW));
        SG_CUDA(cudaMalloc(&w3t, B2 * kW * kW));
        s->P.push_back(p); s->G.push_back(g); s->Mo.push_back(mo); s->Vo.push_back(vo);
        s->W1b.push_back(w1); s->W2b.push_back(w2); s->W3b.push_back(w3);
        s->W2tb.push_back(w2t); s->W3tb.push_back(w3t);
    }
    s->w.st = s->stream;
    int st = sg_work_alloc(s->w, PQ, TR);
    if (st != AMFRW_OK) return st;
    SG_CUDA(cudaMalloc(&s->ys, F4 * PQ * (size_t)s->members));
    SG_CUDA(cudaMalloc(&s->err, sizeof(int)));
    SG_CUDA(cudaMalloc(&s->pmean, F4 * PR));
    SG_CUDA(cudaMalloc(&s->pspread, F4 * PR));
    SG_CUDA(cudaMalloc(&s->pg, sizeof(double) * PR));
    SG_CUDA(cudaMalloc(&s->dpoly, sizeof(double) * kPolyTerms));
    SG_CUDA(cudaMemsetAsync(s->dpoly, 0, sizeof(double) * kPolyTerms, s->stream));
    SG_CUDA(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream));
    return AMFRW_OK;
}

// BF16 weight copies of member m from its FP32 master weights.
void sg_cast(amfrw_surrogate* s, int m, cudaStream_t st)
{
    cast_kernel<<<cdiv(kW * kInPad, 256), 256, 0, st>>>(s->P[m] + oW1, kW, kInPad, s->W1b[m], nullptr);
    cast_kernel<<<cdiv(kW * kW, 256), 256, 0, st>>>(s->P[m] + oW2, kW, kW, s->W2b[m], s->W2tb[m]);
    cast_kernel<<<cdiv(kW * kW, 256), 256, 0, st>>>(s->P[m] + oW3, kW, kW, s->W3b[m], s->W3tb[m]);
}

// Forward pass of member m on B packed rows in w.X; output into y.  With
// train set, keeps the pre-activations and transposes the backward pass needs.
int sg_forward(amfrw_surrogate* s, int m, int B, bool train, float* y, const SgWork& w)
{
    cudaStream_t st = w.st;
    tc::Epi e{};
    e.mode = 1;
    e.error = s->err;
    e.ldt = B;
    e.bias = s->P[m] + ob1; e.Z = train ? w.Z1 : nullptr; e.H = w.H1; e.Ht = train ? w.H1t : nullptr;
    int rc = tc::gemm(w.X, kInPad, s->W1b[m], kInPad, B, kW, kInPad, e, st);
    e.bias = s->P[m] + ob2; e.Z = train ? w.Z2 : nullptr; e.H = w.H2; e.Ht = train ? w.H2t : nullptr;
    if (!rc) rc = tc::gemm(w.H1, kW, s->W2b[m], kW, B, kW, kW, e, st);
    e.bias = s->P[m] + ob3; e.Z = train ? w.Z3 : nullptr; e.H = w.H3; e.Ht = nullptr;
    if (!rc) rc = tc::gemm(w.H2, kW, s->W3b[m], kW, B, kW, kW, e, st);
    if (!rc) out_fwd_kernel<<<cdiv(B * 32, 256), 256, 0, st>>>(w.H3, s->P[m], y, B);
    if (rc) return sg_fail(AMFRW_ECUDA, std::string("surrogate forward: ") + cudaGetErrorString((cudaError_t)rc));
    return AMFRW_OK;
}

// Loss gradient of member m on the packed batch (targets in w.t) into s->G[m].
int sg_backward(amfrw_surrogate* s, int m, int B, const SgWork& w)
{
    cudaStream_t st = w.st;
    float* G = s->G[m];
    out_bwd_kernel<<<cdiv(B * kW, 256), 256, 0, st>>>(w.y, w.t, s->P[m], w.Z3, B, w.dZ3, w.dZ3t, w.dy, w.loss);
    out_wgrad_kernel<<<cdiv(kW + 1, 128), 128, 0, st>>>(w.H3, w.dy, B, G);
    tc::Epi e{};
    e.error = s->err;
    e.ldt = B;
    // W3, b3
    e.mode = 0; e.C = G + oW3; e.ldc = kW;
    int rc = tc::gemm(w.dZ3t, B, w.H2t, B, kW, kW, B, e, st);
    rowsum_kernel<<<cdiv(kW * 32, 256), 256, 0, st>>>(w.dZ3t, kW, B, G + ob3);
    // dZ2 = (dZ3 W3) * gelu'(Z2)
    e.mode = 2; e.H = w.dZ2; e.Ht = w.dZ2t; e.Zprev = w.Z2;
    if (!rc) rc = tc::gemm(w.dZ3, kW, s->W3tb[m], kW, B, kW, kW, e, st);
    e.mode = 0; e.C = G + oW2; e.ldc = kW;
    if (!rc) rc = tc::gemm(w.dZ2t, B, w.H1t, B, kW, kW, B, e, st);
    rowsum_kernel<<<cdiv(kW * 32, 256), 256, 0, st>>>(w.dZ2t, kW, B, G + ob2);
    // dZ1 = (dZ2 W2) * gelu'(Z1)
    e.mode = 2; e.H = w.dZ1; e.Ht = w.dZ1t; e.Zprev = w.Z1;
    if (!rc) rc = tc::gemm(w.dZ2, kW, s->W2tb[m], kW, B, kW, kW, e, st);
    e.mode = 0; e.C = G + oW1; e.ldc = kInPad;
    if (!rc) rc = tc::gemm(w.dZ1t, B, w.Xt, B, kW, kInPad, B, e, st);
    rowsum_kernel<<<cdiv(kW * 32, 256), 256, 0, st>>>(w.dZ1t, kW, B, G + ob1);
    if (rc) return sg_fail(AMFRW_ECUDA, std::string("surrogate backward: ") + cudaGetErrorString((cudaError_t)rc));
    return AMFRW_OK;
}

int sg_check_err(amfrw_surrogate* s)
{
    int h = 0;
    SG_CUDA(cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    SG_CUDA(cudaStreamSynchronize(s->stream));
    if (h) return sg_fail(AMFRW_ETIMEOUT, "a bounded wait in the tensor-core GEMM gave up");
    return AMFRW_OK;
}

// Least-squares coefficients of the cubic control variate: normal equations
// with a relative ridge of 1e-12 (which zeroes the terms of features that do
// not vary), solved by Cholesky.
bool fit_poly(const float* z, const double* g, int64_t n, double* coef)
{
    const int P = kPolyTerms;
    std::vector<double> A((size_t)P * P, 0.0), rhs(P, 0.0);
    double m[kPolyTerms];
    for (int64_t i = 0; i < n; ++i) {
        poly_terms(z + (size_t)i * kIn, m);
        for (int a = 0; a < P; ++a) {
            rhs[a] += m[a] * g[i];
            const double ma = m[a];
            double* row = A.data() + (size_t)a * P;
            for (int b = a; b < P; ++b) row[b] += ma * m[b];
        }
    }
    double tr = 0.0;
    for (int a = 0; a < P; ++a) tr += A[(size_t)a * P + a];
    const double ridge = 1e-12 * tr / P + 1e-300;
    for (int a = 0; a < P; ++a) {
        A[(size_t)a * P + a] += ridge;
        for (int b = 0; b < a; ++b) A[(size_t)a * P + b] = A[(size_t)b * P + a];
    }
    // A = L L^T in place (lower triangle)
    for (int j = 0; j < P; ++j) {
        double d = A[(size_t)j * P + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * P + k] * A[(size_t)j * P + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        A[(size_t)j * P + j] = d;
        for (int i = j + 1; i < P; ++i) {
            double v = A[(size_t)i * P + j];
            for (int k = 0; k < j; ++k) v -= A[(size_t)i * P + k] * A[(size_t)j * P + k];
            A[(size_t)i * P + j] = v / d;
        }
    }
    std::vector<double> y(P);
    for (int i = 0; i < P; ++i) {
        double v = rhs[i];
        for (int k = 0; k < i; ++k) v -= A[(size_t)i * P + k] * y[k];
        y[i] = v / A[(size_t)i * P + i];
    }
    for (int i = P - 1; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < P; ++k) v -= A[(size_t)k * P + i] * coef[k];
        coef[i] = v / A[(size_t)i * P + i];
    }
    for (int i = 0; i < P; ++i)
        if (!std::isfinite(coef[i])) return false;
    return true;
}

// Normalised features (host, n x 8 floats) of n rows of raw features; ok
// entries (may be NULL) cleared for rows outside the trained feature box.
void sg_normalise(const amfrw_surrogate* s, const double* raw, int64_t n, std::vector<float>& out, char* ok)
{
    out.assign((size_t)n * kIn, 0.0f);
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < kIn; ++c) {
            const double f = raw[(size_t)i * kIn + c];
            const double span = s->fmax[c] - s->fmin[c];
            const double z = span > 0 ? 2.0 * (f - s->fmin[c]) / span - 1.0 : (f == s->fmin[c] ? 0.0 : 2.0);
            if (ok && !(z >= -1.0 - 1e-9 && z <= 1.0 + 1e-9)) ok[i] = 0;
            if (ok && s->nlat[c] > 0) {  // a lattice feature: only its training values
                bool on = false;
                for (int q = 0; q < s->nlat[c] && !on; ++q)
                    on = std::fabs(f - s->lat[c][q]) <= 1e-12 * std::max(1.0, std::fabs(f));
                if (!on) ok[i] = 0;
            }
            out[(size_t)i * kIn + c] = (float)z;
        }
    }
}

// Raw features of n instances and whether each belongs to the family.
void sg_raw_features(const amfrw_surrogate* s, const amfrw_params* ps, int64_t n, std::vector<double>& raw,
                     std::vector<char>& ok)
{
    raw.assign((size_t)n * kIn, 0.0);
    ok.assign((size_t)n, 1);
    for (int64_t i = 0; i < n; ++i) {
        features_of(ps[i], raw.data() + (size_t)i * kIn);
        ok[(size_t)i] = in_family(s->fam, ps[i]) ? 1 : 0;
    }
}

// Ensemble mean and spread (price units) of n rows of normalised features on
// the device.
int sg_predict_dev(amfrw_surrogate* s, const float* d_feats, int64_t n, std::vector<double>& mean,
                   std::vector<double>& spread)
{
    cudaStream_t st = s->stream;
    mean.assign((size_t)n, 0.0);
    spread.assign((size_t)n, 0.0);
    std::vector<double> hg;
    std::vector<float> hs;
    for (int64_t r0 = 0; r0 < n; r0 += kPredRows) {
        const int B = (int)std::min<int64_t>(kPredRows, n - r0);
        const float* z = d_feats + (size_t)r0 * kIn;
        pack_kernel<<<cdiv(B * kInPad, 256), 256, 0, st>>>(z, nullptr, nullptr, 0, B, s->w.X, nullptr, nullptr);
        for (int m = 0; m < s->members; ++m) {
            const int rc = sg_forward(s, m, B, false, s->ys + (size_t)m * B, s->w);
            if (rc != AMFRW_OK) return rc;
        }
        ensemble_kernel<<<cdiv(B, 256), 256, 0, st>>>(s->ys, s->members, B, s->pmean, s->pspread);
        finish_kernel<<<cdiv(B, 128), 128, 0, st>>>(z, s->dpoly, s->pmean, B, s->ymu, s->ysd, s->pg);
        hg.resize(B);
        hs.resize(B);
        SG_CUDA(cudaMemcpyAsync(hg.data(), s->pg, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
        SG_CUDA(cudaMemcpyAsync(hs.data(), s->pspread, sizeof(float) * B, cudaMemcpyDeviceToHost, st));
        SG_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < B; ++i) {
            const double g = hg[i], sp = s->ysd * (double)hs[i];
            if (s->log_target) {  // spread to first order in price units
                mean[(size_t)(r0 + i)] = std::exp(g);
                spread[(size_t)(r0 + i)] = std::exp(g) * sp;
            } else {
                mean[(size_t)(r0 + i)] = g;
                spread[(size_t)(r0 + i)] = sp;
            }
        }
    }
    return sg_check_err(s);
}

// Prediction from raw features; ok (n entries, set by the caller for family
// membership) is cleared where a row leaves the feature box.
int sg_predict_raw(amfrw_surrogate* s, const double* raw, int64_t n, std::vector<double>& mean,
                   std::vector<double>& spread, std::vector<char>& ok)
{
    std::vector<float> feats;
    sg_normalise(s, raw, n, feats, ok.data());
    float* d = nullptr;
    SG_CUDA(cudaMalloc(&d, sizeof(float) * std::max<size_t>(1, feats.size())));
    cudaMemcpyAsync(d, feats.data(), sizeof(float) * feats.size(), cudaMemcpyHostToDevice, s->stream);
    const int st = sg_predict_dev(s, d, n, mean, spread);
    cudaFree(d);
    return st;
}

int sg_predict_host(amfrw_surrogate* s, const amfrw_params* ps, int64_t n, std::vector<double>& mean,
                    std::vector<double>& spread, std::vector<char>& ok)
{
    std::vector<double> raw;
    sg_raw_features(s, ps, n, raw, ok);
    return sg_predict_raw(s, raw.data(), n, mean, spread, ok);
}

// Answers from the network where the calibrated estimate is within the bound;
// the batched solver prices every other query (one batch per step count, at
// most 4096 instances each).  param(i) gives query i as amfrw_params.
template <class ParamOf>
int sg_serve(amfrw_surrogate* s, int64_t n, const std::vector<double>& mean, const std::vector<double>& spread,
             const std::vector<char>& ok, ParamOf param, double* prices_out, uint8_t* fell_back_out,
             void* cuda_stream)
{
    std::vector<int64_t> where;
    for (int64_t i = 0; i < n; ++i) {
        const double est = s->calib * spread[(size_t)i];
        const bool fall = !ok[(size_t)i] || !(est <= s->rel_bound * std::fabs(mean[(size_t)i]));
        if (fell_back_out) fell_back_out[i] = fall ? 1 : 0;
        if (fall)
            where.push_back(i);
        else
            prices_out[i] = mean[(size_t)i];
    }
    std::vector<InstanceStore> store;
    std::vector<amfrw_params> fb(where.size());
    store.resize(where.size());
    for (size_t k = 0; k < where.size(); ++k) fb[k] = param(where[k], store[k]);
    std::vector<size_t> order(fb.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return fb[a].n_steps < fb[b].n_steps; });
    std::vector<amfrw_params> grp;
    std::vector<double> pr;
    for (size_t k0 = 0; k0 < order.size();) {
        size_t k1 = k0;
        while (k1 < order.size() && k1 - k0 < 4096 && fb[order[k1]].n_steps == fb[order[k0]].n_steps) ++k1;
        grp.clear();
        for (size_t k = k0; k < k1; ++k) grp.push_back(fb[order[k]]);
        pr.assign(grp.size(), 0.0);
        const int st = amfrw_solve_batch(grp.data(), (int32_t)grp.size(), pr.data(), cuda_stream);
        if (st != AMFRW_OK) return sg_fail(st, std::string("fallback solve: ") + amfrw_last_error());
        for (size_t k = k0; k < k1; ++k) prices_out[where[order[k]]] = pr[k - k0];
        k0 = k1;
    }
    return AMFRW_OK;
}

}  // namespace

extern "C" {

const char* amfrw_surrogate_last_error(void) { return g_sg_error.c_str(); }

int amfrw_surrogate_create(int32_t n_members, uint64_t seed, void* cuda_stream, amfrw_surrogate** out)
{
    if (!out) return sg_fail(AMFRW_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_members < 1 || n_members > 16) return sg_fail(AMFRW_EINVAL, "n_members must be in [1, 16]");
    amfrw_surrogate* s = new (std::nothrow) amfrw_surrogate();
    if (!s) return sg_fail(AMFRW_ENOMEM, "host allocation failed");
    s->members = n_members;
    s->seed = seed;
    s->stream = (cudaStream_t)cuda_stream;
    int st = sg_alloc(s);
    if (st != AMFRW_OK) {
        delete s;
        return st;
    }
    // He-style initialisation of every member from its own seed
    std::vector<float> h(kParams);
    for (int m = 0; m < n_members; ++m) {
        std::mt19937_64 rng(seed * 1000003ull + (uint64_t)m);
        std::normal_distribution<float> nd(0.0f, 1.0f);
        std::fill(h.begin(), h.end(), 0.0f);
        for (int o = 0; o < kW; ++o)
            for (int i = 0; i < kIn; ++i) h[oW1 + o * kInPad + i] = nd(rng) * std::sqrt(2.0f / kIn);
        for (int q = 0; q < kW * kW; ++q) h[oW2 + q] = nd(rng) * std::sqrt(2.0f / kW);
        for (int q = 0; q < kW * kW; ++q) h[oW3 + q] = nd(rng) * std::sqrt(2.0f / kW);
        for (int q = 0; q < kW; ++q) h[ow4 + q] = nd(rng) * std::sqrt(1.0f / kW);
        cudaMemcpyAsync(s->P[m], h.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice, s->stream);
        cudaMemsetAsync(s->Mo[m], 0, sizeof(float) * kParams, s->stream);
        cudaMemsetAsync(s->Vo[m], 0, sizeof(float) * kParams, s->stream);
        sg_cast(s, m, s->stream);
    }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
        delete s;
        return sg_fail(AMFRW_ECUDA, "surrogate initialisation");
    }
    *out = s;
    return AMFRW_OK;
}

int amfrw_surrogate_fit(amfrw_surrogate* s, const amfrw_params* ps, const double* prices, int64_t n,
                        int32_t epochs, float lr, float* final_loss_out)
{
    if (!s || !ps || !prices) return sg_fail(AMFRW_EINVAL, "NULL argument");
    if (n < kTrainRows) return sg_fail(AMFRW_EINVAL, "need at least 1024 training instances");
    if (epochs < 1 || !(lr > 0.0f)) return sg_fail(AMFRW_EINVAL, "epochs >= 1 and lr > 0 required");
    // family, feature box and target scaling from the training set
    s->fam = family_of(ps[0]);
    for (int c = 0; c < kIn; ++c) {
        s->fmin[c] = 1e300;
        s->fmax[c] = -1e300;
    }
    std::vector<double> raw;
    std::vector<char> ok;
    sg_raw_features(s, ps, n, raw, ok);
    bool positive = true;
    for (int64_t i = 0; i < n; ++i) {
        if (!ok[(size_t)i]) return sg_fail(AMFRW_EINVAL, "training instances must share one family");
        if (!std::isfinite(prices[i])) return sg_fail(AMFRW_EINVAL, "non-finite training price");
        positive = positive && prices[i] > 0.0;
        for (int c = 0; c < kIn; ++c) {
            s->fmin[c] = std::min(s->fmin[c], raw[(size_t)i * kIn + c]);
            s->fmax[c] = std::max(s->fmax[c], raw[(size_t)i * kIn + c]);
        }
    }
    // features with at most kMaxLattice distinct training values (and more
    // than one) are lattices: the network is trained, and answers, only there
    for (int c = 0; c < kIn; ++c) {
        std::vector<double> v;
        s->nlat[c] = 0;
        for (int64_t i = 0; i < n && (int)v.size() <= kMaxLattice; ++i) {
            const double x = raw[(size_t)i * kIn + c];
            bool seen = false;
            for (double y : v) seen = seen || std::fabs(x - y) <= 1e-12 * std::max(1.0, std::fabs(x));
            if (!seen) v.push_back(x);
        }
        if (v.size() >= 2 && (int)v.size() <= kMaxLattice) {
            std::sort(v.begin(), v.end());
            s->nlat[c] = (int)v.size();
            for (size_t q = 0; q < v.size(); ++q) s->lat[c][q] = v[q];
        }
    }
    // the network learns log(price) when every price is positive (its squared
    // error is then the squared relative error), else the price itself
    s->log_target = positive;
    std::vector<double> g((size_t)n);
    for (int64_t i = 0; i < n; ++i) g[(size_t)i] = positive ? std::log(prices[i]) : prices[i];
    std::vector<float> feats, targ((size_t)n);
    sg_normalise(s, raw.data(), n, feats, nullptr);
    // control variate: least-squares cubic in the features; the networks
    // learn what it leaves, standardised
    if (!fit_poly(feats.data(), g.data(), n, s->poly)) return sg_fail(AMFRW_EINVAL, "control-variate fit failed");
    double sum = 0.0, sq = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double m[kPolyTerms], base = 0.0;
        poly_terms(feats.data() + (size_t)i * kIn, m);
        for (int q = 0; q < kPolyTerms; ++q) base += s->poly[q] * m[q];
        g[(size_t)i] -= base;
        sum += g[(size_t)i];
        sq += g[(size_t)i] * g[(size_t)i];
    }
    s->ymu = sum / (double)n;
    s->ysd = std::sqrt(std::max(sq / (double)n - s->ymu * s->ymu, 1e-300));
    for (int64_t i = 0; i < n; ++i) targ[(size_t)i] = (float)((g[(size_t)i] - s->ymu) / s->ysd);
    SG_CUDA(cudaMemcpyAsync(s->dpoly, s->poly, sizeof(double) * kPolyTerms, cudaMemcpyHostToDevice, s->stream));
    cudaStream_t st = s->stream;
    float *d_feats = nullptr, *d_targ = nullptr;
    SG_CUDA(cudaMalloc(&d_feats, sizeof(float) * feats.size()));
    SG_CUDA(cudaMalloc(&d_targ, sizeof(float) * n));
    cudaMemcpyAsync(d_feats, feats.data(), sizeof(float) * feats.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_targ, targ.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st);
    const int B = kTrainRows;
    const int64_t steps_per_epoch = n / B;
    const int64_t total = steps_per_epoch * epochs;
    // every member trains on its own stream with its own work buffers; the
    // members' steps are issued in turn, so their small kernels overlap
    const int M = s->members;
    std::vector<SgWork> tw((size_t)M);
    std::vector<std::mt19937_64> rng;
    std::vector<std::vector<int>> perm((size_t)M, std::vector<int>((size_t)n));
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> done((size_t)M, nullptr);
    int rc = AMFRW_OK;
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) rc = sg_fail(AMFRW_ECUDA, "event");
    if (rc == AMFRW_OK) cudaEventRecord(fork, st);
    for (int m = 0; m < M; ++m) {
        rng.emplace_back(s->seed * 7919ull + 17ull * (uint64_t)m + 1ull);
        if (rc != AMFRW_OK) continue;
        if (cudaStreamCreateWithFlags(&tw[(size_t)m].st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&done[(size_t)m], cudaEventDisableTiming) != cudaSuccess) {
            rc = sg_fail(AMFRW_ECUDA, "training streams");
            continue;
        }
        tw[(size_t)m].own_stream = true;
        rc = sg_work_alloc(tw[(size_t)m], B, B);
        if (rc == AMFRW_OK && cudaMalloc(&tw[(size_t)m].idx, sizeof(int) * n) != cudaSuccess)
            rc = sg_fail(AMFRW_ENOMEM, "training permutation");
        if (rc == AMFRW_OK) cudaStreamWaitEvent(tw[(size_t)m].st, fork, 0);  // after the uploads
    }
    float last = 0.0f;
    for (int ep = 0; ep < epochs && rc == AMFRW_OK; ++ep) {
        for (int m = 0; m < M; ++m) {
            SgWork& w = tw[(size_t)m];
            std::vector<int>& pm = perm[(size_t)m];
            for (int64_t i = 0; i < n; ++i) pm[(size_t)i] = (int)i;
            std::shuffle(pm.begin(), pm.end(), rng[(size_t)m]);
            cudaMemcpyAsync(w.idx, pm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, w.st);
            cudaMemsetAsync(w.loss, 0, sizeof(float), w.st);
        }
        for (int64_t k = 0; k < steps_per_epoch && rc == AMFRW_OK; ++k) {
            const int64_t step = (int64_t)ep * steps_per_epoch + k;
            // Adam with cosine decay to 1% of lr
            const double frac = (double)step / (double)std::max<int64_t>(1, total - 1);
            const float lr_t = (float)(lr * (0.01 + 0.99 * 0.5 * (1.0 + std::cos(M_PI * frac))));
            const int t = (int)step + 1;
            const float bc1 = 1.0f - std::pow(0.9f, (float)t), bc2 = 1.0f - std::pow(0.999f, (float)t);
            for (int m = 0; m < M && rc == AMFRW_OK; ++m) {
                const SgWork& w = tw[(size_t)m];
                pack_kernel<<<cdiv(B * kInPad, 256), 256, 0, w.st>>>(d_feats, d_targ, w.idx + k * B, 0, B, w.X,
                                                                    w.Xt, w.t);
                rc = sg_forward(s, m, B, true, w.y, w);
                if (rc == AMFRW_OK) rc = sg_backward(s, m, B, w);
                adam_kernel<<<cdiv(kParams, 256), 256, 0, w.st>>>(s->P[m], s->G[m], s->Mo[m], s->Vo[m], kParams,
                                                                 lr_t, 0.9f, 0.999f, 1e-8f, bc1, bc2);
                sg_cast(s, m, w.st);
            }
        }
        if (rc == AMFRW_OK && ep == epochs - 1) {
            for (int m = 0; m < M; ++m) {
                float hl = 0.0f;
                cudaMemcpyAsync(&hl, tw[(size_t)m].loss, sizeof(float), cudaMemcpyDeviceToHost, tw[(size_t)m].st);
                cudaStreamSynchronize(tw[(size_t)m].st);
                last += hl / (float)steps_per_epoch / (float)M;
            }
        }
    }
    // join: the caller's stream waits for every member
    for (int m = 0; m < M; ++m) {
        if (tw[(size_t)m].st && done[(size_t)m]) {
            cudaEventRecord(done[(size_t)m], tw[(size_t)m].st);
            cudaStreamWaitEvent(st, done[(size_t)m], 0);
        }
    }
    cudaStreamSynchronize(st);
    for (int m = 0; m < M; ++m) {
        tw[(size_t)m].release();
        if (done[(size_t)m]) cudaEventDestroy(done[(size_t)m]);
    }
    if (fork) cudaEventDestroy(fork);
    cudaFree(d_feats);
    cudaFree(d_targ);
    if (rc != AMFRW_OK) return rc;
    rc = sg_check_err(s);
    if (rc != AMFRW_OK) return rc;
    if (cudaGetLastError() != cudaSuccess) return sg_fail(AMFRW_ECUDA, "surrogate training kernels");
    s->trained = true;
    if (final_loss_out) *final_loss_out = last;
    return AMFRW_OK;
}

int amfrw_surrogate_predict(amfrw_surrogate* s, const amfrw_params* ps, int64_t n, double* mean_out,
                            double* spread_out, uint8_t* in_domain_out)
{
    if (!s || !ps || !mean_out || !spread_out) return sg_fail(AMFRW_EINVAL, "NULL argument");
    if (!s->trained) return sg_fail(AMFRW_EINVAL, "surrogate is not trained");
    std::vector<double> mean, spread;
    std::vector<char> ok;
    int st = sg_predict_host(s, ps, n, mean, spread, ok);
    if (st != AMFRW_OK) return st;
    for (int64_t i = 0; i < n; ++i) {
        mean_out[i] = mean[(size_t)i];
        spread_out[i] = spread[(size_t)i];
        if (in_domain_out) in_domain_out[i] = ok[(size_t)i] ? 1 : 0;
    }
    return AMFRW_OK;
}

int amfrw_surrogate_predict_features(amfrw_surrogate* s, const double* features, int64_t n, double* mean_out,
                                     double* spread_out, uint8_t* in_box_out)
{
    if (!s || !features || !mean_out || !spread_out) return sg_fail(AMFRW_EINVAL, "NULL argument");
    if (n < 0) return sg_fail(AMFRW_EINVAL, "n < 0");
    if (!s->trained) return sg_fail(AMFRW_EINVAL, "surrogate is not trained");
    std::vector<double> mean, spread;
    std::vector<char> ok((size_t)n, 1);
    int st = sg_predict_raw(s, features, n, mean, spread, ok);
    if (st != AMFRW_OK) return st;
    for (int64_t i = 0; i < n; ++i) {
        mean_out[i] = mean[(size_t)i];
        spread_out[i] = spread[(size_t)i];
        if (in_box_out) in_box_out[i] = ok[(size_t)i] ? 1 : 0;
    }
    return AMFRW_OK;
}

int amfrw_surrogate_calibrate(amfrw_surrogate* s, const amfrw_params* ps, const double* prices, int64_t n,
                              double rel_bound, double quantile, double* calib_out)
{
    if (!s || !ps || !prices) return sg_fail(AMFRW_EINVAL, "NULL argument");
    if (!s->trained) return sg_fail(AMFRW_EINVAL, "surrogate is not trained");
    if (n < 16 || !(rel_bound > 0) || !(quantile > 0 && quantile <= 1))
        return sg_fail(AMFRW_EINVAL, "need n >= 16, rel_bound > 0, quantile in (0, 1]");
    std::vector<double> mean, spread;
    std::vector<char> ok;
    int st = sg_predict_host(s, ps, n, mean, spread, ok);
    if (st != AMFRW_OK) return st;
    std::vector<double> ratio;
    for (int64_t i = 0; i < n; ++i) {
        if (!ok[(size_t)i]) continue;
        const double e = std::fabs(mean[(size_t)i] - prices[i]);
        ratio.push_back(e / std::max(spread[(size_t)i], 1e-300));
    }
    if (ratio.size() < 16) return sg_fail(AMFRW_EINVAL, "too few audit instances inside the family");
    std::sort(ratio.begin(), ratio.end());
    const size_t k = std::min(ratio.size() - 1, (size_t)std::ceil(quantile * (double)ratio.size()) - 1);
    s->calib = ratio[k];
    s->rel_bound = rel_bound;
    s->calibrated = true;
    if (calib_out) *calib_out = s->calib;
    return AMFRW_OK;
}

int amfrw_surrogate_eval(amfrw_surrogate* s, const amfrw_params* ps, int64_t n, double* prices_out,
                         uint8_t* fell_back_out, void* cuda_stream)
{
    if (!s || !ps || !prices_out) return sg_fail(AMFRW_EINVAL, "NULL argument");
    if (!s->trained || !s->calibrated) return sg_fail(AMFRW_EINVAL, "surrogate is not trained and calibrated");
    std::vector<double> mean, spread;
    std::vector<char> ok;
    int st = sg_predict_host(s, ps, n, mean, spread, ok);
    if (st != AMFRW_OK) return st;
    return sg_serve(
        s, n, mean, spread, ok, [&](int64_t i, InstanceStore&) { return ps[i]; }, prices_out, fell_back_out,
        cuda_stream);
}

int amfrw_surrogate_eval_features(amfrw_surrogate* s, const double* features, int64_t n, double* prices_out,
                                  uint8_t* fell_back_out, void* cuda_stream)
{
    if (!s || !features || !prices_out) return sg_fail(AMFRW_EINVAL, "NULL argument");
    if (n < 0) return sg_fail(AMFRW_EINVAL, "n < 0");
    if (!s->trained || !s->calibrated) return sg_fail(AMFRW_EINVAL, "surrogate is not trained and calibrated");
    for (int64_t i = 0; i < n * kIn; ++i)
        if (!std::isfinite(features[i])) return sg_fail(AMFRW_EINVAL, "non-finite feature");
    std::vector<double> mean, spread;
    std::vector<char> ok((size_t)n, 1);
    int st = sg_predict_raw(s, features, n, mean, spread, ok);
    if (st != AMFRW_OK) return st;
    return sg_serve(
        s, n, mean, spread, ok,
        [&](int64_t i, InstanceStore& store) { return params_from(s->fam, features + (size_t)i * kIn, store); },
        prices_out, fell_back_out, cuda_stream);
}

int amfrw_surrogate_save(const amfrw_surrogate* s, const char* path)
{
    if (!s || !path) return sg_fail(AMFRW_EINVAL, "NULL argument");
    FILE* f = fopen(path, "wb");
    if (!f) return sg_fail(AMFRW_EINVAL, std::string("cannot open ") + path);
    const char magic[8] = {'A', 'M', 'F', 'R', 'W', 'S', 'G', '3'};
    std::vector<float> h(kParams);
    bool ok = fwrite(magic, 1, 8, f) == 8;
    ok = ok && fwrite(&s->members, sizeof(int), 1, f) == 1;
    ok = ok && fwrite(s->fmin, sizeof(double), kIn, f) == (size_t)kIn;
    ok = ok && fwrite(s->fmax, sizeof(double), kIn, f) == (size_t)kIn;
    const double sc[4] = {s->ymu, s->ysd, s->calib, s->rel_bound};
    ok = ok && fwrite(sc, sizeof(double), 4, f) == 4;
    const int flags[3] = {s->trained ? 1 : 0, s->calibrated ? 1 : 0, s->log_target ? 1 : 0};
    ok = ok && fwrite(flags, sizeof(int), 3, f) == 3;
    ok = ok && fwrite(&s->fam, sizeof(Family), 1, f) == 1;
    ok = ok && fwrite(s->poly, sizeof(double), kPolyTerms, f) == (size_t)kPolyTerms;
    ok = ok && fwrite(s->nlat, sizeof(int), kIn, f) == (size_t)kIn;
    ok = ok && fwrite(s->lat, sizeof(double), kIn * kMaxLattice, f) == (size_t)(kIn * kMaxLattice);
    for (int m = 0; m < s->members && ok; ++m) {
        ok = cudaMemcpy(h.data(), s->P[m], sizeof(float) * kParams, cudaMemcpyDeviceToHost) == cudaSuccess;
        ok = ok && fwrite(h.data(), sizeof(float), kParams, f) == (size_t)kParams;
    }
    fclose(f);
    return ok ? AMFRW_OK : sg_fail(AMFRW_ECUDA, "surrogate save failed");
}

int amfrw_surrogate_load(const char* path, void* cuda_stream, amfrw_surrogate** out)
{
    if (!path || !out) return sg_fail(AMFRW_EINVAL, "NULL argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return sg_fail(AMFRW_EINVAL, std::string("cannot open ") + path);
    char magic[8];
    int members = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "AMFRWSG3", 8) == 0;
    ok = ok && fread(&members, sizeof(int), 1, f) == 1 && members >= 1 && members <= 16;
    amfrw_surrogate* s = nullptr;
    if (ok && amfrw_surrogate_create(members, 0, cuda_stream, &s) != AMFRW_OK) ok = false;
    double sc[4];
    int flags[3];
    if (ok) {
        ok = fread(s->fmin, sizeof(double), kIn, f) == (size_t)kIn && fread(s->fmax, sizeof(double), kIn, f) == (size_t)kIn;
        ok = ok && fread(sc, sizeof(double), 4, f) == 4 && fread(flags, sizeof(int), 3, f) == 3;
        ok = ok && fread(&s->fam, sizeof(Family), 1, f) == 1;
        ok = ok && fread(s->poly, sizeof(double), kPolyTerms, f) == (size_t)kPolyTerms;
        ok = ok && fread(s->nlat, sizeof(int), kIn, f) == (size_t)kIn;
        ok = ok && fread(s->lat, sizeof(double), kIn * kMaxLattice, f) == (size_t)(kIn * kMaxLattice);
        for (int c = 0; c < kIn && ok; ++c) ok = s->nlat[c] >= 0 && s->nlat[c] <= kMaxLattice;
        ok = ok && cudaMemcpy(s->dpoly, s->poly, sizeof(double) * kPolyTerms, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    std::vector<float> h(kParams);
    for (int m = 0; ok && m < members; ++m) {
        ok = fread(h.data(), sizeof(float), kParams, f) == (size_t)kParams;
        ok = ok && cudaMemcpy(s->P[m], h.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice) == cudaSuccess;
        if (ok) sg_cast(s, m, s->stream);
    }
    fclose(f);
    if (!ok) {
        delete s;
        return sg_fail(AMFRW_EINVAL, std::string("not a surrogate file: ") + path);
    }
    s->ymu = sc[0]; s->ysd = sc[1]; s->calib = sc[2]; s->rel_bound = sc[3];
    s->trained = flags[0] != 0;
    s->calibrated = flags[1] != 0;
    s->log_target = flags[2] != 0;
    cudaStreamSynchronize(s->stream);
    *out = s;
    return AMFRW_OK;
}

// Parameters of one member (FP32, the layout described in include/amfrw.h)
// and the loss gradient of one packed batch, for gradient checks.
int amfrw_surrogate_params(amfrw_surrogate* s, int32_t member, float* params_out, const float* params_in)
{
    if (!s || member < 0 || member >= s->members) return sg_fail(AMFRW_EINVAL, "bad member");
    if (params_in) {
        SG_CUDA(cudaMemcpy(s->P[member], params_in, sizeof(float) * kParams, cudaMemcpyHostToDevice));
        sg_cast(s, member, s->stream);
        SG_CUDA(cudaStreamSynchronize(s->stream));
    }
    if (params_out) SG_CUDA(cudaMemcpy(params_out, s->P[member], sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    return AMFRW_OK;
}

int amfrw_surrogate_grad(amfrw_surrogate* s, int32_t member, const float* x_norm, const float* targets,
                         int32_t rows, float* grad_out, float* loss_out)
{
    if (!s || !x_norm || !targets || !grad_out || member < 0 || member >= s->members)
        return sg_fail(AMFRW_EINVAL, "bad argument");
    if (rows < 16 || rows > kTrainRows || rows % 16) return sg_fail(AMFRW_EINVAL, "rows must be a multiple of 16 in [16, 1024]");
    cudaStream_t st = s->stream;
    float *d_x = nullptr, *d_t = nullptr;
    SG_CUDA(cudaMalloc(&d_x, sizeof(float) * rows * kIn));
    SG_CUDA(cudaMalloc(&d_t, sizeof(float) * rows));
    cudaMemcpyAsync(d_x, x_norm, sizeof(float) * rows * kIn, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_t, targets, sizeof(float) * rows, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(s->w.loss, 0, sizeof(float), st);
    cudaMemsetAsync(s->G[member], 0, sizeof(float) * kParams, st);
    pack_kernel<<<cdiv(rows * kInPad, 256), 256, 0, st>>>(d_x, d_t, nullptr, 0, rows, s->w.X, s->w.Xt, s->w.t);
    int rc = sg_forward(s, member, rows, true, s->w.y, s->w);
    if (rc == AMFRW_OK) rc = sg_backward(s, member, rows, s->w);
    if (rc == AMFRW_OK) {
        cudaMemcpyAsync(grad_out, s->G[member], sizeof(float) * kParams, cudaMemcpyDeviceToHost, st);
        if (loss_out) cudaMemcpyAsync(loss_out, s->w.loss, sizeof(float), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
    }
    cudaFree(d_x);
    cudaFree(d_t);
    if (rc != AMFRW_OK) return rc;
    return sg_check_err(s);
}

void amfrw_surrogate_destroy(amfrw_surrogate* s) { delete s; }

}  // extern "C"
