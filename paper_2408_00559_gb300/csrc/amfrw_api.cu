// Host side of the C ABI declared in include/amfrw.h: parameter validation,
// component-grid enumeration, work partitioning, device buffers and launches.
// No arithmetic of the method runs here; it all runs in the kernels.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <cstdlib>
#include <string>
#include <tuple>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/amfrw.h"
#include "amfrw_internal.h"

using namespace amfrw;

namespace {

thread_local std::string g_last_error;

int fail(int status, const std::string& msg)
{
    g_last_error = msg;
    return status;
}

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(AMFRW_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr int kWarpMaxL = 64;          // grids up to this many Inner nodes: warp groups
// Default condition bound above which a mixed-precision instance is re-solved
// in FP64 (the mixed error measured relative to sum_l |c_l u_l| stays below
// about 3e-11, so kappa <= 1e5 keeps the relative price error below 1e-5).
constexpr double kKappaMaxDefault = 1e5;
constexpr int kWarpsPerBlock = 4;

// Warp groups have at least 4 lanes for FP64 (at most 8 grids per warp) and
// at least 8 for mixed precision, where smaller groups measured slower.
constexpr int kMinGroupLogF64 = 2;
constexpr int kMinGroupLogMixed = 3;

// Lanes (as log2) of the warp group that solves a grid of 2^llog Inner
// nodes: two nodes per lane (the most a lane's line-solve registers take), so
// that a line solve runs one PCR level fewer than with one node per lane and
// twice as many grids share a warp; at most 32 lanes.  Each PCR level costs
// two FP64 FMAs per row, which is what bounds the warp kernels, so the fewer
// levels outweigh the lower occupancy of the larger per-warp shared memory.
int warp_group_log(int llog, bool mixed)
{
    return std::max(std::min(llog - kRowsLogWarp, 5), mixed ? kMinGroupLogMixed : kMinGroupLogF64);
}

bool finite(double x) { return std::isfinite(x); }

// Smallest eigenvalue check of the joint correlation of (F_1..F_{N-1}, V) by a
// Cholesky factorisation with a small tolerance (PSD, not only PD).
bool joint_correlation_psd(int nr, const double* rho, const double* phi)
{
    const int n = nr + 1;
    std::vector<double> A(n * n), Lc(n * n, 0.0);
    for (int i = 0; i < nr; ++i)
        for (int k = 0; k < nr; ++k) A[i * n + k] = rho[i * nr + k];
    for (int i = 0; i < nr; ++i) {
        A[i * n + nr] = phi[i];
        A[nr * n + i] = phi[i];
    }
    A[nr * n + nr] = 1.0;
    const double tol = 1e-10;
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= Lc[j * n + k] * Lc[j * n + k];
        if (d < -tol) return false;
        const double ljj = d > 0.0 ? std::sqrt(d) : 0.0;
        Lc[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double v = A[i * n + j];
            for (int k = 0; k < j; ++k) v -= Lc[i * n + k] * Lc[j * n + k];
            if (ljj > 0.0) {
                Lc[i * n + j] = v / ljj;
            } else if (std::fabs(v) > tol) {
                return false;  // zero pivot with a non-zero remainder: not PSD
            }
        }
    }
    return true;
}

int validate(const amfrw_params* p)
{
    if (!p) return fail(AMFRW_EINVAL, "params is NULL");
    const int nr = p->n_rates;
    if (nr < 1 || nr > kMaxDim - 1) return fail(AMFRW_EINVAL, "n_rates must be in [1, 7]");
    if (!p->alpha || !p->phi || !p->rho || !p->tau || !p->F0 || !p->Fmax)
        return fail(AMFRW_EINVAL, "a parameter array is NULL");
    if (p->payoff != AMFRW_CAPLET && p->payoff != AMFRW_SWAPTION)
        return fail(AMFRW_EINVAL, "unknown payoff");
    if (p->precision != AMFRW_FP64 && p->precision != AMFRW_MIXED)
        return fail(AMFRW_EINVAL, "unknown precision");
    if (p->n_steps < 1) return fail(AMFRW_EINVAL, "n_steps must be >= 1");
    if (p->flags & ~(AMFRW_FLAG_GLOBAL_GRIDS | AMFRW_FLAG_DIRICHLET)) return fail(AMFRW_EINVAL, "unknown flag bits");
    if (p->level < 0 || p->psi < 0) return fail(AMFRW_EINVAL, "level and psi must be >= 0");
    const double sc[] = {p->sigma, p->beta, p->V0, p->Vmax, p->K, p->T, p->discount, p->theta, p->nu_amf};
    for (double v : sc)
        if (!finite(v)) return fail(AMFRW_EINVAL, "a scalar parameter is not finite");
    if (p->sigma < 0.0) return fail(AMFRW_EINVAL, "sigma must be >= 0");
    if (p->beta < 0.0 || p->beta > 1.0) return fail(AMFRW_EINVAL, "beta must be in [0, 1]");
    if (!(p->Vmax > 0.0) || p->V0 < 0.0 || p->V0 > p->Vmax)
        return fail(AMFRW_EINVAL, "need 0 <= V0 <= Vmax and Vmax > 0");
    if (!(p->T > 0.0)) return fail(AMFRW_EINVAL, "T must be > 0");
    if (!(p->theta > 0.0) || !(p->nu_amf > 0.0)) return fail(AMFRW_EINVAL, "theta and nu_amf must be > 0");
    for (int i = 0; i < nr; ++i) {
        if (!finite(p->alpha[i]) || !finite(p->phi[i]) || !finite(p->tau[i]) || !finite(p->F0[i]) ||
            !finite(p->Fmax[i]))
            return fail(AMFRW_EINVAL, "a per-rate parameter is not finite");
        if (p->alpha[i] < 0.0) return fail(AMFRW_EINVAL, "alpha_i must be >= 0");
        if (!(p->tau[i] > 0.0)) return fail(AMFRW_EINVAL, "tau_i must be > 0");
        if (!(p->Fmax[i] > 0.0) || p->F0[i] < 0.0 || p->F0[i] > p->Fmax[i])
            return fail(AMFRW_EINVAL, "need 0 <= F0_i <= Fmax_i and Fmax_i > 0");
        if (p->phi[i] < -1.0 || p->phi[i] > 1.0) return fail(AMFRW_EINVAL, "phi_i must be in [-1, 1]");
        for (int k = 0; k < nr; ++k) {
            const double r = p->rho[i * nr + k];
            if (!finite(r)) return fail(AMFRW_EINVAL, "rho is not finite");
            if (std::fabs(r - p->rho[k * nr + i]) > 1e-12) return fail(AMFRW_EINVAL, "rho is not symmetric");
        }
        if (std::fabs(p->rho[i * nr + i] - 1.0) > 1e-12) return fail(AMFRW_EINVAL, "rho must have a unit diagonal");
    }
    if (!joint_correlation_psd(nr, p->rho, p->phi))
        return fail(AMFRW_ENOTPSD, "correlation of (F_1..F_{N-1}, V) is not positive semi-definite");
    return AMFRW_OK;
}

struct GridSpec {
    int8_t lv[kMaxDim];
    double coef;
};

// Component grids of the combination technique: every composition l of
// n - q into d non-negative parts for q = 0..d-1, coefficient (-1)^q C(d-1,q),
// levels psi + l_i; or the single full grid.  Order: q ascending, then the
// compositions with the last axis varying slowest.
void compositions(int d, int m, int axis, int8_t* cur, int psi, double coef, std::vector<GridSpec>& out)
{
    if (axis == d - 1) {
        cur[axis] = (int8_t)(psi + m);
        GridSpec g{};
        memcpy(g.lv, cur, sizeof(g.lv));
        g.coef = coef;
        out.push_back(g);
        return;
    }
    for (int v = 0; v <= m; ++v) {
        cur[axis] = (int8_t)(psi + v);
        compositions(d, m - v, axis + 1, cur, psi, coef, out);
    }
}

std::vector<GridSpec> enumerate(int d, int n, int psi, bool full)
{
    std::vector<GridSpec> out;
    if (full) {
        GridSpec g{};
        for (int i = 0; i < d; ++i) g.lv[i] = (int8_t)n;
        g.coef = 1.0;
        out.push_back(g);
        return out;
    }
    int8_t cur[kMaxDim] = {0};
    double binom = 1.0;  // C(d-1, q)
    for (int q = 0; q < d; ++q) {
        if (q > 0) binom = binom * (double)(d - q) / (double)q;
        if (n - q < 0) break;
        compositions(d, n - q, 0, cur, psi, (q & 1 ? -1.0 : 1.0) * binom, out);
    }
    return out;
}

InstDev to_device(const amfrw_params* p)
{
    InstDev I;
    memset(&I, 0, sizeof(I));
    const int nr = p->n_rates;
    I.N = nr + 1;
    I.payoff = p->payoff;
    I.n_steps = p->n_steps;
    I.precision = p->precision;
    I.bc = (p->flags & AMFRW_FLAG_DIRICHLET) ? 1 : 0;
    for (int i = 0; i < nr; ++i) {
        I.alpha[i] = p->alpha[i];
        I.phi[i] = p->phi[i];
        I.tau[i] = p->tau[i];
        I.F0[i] = p->F0[i];
        I.Fmax[i] = p->Fmax[i];
        for (int k = 0; k < nr; ++k) I.rho[i * kMaxDim + k] = p->rho[i * nr + k];
    }
    I.Fmax[nr] = p->Vmax;
    I.sigma = p->sigma;
    I.beta = p->beta;
    I.V0 = p->V0;
    I.K = p->K;
    I.T = p->T;
    I.discount = p->discount;
    I.theta = p->theta;
    I.nu = p->nu_amf;
    I.dt = p->T / (double)p->n_steps;
    // level-free constant factors, in the operation order of the kernels'
    // per-grid formulas with h replaced by Fmax (products by powers of two
    // are exact, so the scaled values equal the direct ones bit for bit)
    const int N = I.N;
    const double Vm = I.Fmax[N - 1];
    I.cVb = 0.5 * I.sigma * I.sigma / (Vm * Vm);
    for (int i = 0; i < N - 1; ++i) {
        const double Fm = I.Fmax[i];
        I.dcb[i] = 0.5 * I.alpha[i] * I.alpha[i] * I.rho[i * kMaxDim + i] / (Fm * Fm);
        I.smb[i] = I.sigma * I.phi[i] / (4.0 * Fm * Vm);
        for (int k = i + 1; k < N - 1; ++k)
            I.rmb[upair(i, k)] = I.rho[i * kMaxDim + k] / (4.0 * Fm * I.Fmax[k]);
    }
    for (int i = 0; i < N; ++i) {
        I.g2b[i] = 1.0 / (2.0 * I.Fmax[i]);
        I.xs[i] = ((i < N - 1) ? I.F0[i] : I.V0) / I.Fmax[i];
    }
    return I;
}

LaunchFn launch_for(int N)
{
    static const LaunchFn t[] = {nullptr, nullptr, launch_n2, launch_n3, launch_n4,
                                 launch_n5, launch_n6, launch_n7, launch_n8};
    return t[N];
}
OccFn occ_for(int N)
{
    static const OccFn t[] = {nullptr, nullptr, occupancy_n2, occupancy_n3, occupancy_n4,
                              occupancy_n5, occupancy_n6, occupancy_n7, occupancy_n8};
    return t[N];
}

int max_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v > 0 ? v : 232448;
}
int num_sms()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

// One launch: all grids of one (N, precision, group kind).
struct LaunchClass {
    int N;
    bool mixed, warp;
    int kind;            // kWarpGroup, kCtaGroup or kMemGroup
    int item_begin, item_count;
    int block, grid;
    size_t smem;
    int smem_group;
    int glog;            // warp groups: log2 lanes per group
    int64_t lu_stride;   // bytes of scratch per block: Thomas factors (CTA
                         // groups) or the whole grid state (global-memory groups)
    int64_t lu_offset;   // this class's part of the plan's scratch array
};

// Global-memory groups: at most this much scratch per launch class (it bounds
// the number of resident blocks, each holding one grid's state).
constexpr int64_t kMemScratchBudget = int64_t(8) << 30;
constexpr int kMemBlock = 256;

struct Plan {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_inst = 0, n_grids = 0, dim = 0;
    std::vector<InstDev> insts;
    std::vector<Item> items;          // grouped by launch class, largest grids first
    std::vector<double> coefs;        // per grid, instance order
    std::vector<int8_t> levels;       // per grid (dim = 8 each), instance order
    std::vector<LaunchClass> classes;
    // device
    InstDev* d_insts = nullptr;
    Item* d_items = nullptr;
    double* d_coefs = nullptr;
    double* d_u = nullptr;
    double* d_prices = nullptr;
    int32_t* d_queue = nullptr;
    int32_t* d_flag = nullptr;
    double* d_state = nullptr;
    int64_t state_len = 0;
    unsigned char* d_lu = nullptr;   // scratch: Thomas factors of CTA-group grids
    int64_t lu_scratch_len = 0;
    // warp-group launches: with the merged strategy one persistent launch per
    // (N, precision) walks all its grid classes; split: one launch per class
    struct WarpLaunch {
        int N = 0;
        bool mixed = false;
        std::vector<ClassDesc> cls;
        std::vector<int> covers;  // indices into `classes`
        int block = 128, grid = 1, smem_warp = 0;
        size_t smem = 0;
        int64_t desc_offset = 0;  // into d_cdesc
    };
    std::vector<WarpLaunch> wl;
    ClassDesc* d_cdesc = nullptr;
    int64_t n_cdesc = 0;
    bool use_multi = true;  // launch strategy (the autotuner may switch it)
    int glog_delta = 0;     // warp groups: lanes per grid widened by 2^glog_delta (autotuned)
    bool shared_u = false;  // d_u belongs to another plan (the FP64 re-solve writes there)
    const int32_t* inst_mask = nullptr;  // instances to solve, or null for all

    ~Plan() { release(); }
    void release()
    {
        cudaFree(d_insts);
        cudaFree(d_items);
        cudaFree(d_coefs);
        if (!shared_u) cudaFree(d_u);
        cudaFree(d_prices);
        cudaFree(d_queue);
        cudaFree(d_flag);
        cudaFree(d_state);
        cudaFree(d_lu);
        cudaFree(d_cdesc);
        d_lu = nullptr;
        d_cdesc = nullptr;
        d_insts = nullptr; d_items = nullptr; d_coefs = nullptr; d_u = nullptr;
        d_prices = nullptr; d_queue = nullptr; d_flag = nullptr; d_state = nullptr;
    }
};

int log2i(int v)
{
    int r = 0;
    while ((1 << (r + 1)) <= v) ++r;
    return r;
}

// Host-side plan: validated instances, grid list grouped into launch classes
// (largest grids first), launch shapes and the size of the line-solve scratch.
// No device memory is touched.
int plan_host(const amfrw_params* ps, int n, bool keep_state, Plan& P)
{
    if (n < 1) return fail(AMFRW_EINVAL, "need at least one instance");
    if (!ps) return fail(AMFRW_EINVAL, "params is NULL");
    // every instance is validated before any CUDA call
    for (int i = 0; i < n; ++i) {
        int st = validate(ps + i);
        if (st != AMFRW_OK) {
            g_last_error = "instance " + std::to_string(i) + ": " + g_last_error;
            return st;
        }
    }
    P.n_inst = n;
    const int smem_cap = max_smem_optin();
    // The grids of one instance shape (N, level, psi, full grid, precision,
    // flags) with their work-group kind and layout size, shared by every
    // instance of that shape.
    struct GridInfo { GridSpec g; int L; int kind; bool warp; int smem_group; int rank; };
    using ShapeId = std::tuple<int, int, int, int, int, int>;
    std::map<ShapeId, std::vector<GridInfo>> shapes;
    std::vector<std::vector<GridInfo>*> inst_shape((size_t)n);
    for (int i = 0; i < n; ++i) {
        const amfrw_params* p = ps + i;
        const int N = p->n_rates + 1;
        const bool mixed = p->precision == AMFRW_MIXED;
        const bool force_mem = (p->flags & AMFRW_FLAG_GLOBAL_GRIDS) != 0;
        const ShapeId id{N, p->level, p->psi, p->full_grid != 0, mixed, force_mem};
        auto it = shapes.find(id);
        if (it == shapes.end()) {
            std::vector<GridInfo> gi;
            for (const GridSpec& g : enumerate(N, p->level, p->psi, p->full_grid != 0)) {
                int llog = 0, maxlv = 0;
                for (int a = 0; a < N; ++a) {
                    llog += g.lv[a];
                    maxlv = std::max(maxlv, (int)g.lv[a]);
                }
                if (llog > 22)
                    return fail(AMFRW_ETOOBIG, "instance " + std::to_string(i) +
                                                   ": a component grid has more than 2^22 Inner nodes");
                const bool warp = (1 << llog) <= kWarpMaxL && !force_mem;
                // warp groups: two nodes per lane, so small grids share a warp
                int kind = warp ? kWarpGroup : kCtaGroup;
                Layout lay = make_layout(N, g.lv, mixed, kind,
                                         warp ? warp_group_log(llog, mixed) : 5);
                // grids beyond shared memory, or with lines longer than the register
                // sweeps take, keep their state in global memory
                if (force_mem || lay.total > smem_cap || (!warp && maxlv > 5 + rows_log(kCtaGroup, mixed))) {
                    kind = kMemGroup;
                    lay = make_layout(N, g.lv, mixed, kind, log2i(kMemBlock));
                }
                gi.push_back(GridInfo{g, lay.L, kind, warp, lay.total, 0});
            }
            it = shapes.emplace(id, std::move(gi)).first;
        }
        inst_shape[(size_t)i] = &it->second;
    }
    // classes: (N, precision, group kind) and, for warp groups, the grid size;
    // inside a class the largest grids first, equal shapes adjacent and, for
    // equal shapes, instance order.  Rank the distinct grid shapes once, then
    // place the grids by a counting sort over the ranks.
    struct Key { int N; bool mixed; int kind; int wl; int L; int8_t lv[kMaxDim]; };
    auto key_less = [](const Key& a, const Key& b) {
        const auto ta = std::make_tuple(a.N, a.mixed, a.kind, -a.wl, -a.L);
        const auto tb = std::make_tuple(b.N, b.mixed, b.kind, -b.wl, -b.L);
        if (ta != tb) return ta < tb;
        return memcmp(a.lv, b.lv, sizeof(a.lv)) < 0;
    };
    std::vector<std::pair<Key, GridInfo*>> keys;
    for (auto& kv : shapes) {
        const int N = std::get<0>(kv.first);
        const bool mixed = std::get<4>(kv.first) != 0;
        for (GridInfo& gi : kv.second) {
            Key k{};
            k.N = N;
            k.mixed = mixed;
            k.kind = gi.kind;
            k.wl = gi.warp ? gi.L : 0;
            k.L = gi.L;
            memcpy(k.lv, gi.g.lv, sizeof(k.lv));
            keys.push_back({k, &gi});
        }
    }
    std::sort(keys.begin(), keys.end(),
              [&](const std::pair<Key, GridInfo*>& a, const std::pair<Key, GridInfo*>& b) { return key_less(a.first, b.first); });
    int nrank = 0;
    for (size_t q = 0; q < keys.size(); ++q) {
        if (q > 0 && key_less(keys[q - 1].first, keys[q].first)) ++nrank;
        keys[q].second->rank = nrank;
    }
    ++nrank;
    struct Tmp { Item it; int L; int N; bool mixed; bool warp; int kind; int smem_group; };
    std::vector<int64_t> start((size_t)nrank + 1, 0);
    for (int i = 0; i < n; ++i)
        for (const GridInfo& gi : *inst_shape[(size_t)i]) ++start[(size_t)gi.rank + 1];
    for (int r = 0; r < nrank; ++r) start[(size_t)r + 1] += start[(size_t)r];
    std::vector<Tmp> all((size_t)start[(size_t)nrank]);
    int64_t state_off = 0;
    for (int i = 0; i < n; ++i) {
        const amfrw_params* p = ps + i;
        InstDev I = to_device(p);
        const int N = I.N;
        const bool mixed = p->precision == AMFRW_MIXED;
        const std::vector<GridInfo>& grids = *inst_shape[(size_t)i];
        I.grid_begin = (int32_t)P.coefs.size();
        I.grid_count = (int32_t)grids.size();
        for (const GridInfo& gi : grids) {
            Tmp t{};
            t.it.inst = i;
            t.it.out_idx = (int32_t)P.coefs.size();
            t.it.L = gi.L;
            memcpy(t.it.lv, gi.g.lv, sizeof(t.it.lv));
            t.it.state_off = keep_state ? state_off : -1;
            if (keep_state) state_off += gi.L;
            t.L = gi.L;
            t.N = N;
            t.mixed = mixed;
            t.warp = gi.warp;
            t.kind = gi.kind;
            t.smem_group = gi.smem_group;
            all[(size_t)start[(size_t)gi.rank]++] = t;
            P.coefs.push_back(gi.g.coef);
            for (int a = 0; a < kMaxDim; ++a) P.levels.push_back(a < N ? gi.g.lv[a] : 0);
        }
        P.insts.push_back(I);
        P.dim = N;
    }
    P.n_grids = (int)P.coefs.size();
    P.state_len = state_off;
    const int sms = num_sms();
    for (size_t k = 0; k < all.size();) {
        size_t e = k;
        int gmax = 0, lmax = 0;
        while (e < all.size() && all[e].N == all[k].N && all[e].mixed == all[k].mixed &&
               all[e].kind == all[k].kind && (!all[k].warp || all[e].L == all[k].L)) {
            gmax = std::max(gmax, all[e].smem_group);
            lmax = std::max(lmax, all[e].L);
            ++e;
        }
        LaunchClass c{};
        c.N = all[k].N;
        c.mixed = all[k].mixed;
        c.warp = all[k].warp;
        c.kind = all[k].kind;
        c.item_begin = (int)P.items.size();
        c.item_count = (int)(e - k);
        c.smem_group = gmax;
        int64_t lumax = 0;
        if (c.warp) {
            c.glog = warp_group_log(log2i(lmax), c.mixed);
            const int gpw = 32 >> c.glog;  // groups per warp
            int wpb = std::min(kWarpsPerBlock, std::max(1, smem_cap / (gmax * gpw)));
            if ((size_t)gmax * gpw > (size_t)smem_cap)
                return fail(AMFRW_ETOOBIG, "warp groups of a launch class do not fit in shared memory");
            c.block = 32 * wpb;
            c.smem = (size_t)gmax * gpw * wpb;
        } else if (c.kind == kCtaGroup) {
            int b = 64;
            while (b < kCtaMaxThreads && b * 8 < lmax) b *= 2;
            c.block = b;
            c.smem = (size_t)gmax;
            for (size_t q = k; q < e; ++q) {
                Layout lay = make_layout(c.N, all[q].it.lv, c.mixed, kCtaGroup, log2i(b));
                lumax = std::max<int64_t>(lumax, (int64_t)lay.gbytes);
            }
        } else {  // global-memory groups: each block's slice holds a whole grid state
            c.block = kMemBlock;
            c.smem = 0;
            lumax = gmax;
        }
        const int per_sm = occ_for(c.N)(c.mixed, c.kind, c.block, c.smem);
        if (per_sm < 1)
            return fail(AMFRW_ETOOBIG, "no resident block possible for a launch class (shared memory " +
                                           std::to_string(c.smem) + " bytes)");
        const int groups_per_block = c.warp ? (c.block >> c.glog) : 1;
        const int need = (c.item_count + groups_per_block - 1) / groups_per_block;
        c.grid = std::max(1, std::min(need, per_sm * sms));
        c.lu_stride = (lumax + 255) & ~(int64_t)255;
        if (c.kind == kMemGroup && c.lu_stride > 0)
            c.grid = (int)std::max<int64_t>(1, std::min<int64_t>(c.grid, kMemScratchBudget / c.lu_stride));
        c.lu_offset = P.lu_scratch_len;
        P.lu_scratch_len += c.lu_stride * c.grid;
        for (size_t q = k; q < e; ++q) P.items.push_back(all[q].it);
        P.classes.push_back(c);
        k = e;
    }
    return AMFRW_OK;
}

// Warp-group launches for the current strategy.  Merged: per (N, precision)
// one launch over all its classes, largest grids first.  Split: one launch
// per class.  Descriptors are laid out in launch order.
int build_warp_launches(Plan& P)
{
    P.wl.clear();
    const int smem_cap = max_smem_optin();
    const int sms = num_sms();
    std::vector<std::vector<int>> groups;
    for (int N = 2; N <= kMaxDim; ++N) {
        for (int mixed = 0; mixed < 2; ++mixed) {
            std::vector<int> cs;
            for (size_t c = 0; c < P.classes.size(); ++c)
                if (P.classes[c].warp && P.classes[c].N == N && (int)P.classes[c].mixed == mixed)
                    cs.push_back((int)c);
            if (cs.empty()) continue;
            std::sort(cs.begin(), cs.end(), [&](int x, int y) {
                return P.items[P.classes[x].item_begin].L > P.items[P.classes[y].item_begin].L;
            });
            if (P.use_multi) {
                groups.push_back(cs);
            } else {
                for (int c : cs) groups.push_back({c});
            }
        }
    }
    int64_t off = 0;
    int smem_sm = 0, reserved = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    for (const std::vector<int>& g : groups) {
        Plan::WarpLaunch w;
        w.N = P.classes[g[0]].N;
        w.mixed = P.classes[g[0]].mixed;
        w.covers = g;
        // A multi-class launch sizes every warp's shared memory for its most
        // demanding class.  So that this does not cost residency, a class
        // whose groups of one warp need more than the share of an SM that
        // the register-limited number of warps leaves each warp gets fewer,
        // wider groups (more lanes per grid).
        int budget = 1 << 30;
        if (g.size() > 1 && smem_sm > 0) {
            const int blocks = occ_for(w.N)(w.mixed, kWarpGroup, 32 * kWarpsPerBlock, 0);
            if (blocks > 0)
                budget = (smem_sm - blocks * reserved) / (blocks * kWarpsPerBlock);
        }
        int items = 0;
        for (int c : g) {
            const LaunchClass& L = P.classes[c];
            ClassDesc d{};
            d.glog = L.glog;
            d.item_begin = L.item_begin;
            d.item_count = L.item_count;
            d.qidx = c;
            // the group's shared memory for a width of 2^g lanes, padded so
            // that the groups sharing a warp start 128 / (groups per warp)
            // bytes apart modulo 128: their lanes, which touch nearby words of
            // their own grids, then fall into different banks
            auto group_smem = [&](int g) {
                int sg = 0;
                for (int q = L.item_begin; q < L.item_begin + L.item_count; ++q) {
                    if (q > L.item_begin && memcmp(P.items[q].lv, P.items[q - 1].lv, sizeof(P.items[q].lv)) == 0)
                        continue;  // equal shapes are adjacent
                    sg = std::max(sg, make_layout(L.N, P.items[q].lv, L.mixed, kWarpGroup, g).total);
                }
                const int gpw = 32 >> g;
                if (gpw > 1) sg += ((128 / gpw) - sg % 128 + 128) % 128;
                return sg;
            };
            // the tuned width: more lanes per grid, so more lanes per line (one
            // more PCR level, fewer Thomas rows) and fewer nodes per lane
            d.glog = std::min(5, d.glog + P.glog_delta);
            d.smem_group = group_smem(d.glog);
            while (d.glog < 5 && ((int64_t)d.smem_group << (5 - d.glog)) > budget) {
                ++d.glog;
                d.smem_group = group_smem(d.glog);
            }
            w.cls.push_back(d);
            w.smem_warp = std::max(w.smem_warp, d.smem_group << (5 - d.glog));
            items += d.item_count << d.glog;  // lanes of work
        }
        if (w.smem_warp > smem_cap)
            return fail(AMFRW_ETOOBIG, "the work groups of one warp do not fit in shared memory");
        const int wpb = std::min(kWarpsPerBlock, std::max(1, smem_cap / w.smem_warp));
        w.block = 32 * wpb;
        w.smem = (size_t)w.smem_warp * wpb;
        const int per_sm = occ_for(w.N)(w.mixed, kWarpGroup, w.block, w.smem);
        if (per_sm < 1) return fail(AMFRW_ETOOBIG, "no resident block possible for a warp-group launch");
        const int need = (items + w.block - 1) / w.block;
        w.grid = std::max(1, std::min(need, per_sm * sms));
        w.desc_offset = off;
        off += (int64_t)w.cls.size();
        P.wl.push_back(w);
    }
    P.n_cdesc = off;
    return AMFRW_OK;
}

int upload_warp_launches(Plan& P)
{
    if (P.n_cdesc == 0) return AMFRW_OK;
    std::vector<ClassDesc> all;
    for (const Plan::WarpLaunch& w : P.wl) all.insert(all.end(), w.cls.begin(), w.cls.end());
    if (!P.d_cdesc) CUDA_TRY(cudaMalloc(&P.d_cdesc, sizeof(ClassDesc) * all.size()));
    CUDA_TRY(cudaMemcpyAsync(P.d_cdesc, all.data(), sizeof(ClassDesc) * all.size(),
                             cudaMemcpyHostToDevice, P.stream));
    // the upload must complete before `all` goes away
    CUDA_TRY(cudaStreamSynchronize(P.stream));
    return AMFRW_OK;
}

int build_plan(const amfrw_params* ps, int n, void* stream, bool keep_state, Plan& P)
{
    int st = plan_host(ps, n, keep_state, P);
    if (st != AMFRW_OK) return st;
    CUDA_TRY(cudaGetDevice(&P.device));
    P.stream = (cudaStream_t)stream;
    // device buffers
    CUDA_TRY(cudaMalloc(&P.d_insts, sizeof(InstDev) * P.insts.size()));
    CUDA_TRY(cudaMalloc(&P.d_items, sizeof(Item) * P.items.size()));
    CUDA_TRY(cudaMalloc(&P.d_coefs, sizeof(double) * P.coefs.size()));
    CUDA_TRY(cudaMalloc(&P.d_u, sizeof(double) * P.coefs.size()));
    CUDA_TRY(cudaMalloc(&P.d_prices, sizeof(double) * P.n_inst));
    CUDA_TRY(cudaMalloc(&P.d_queue, sizeof(int32_t) * std::max<size_t>(1, P.classes.size())));
    CUDA_TRY(cudaMalloc(&P.d_flag, sizeof(int32_t)));
    if (keep_state) CUDA_TRY(cudaMalloc(&P.d_state, sizeof(double) * std::max<int64_t>(1, P.state_len)));
    if (P.lu_scratch_len > 0) CUDA_TRY(cudaMalloc(&P.d_lu, (size_t)P.lu_scratch_len));
    int st2 = build_warp_launches(P);
    if (st2 != AMFRW_OK) return st2;
    st2 = upload_warp_launches(P);
    if (st2 != AMFRW_OK) return st2;
    CUDA_TRY(cudaMemcpyAsync(P.d_insts, P.insts.data(), sizeof(InstDev) * P.insts.size(),
                             cudaMemcpyHostToDevice, P.stream));
    CUDA_TRY(cudaMemcpyAsync(P.d_items, P.items.data(), sizeof(Item) * P.items.size(),
                             cudaMemcpyHostToDevice, P.stream));
    CUDA_TRY(cudaMemcpyAsync(P.d_coefs, P.coefs.data(), sizeof(double) * P.coefs.size(),
                             cudaMemcpyHostToDevice, P.stream));
    CUDA_TRY(cudaMemsetAsync(P.d_u, 0, sizeof(double) * P.coefs.size(), P.stream));
    return AMFRW_OK;
}

// Promotion of ill-conditioned mixed-precision instances.  The error of a
// mixed-precision price is a small multiple of the combination's scale
// sum_l |c_l u_l| (the FP32 increments perturb every u_l relative to its own
// size), so where the sum cancels -- kappa = sum_l |c_l u_l| / |sum_l c_l u_l|
// above kappa_max -- the relative error of the price is not bounded by that
// of the grid values.  Those instances are marked and re-solved in FP64 by a
// conditional body of the batch's graph, which runs only when one is marked.
struct Promote {
    double kappa_max;
    int32_t* mask = nullptr;    // [n] 1: re-solve in FP64
    double* kappa = nullptr;    // [n] kappa of the last mixed solve
    int32_t* count = nullptr;   // instances marked
    unsigned* done = nullptr;   // blocks finished (the last one sets the conditional)
    cudaGraphConditionalHandle cond = 0;
};

// price = discount * sum_l c_l u_l in FP64, grids in a fixed order
// (eqs. standardCombTechnique / modifiedCombTechnique).  only != null: the
// marked instances alone (after their FP64 re-solve).
__global__ void combine_kernel(const InstDev* __restrict__ insts, int n, const double* __restrict__ coefs,
                               const double* __restrict__ u, double* __restrict__ prices,
                               int32_t* __restrict__ nonfinite, Promote pr, const int32_t* __restrict__ only)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (!only || only[i])) {
        const InstDev& I = insts[i];
        double s = 0.0, sc = 0.0;
        for (int k = I.grid_begin; k < I.grid_begin + I.grid_count; ++k) {
            s = fma(coefs[k], u[k], s);
            sc += fabs(coefs[k] * u[k]);
        }
        const double p = I.discount * s;
        prices[i] = p;
        if (!isfinite(p)) atomicOr(nonfinite, 1);
        if (pr.mask) {
            const double kappa = sc / fabs(s);
            pr.kappa[i] = kappa;
            const bool bad = I.precision == AMFRW_MIXED && !(kappa <= pr.kappa_max);
            pr.mask[i] = bad ? 1 : 0;
            if (bad) atomicAdd(pr.count, 1);
        }
    }
    if (pr.cond) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(pr.done, 1u) == gridDim.x - 1) {
                __threadfence();
                cudaGraphSetConditional(pr.cond, atomicAdd(pr.count, 0) > 0 ? 1u : 0u);
            }
        }
    }
}

// Solve launches for every class.  steps < 0: each instance's own n_steps.
SolveArgs class_args(const Plan& P, const LaunchClass& L, int c, int steps, int flags)
{
    SolveArgs a{};
    a.items = P.d_items + L.item_begin;
    a.n_items = L.item_count;
    a.steps = steps;
    a.flags = flags;
    a.smem_group = L.smem_group;
    a.insts = P.d_insts;
    a.u_out = P.d_u;
    a.state = P.d_state;
    a.queue = P.d_queue + c;
    a.lu_scratch = P.d_lu ? P.d_lu + L.lu_offset : nullptr;
    a.lu_stride = L.lu_stride;
    a.inst_mask = P.inst_mask;
    return a;
}

// The launches of one solve, in order: the warp-group launches, then the CTA
// classes.  Each record is (warp launch index or -1, class index or -1).
std::vector<std::pair<int, int>> launch_records(const Plan& P)
{
    std::vector<std::pair<int, int>> r;
    for (size_t w = 0; w < P.wl.size(); ++w) r.push_back({(int)w, -1});
    for (size_t c = 0; c < P.classes.size(); ++c)
        if (!P.classes[c].warp) r.push_back({-1, (int)c});
    return r;
}

int run_solve(Plan& P, int steps, int flags, cudaEvent_t* ev = nullptr)
{
    CUDA_TRY(cudaMemsetAsync(P.d_queue, 0, sizeof(int32_t) * P.classes.size(), P.stream));
    const std::vector<std::pair<int, int>> recs = launch_records(P);
    // inside a graph capture the records are external, so that they also
    // record when the graph is replayed; outside they are plain records
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (ev) CUDA_TRY(cudaStreamIsCapturing(P.stream, &cap));
    const unsigned rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    for (size_t r = 0; r < recs.size(); ++r) {
        int rc = 0;
        if (ev) CUDA_TRY(cudaEventRecordWithFlags(ev[2 * r], P.stream, rec_flags));
        if (recs[r].first >= 0) {
            const Plan::WarpLaunch& w = P.wl[recs[r].first];
            SolveArgs a = class_args(P, P.classes[w.covers[0]], 0, steps, flags);
            a.items = P.d_items;
            a.queue = P.d_queue;
            a.classes = P.d_cdesc + w.desc_offset;
            a.n_classes = (int32_t)w.cls.size();
            a.smem_warp = w.smem_warp;
            rc = launch_for(w.N)(a, w.mixed, kWarpGroup, w.block, w.grid, w.smem, P.stream);
        } else {
            const int c = recs[r].second;
            const LaunchClass& L = P.classes[c];
            rc = launch_for(L.N)(class_args(P, L, c, steps, flags), L.mixed, L.kind, L.block, L.grid,
                                 L.smem, P.stream);
        }
        if (ev) CUDA_TRY(cudaEventRecordWithFlags(ev[2 * r + 1], P.stream, rec_flags));
        if (rc != 0) return fail(AMFRW_ECUDA, std::string("solver launch: ") + cudaGetErrorString((cudaError_t)rc));
    }
    return AMFRW_OK;
}

int run_combine(Plan& P, double* d_out, const Promote* pr = nullptr, const int32_t* only = nullptr)
{
    if (!only) CUDA_TRY(cudaMemsetAsync(P.d_flag, 0, sizeof(int32_t), P.stream));
    Promote none{};
    if (pr && pr->mask) {
        CUDA_TRY(cudaMemsetAsync(pr->count, 0, sizeof(int32_t), P.stream));
        CUDA_TRY(cudaMemsetAsync(pr->done, 0, sizeof(unsigned), P.stream));
    }
    const int b = 128;
    combine_kernel<<<(P.n_inst + b - 1) / b, b, 0, P.stream>>>(P.d_insts, P.n_inst, P.d_coefs, P.d_u,
                                                               d_out, P.d_flag, pr ? *pr : none, only);
    CUDA_TRY(cudaGetLastError());
    return AMFRW_OK;
}

// Move CTA class c (grids in shared memory) to a global-memory class: same
// grids, each block's state in its slice of the plan's scratch array.
int class_to_global(Plan& P, int c)
{
    LaunchClass& L = P.classes[(size_t)c];
    if (L.kind != kCtaGroup) return AMFRW_OK;
    int64_t lumax = 0;
    for (int q = L.item_begin; q < L.item_begin + L.item_count; ++q) {
        const Layout lay = make_layout(L.N, P.items[(size_t)q].lv, L.mixed, kMemGroup, log2i(kMemBlock));
        lumax = std::max<int64_t>(lumax, lay.total);
    }
    const int per_sm = occ_for(L.N)(L.mixed, kMemGroup, kMemBlock, 0);
    if (per_sm < 1) return fail(AMFRW_ETOOBIG, "no resident block possible for a global-memory class");
    L.kind = kMemGroup;
    L.block = kMemBlock;
    L.smem = 0;
    L.lu_stride = (lumax + 255) & ~(int64_t)255;
    L.grid = std::max(1, std::min(L.item_count, per_sm * num_sms()));
    if (L.lu_stride > 0)
        L.grid = (int)std::max<int64_t>(1, std::min<int64_t>(L.grid, kMemScratchBudget / L.lu_stride));
    return AMFRW_OK;
}

// Reassign every class's part of the scratch array and reallocate it when
// its length changes.
int relayout_scratch(Plan& P)
{
    int64_t off = 0;
    for (LaunchClass& c : P.classes) {
        c.lu_offset = off;
        off += c.lu_stride * c.grid;
    }
    if (off != P.lu_scratch_len) {
        CUDA_TRY(cudaStreamSynchronize(P.stream));
        cudaFree(P.d_lu);
        P.d_lu = nullptr;
        P.lu_scratch_len = off;
        if (off > 0) CUDA_TRY(cudaMalloc(&P.d_lu, (size_t)off));
    }
    return AMFRW_OK;
}

int all_same_steps(const Plan& P)
{
    int s = P.insts[0].n_steps;
    for (const InstDev& I : P.insts)
        if (I.n_steps != s) return -1;
    return s;
}

}  // namespace

struct amfrw_problem {
    Plan plan;
    int steps_done = 0;
};

struct amfrw_batch {
    Plan plan;
    bool timing = false;
    std::vector<cudaEvent_t> ev;       // two per launch record
    cudaStream_t capture = nullptr;    // private stream the graph is captured on
    cudaStream_t side = nullptr;       // stream the conditional body is captured on
    cudaGraphExec_t exec = nullptr;    // the captured solve + combination
    bool exec_timing = false;          // whether the graph records the timing events
    // FP64 re-solve of ill-conditioned mixed-precision instances: the batch
    // planned in FP64 (its grid values go to plan.d_u), the marks and counters
    std::unique_ptr<Plan> promo;
    double kappa_max = 0.0;            // <= 0: no promotion
    int32_t* d_mask = nullptr;
    double* d_kappa = nullptr;
    int32_t* d_pcount = nullptr;
    unsigned* d_done = nullptr;
    ~amfrw_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (capture) cudaStreamDestroy(capture);
        if (side) cudaStreamDestroy(side);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        cudaFree(d_mask);
        cudaFree(d_kappa);
        cudaFree(d_pcount);
        cudaFree(d_done);
    }
};

namespace {

// Cache of the autotuner: class signature -> choice bits (bit 0: one
// persistent multi-class launch for the warp groups; bit 1 + k: the k-th CTA
// class keeps its grids in global memory instead of shared memory).
std::mutex g_tune_mutex;
std::map<std::string, int> g_tune_cache;

std::string class_signature(const Plan& P)
{
    std::string sig;
    for (const LaunchClass& c : P.classes) {
        sig += std::to_string(c.N) + (c.mixed ? "m" : "d") + (c.kind == kWarpGroup ? "w" : (c.kind == kCtaGroup ? "c" : "g")) +
               std::to_string(P.items[c.item_begin].L) + ":" +
               std::to_string(c.item_count > 4096 ? 4096 : c.item_count) + ";";
    }
    return sig;
}

void load_tune_file()
{
    static bool loaded = false;
    if (loaded) return;
    loaded = true;
    const char* path = getenv("AMFRW_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char line[8192];
    while (fgets(line, sizeof(line), f)) {
        char* sp = strrchr(line, ' ');
        if (!sp) continue;
        *sp = 0;
        g_tune_cache[line] = atoi(sp + 1);
    }
    fclose(f);
}

void save_tune_entry(const std::string& sig, int choice)
{
    const char* path = getenv("AMFRW_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d\n", sig.c_str(), choice);
    fclose(f);
}

// Bits of a cached choice: bit 0 one persistent multi-class launch; bit 1 + k
// the k-th CTA class in global memory; bits kChoiceWidthShift.. the widening of
// the warp groups (log2).
constexpr int kChoiceWidthShift = 24;

// Apply cached choice bits to a freshly planned batch.
int apply_choice(Plan& P, int choice)
{
    int st = AMFRW_OK;
    int k = 0;
    bool moved = false;
    for (size_t c = 0; c < P.classes.size() && st == AMFRW_OK; ++c) {
        if (P.classes[c].kind != kCtaGroup) continue;
        if ((choice >> (1 + k)) & 1) {
            st = class_to_global(P, (int)c);
            moved = true;
        }
        ++k;
    }
    if (st == AMFRW_OK && moved) st = relayout_scratch(P);
    const bool multi = (choice & 1) != 0;
    const int delta = (choice >> kChoiceWidthShift) & 3;
    if (st == AMFRW_OK && (multi != P.use_multi || delta != P.glog_delta)) {
        P.use_multi = multi;
        P.glog_delta = delta;
        st = build_warp_launches(P);
        if (st == AMFRW_OK) st = upload_warp_launches(P);
    }
    return st;
}

// Capture solve + combination into a CUDA graph on the batch's private
// stream.  With promotion on, the combination also marks the ill-conditioned
// mixed-precision instances and sets a conditional; the conditional node's
// body re-solves the marked instances in FP64 and recombines them.
int capture_graph(amfrw_batch* b)
{
    Plan& P = b->plan;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (!b->capture) CUDA_TRY(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
    const bool promote = b->promo && b->kappa_max > 0.0;
    if (promote && !b->side) CUDA_TRY(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
    cudaStream_t user = P.stream;
    P.stream = b->capture;
    CUDA_TRY(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t g = nullptr;
    int st = run_solve(P, P.insts[0].n_steps, 0, b->timing ? b->ev.data() : nullptr);
    Promote pr{};
    if (st == AMFRW_OK && promote) {
        pr.kappa_max = b->kappa_max;
        pr.mask = b->d_mask;
        pr.kappa = b->d_kappa;
        pr.count = b->d_pcount;
        pr.done = b->d_done;
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        if (cudaStreamGetCaptureInfo(b->capture, &cs, nullptr, &cg) != cudaSuccess ||
            cudaGraphConditionalHandleCreate(&pr.cond, cg, 0, cudaGraphCondAssignDefault) != cudaSuccess)
            st = fail(AMFRW_ECUDA, "conditional handle");
    }
    if (st == AMFRW_OK) st = run_combine(P, P.d_prices, promote ? &pr : nullptr);
    if (st == AMFRW_OK && promote) {
        // if (any instance marked) { FP64 re-solve of the marked instances; recombine them }
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        cudaGraphNode_t node = nullptr;
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = pr.cond;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        if (cudaStreamGetCaptureInfo(b->capture, &cs, nullptr, &cg, &deps, nullptr, &nd) != cudaSuccess ||
            cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np) != cudaSuccess ||
            cudaStreamUpdateCaptureDependencies(b->capture, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
                cudaSuccess)
            st = fail(AMFRW_ECUDA, "conditional node");
        if (st == AMFRW_OK) {
            cudaGraph_t body = np.conditional.phGraph_out[0];
            Plan& Q = *b->promo;
            Q.stream = b->side;
            P.stream = b->side;
            cudaError_t e = cudaStreamBeginCaptureToGraph(b->side, body, nullptr, nullptr, 0,
                                                          cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) st = fail(AMFRW_ECUDA, std::string("body capture: ") + cudaGetErrorString(e));
            if (st == AMFRW_OK) st = run_solve(Q, Q.insts[0].n_steps, 0);
            if (st == AMFRW_OK) st = run_combine(P, P.d_prices, nullptr, b->d_mask);
            cudaGraph_t body_out = nullptr;
            e = cudaStreamEndCapture(b->side, &body_out);
            if (st == AMFRW_OK && e != cudaSuccess)
                st = fail(AMFRW_ECUDA, std::string("body capture: ") + cudaGetErrorString(e));
            P.stream = b->capture;
            Q.stream = user;
        }
    }
    cudaError_t e = cudaStreamEndCapture(b->capture, &g);
    P.stream = user;
    if (st != AMFRW_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(AMFRW_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(AMFRW_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    b->exec_timing = b->timing;
    return AMFRW_OK;
}

// The FP64 plan of a batch's instances for the re-solve of ill-conditioned
// mixed-precision instances; its grid values go to the batch's own array.
int build_promotion(amfrw_batch* b, const amfrw_params* ps, int n, void* stream)
{
    bool any = false;
    for (int i = 0; i < n; ++i) any |= ps[i].precision == AMFRW_MIXED;
    if (!any) return AMFRW_OK;
    std::vector<amfrw_params> q(ps, ps + n);
    for (amfrw_params& x : q) x.precision = AMFRW_FP64;
    b->promo.reset(new (std::nothrow) Plan());
    if (!b->promo) return fail(AMFRW_ENOMEM, "host allocation failed");
    Plan& Q = *b->promo;
    int st = build_plan(q.data(), n, stream, false, Q);
    if (st != AMFRW_OK) return st;
    cudaFree(Q.d_u);
    Q.d_u = b->plan.d_u;
    Q.shared_u = true;
    CUDA_TRY(cudaMalloc(&b->d_mask, sizeof(int32_t) * n));
    CUDA_TRY(cudaMalloc(&b->d_kappa, sizeof(double) * n));
    CUDA_TRY(cudaMalloc(&b->d_pcount, sizeof(int32_t)));
    CUDA_TRY(cudaMalloc(&b->d_done, sizeof(unsigned)));
    CUDA_TRY(cudaMemsetAsync(b->d_mask, 0, sizeof(int32_t) * n, (cudaStream_t)stream));
    CUDA_TRY(cudaMemsetAsync(b->d_kappa, 0, sizeof(double) * n, (cudaStream_t)stream));
    CUDA_TRY(cudaMemsetAsync(b->d_pcount, 0, sizeof(int32_t), (cudaStream_t)stream));
    Q.inst_mask = b->d_mask;
    b->kappa_max = kKappaMaxDefault;
    return AMFRW_OK;
}

int ensure_events(amfrw_batch* b)
{
    const size_t need = 2 * b->plan.classes.size();
    while (b->ev.size() < need) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        b->ev.push_back(e);
    }
    return AMFRW_OK;
}

}  // namespace


extern "C" {

const char* amfrw_status_string(int status)
{
    switch (status) {
        case AMFRW_OK: return "AMFRW_OK";
        case AMFRW_EINVAL: return "AMFRW_EINVAL";
        case AMFRW_ENOTPSD: return "AMFRW_ENOTPSD";
        case AMFRW_ENOMEM: return "AMFRW_ENOMEM";
        case AMFRW_ECUDA: return "AMFRW_ECUDA";
        case AMFRW_ETIMEOUT: return "AMFRW_ETIMEOUT";
        case AMFRW_ENONFINITE: return "AMFRW_ENONFINITE";
        case AMFRW_ETOOBIG: return "AMFRW_ETOOBIG";
        default: return "AMFRW_UNKNOWN";
    }
}

const char* amfrw_last_error(void) { return g_last_error.c_str(); }

int amfrw_problem_create(const amfrw_params* p, void* cuda_stream, amfrw_problem** out)
{
    if (!out) return fail(AMFRW_EINVAL, "out is NULL");
    *out = nullptr;
    amfrw_problem* h = new (std::nothrow) amfrw_problem();
    if (!h) return fail(AMFRW_ENOMEM, "host allocation failed");
    int st = build_plan(p, 1, cuda_stream, true, h->plan);
    if (st != AMFRW_OK) {
        delete h;
        return st;
    }
    // state = payoff: zero steps with a store writes Y = G on every grid
    st = run_solve(h->plan, 0, kStoreState);
    if (st != AMFRW_OK) {
        delete h;
        return st;
    }
    *out = h;
    return AMFRW_OK;
}

int amfrw_step(amfrw_problem* h, int32_t n_steps)
{
    if (!h) return fail(AMFRW_EINVAL, "handle is NULL");
    if (n_steps < 0) return fail(AMFRW_EINVAL, "n_steps must be >= 0");
    int st = run_solve(h->plan, n_steps, kLoadState | kStoreState);
    if (st == AMFRW_OK) h->steps_done += n_steps;
    return st;
}

int amfrw_combine(amfrw_problem* h, double* price_out)
{
    if (!h || !price_out) return fail(AMFRW_EINVAL, "NULL argument");
    Plan& P = h->plan;
    int st = run_combine(P, P.d_prices);
    if (st != AMFRW_OK) return st;
    double v = 0.0;
    int32_t flag = 0;
    CUDA_TRY(cudaMemcpyAsync(&v, P.d_prices, sizeof(double), cudaMemcpyDeviceToHost, P.stream));
    CUDA_TRY(cudaMemcpyAsync(&flag, P.d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, P.stream));
    CUDA_TRY(cudaStreamSynchronize(P.stream));
    if (flag) return fail(AMFRW_ENONFINITE, "the combined price is not finite");
    *price_out = v;
    return AMFRW_OK;
}

int amfrw_problem_num_grids(const amfrw_problem* h, int32_t* n_grids, int32_t* dim)
{
    if (!h || !n_grids || !dim) return fail(AMFRW_EINVAL, "NULL argument");
    *n_grids = h->plan.n_grids;
    *dim = h->plan.dim;
    return AMFRW_OK;
}

int amfrw_problem_grid_info(const amfrw_problem* h, int32_t* levels_out, double* coefs_out)
{
    if (!h) return fail(AMFRW_EINVAL, "handle is NULL");
    const Plan& P = h->plan;
    for (int g = 0; g < P.n_grids; ++g) {
        if (levels_out)
            for (int a = 0; a < P.dim; ++a) levels_out[g * P.dim + a] = P.levels[g * kMaxDim + a];
        if (coefs_out) coefs_out[g] = P.coefs[g];
    }
    return AMFRW_OK;
}

int amfrw_problem_grid_values(amfrw_problem* h, double* u_out)
{
    if (!h || !u_out) return fail(AMFRW_EINVAL, "NULL argument");
    Plan& P = h->plan;
    CUDA_TRY(cudaMemcpyAsync(u_out, P.d_u, sizeof(double) * P.n_grids, cudaMemcpyDeviceToHost, P.stream));
    CUDA_TRY(cudaStreamSynchronize(P.stream));
    return AMFRW_OK;
}

int amfrw_problem_read_grid(amfrw_problem* h, int32_t grid, double* Y_out)
{
    if (!h || !Y_out) return fail(AMFRW_EINVAL, "NULL argument");
    Plan& P = h->plan;
    if (grid < 0 || grid >= P.n_grids) return fail(AMFRW_EINVAL, "grid index out of range");
    int64_t off = -1, L = 0;
    for (const Item& it : P.items)
        if (it.out_idx == grid) {
            off = it.state_off;
            L = it.L;
        }
    if (off < 0) return fail(AMFRW_EINVAL, "grid has no stored state");
    CUDA_TRY(cudaMemcpyAsync(Y_out, P.d_state + off, sizeof(double) * L, cudaMemcpyDeviceToHost, P.stream));
    CUDA_TRY(cudaStreamSynchronize(P.stream));
    return AMFRW_OK;
}

void amfrw_problem_destroy(amfrw_problem* h) { delete h; }

int amfrw_batch_create(const amfrw_params* ps, int32_t n, void* cuda_stream, amfrw_batch** out)
{
    if (!out) return fail(AMFRW_EINVAL, "out is NULL");
    *out = nullptr;
    amfrw_batch* b = new (std::nothrow) amfrw_batch();
    if (!b) return fail(AMFRW_ENOMEM, "host allocation failed");
    int st = build_plan(ps, n, cuda_stream, false, b->plan);
    if (st != AMFRW_OK) {
        delete b;
        return st;
    }
    if (all_same_steps(b->plan) < 0) {
        delete b;
        return fail(AMFRW_EINVAL, "all instances of a batch must use the same n_steps");
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        load_tune_file();
        auto it = g_tune_cache.find(class_signature(b->plan));
        if (it != g_tune_cache.end()) {
            st = apply_choice(b->plan, it->second);
            if (st != AMFRW_OK) {
                delete b;
                return st;
            }
        }
    }
    st = build_promotion(b, ps, n, cuda_stream);
    if (st != AMFRW_OK) {
        delete b;
        return st;
    }
    *out = b;
    return AMFRW_OK;
}

int amfrw_batch_run(amfrw_batch* b, double* d_prices_out)
{
    if (!b || !d_prices_out) return fail(AMFRW_EINVAL, "NULL argument");
    Plan& P = b->plan;
    // the solve and the combination are replayed from a CUDA graph
    if (!b->exec || b->exec_timing != b->timing) {
        int st = capture_graph(b);
        if (st != AMFRW_OK) return st;
    }
    CUDA_TRY(cudaGraphLaunch(b->exec, P.stream));
    if (d_prices_out != P.d_prices)
        CUDA_TRY(cudaMemcpyAsync(d_prices_out, P.d_prices, sizeof(double) * P.n_inst,
                                 cudaMemcpyDeviceToDevice, P.stream));
    return AMFRW_OK;
}

int amfrw_batch_autotune(amfrw_batch* b, int32_t trials, int32_t* use_multi_out)
{
    if (!b) return fail(AMFRW_EINVAL, "NULL argument");
    Plan& P = b->plan;
    if (trials < 1) trials = 1;
    const int steps = P.insts[0].n_steps;
    const std::string sig = class_signature(P);  // of the plan as built, before any move
    const std::vector<LaunchClass> base = P.classes;
    // time `trials` solves (after a warm-up); per-record times if rec != nullptr
    auto timed = [&](float& total, std::vector<float>* rec) -> int {
        const size_t nrec = launch_records(P).size();
        std::vector<cudaEvent_t> ev(2 * nrec, nullptr);
        for (cudaEvent_t& e : ev) CUDA_TRY(cudaEventCreate(&e));
        int st = run_solve(P, steps, 0);
        total = 0.f;
        if (rec) rec->assign(nrec, 0.f);
        for (int k = 0; k < trials && st == AMFRW_OK; ++k) {
            st = run_solve(P, steps, 0, ev.data());
            if (st == AMFRW_OK && cudaEventSynchronize(ev.back()) != cudaSuccess) st = fail(AMFRW_ECUDA, "timing");
            for (size_t r = 0; r < nrec && st == AMFRW_OK; ++r) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]);
                total += ms;
                if (rec) (*rec)[r] += ms;
            }
        }
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        return st;
    };
    int st = AMFRW_OK;
    // 1. warp groups: per-class launches against one persistent multi-class launch
    bool best = P.use_multi;
    bool differs = false;
    for (size_t c = 0; c < P.classes.size(); ++c)
        for (size_t d = c + 1; d < P.classes.size(); ++d)
            if (P.classes[c].warp && P.classes[d].warp && P.classes[c].N == P.classes[d].N &&
                P.classes[c].mixed == P.classes[d].mixed)
                differs = true;
    if (differs) {
        float t[2] = {0.f, 0.f};
        for (int m = 0; m < 2 && st == AMFRW_OK; ++m) {
            P.use_multi = m == 1;
            st = build_warp_launches(P);
            if (st == AMFRW_OK) st = upload_warp_launches(P);
            if (st == AMFRW_OK) st = timed(t[m], nullptr);
        }
        if (st != AMFRW_OK) return st;
        // one persistent launch per (N, precision) unless the per-class
        // launches are clearly faster: a launch count that does not grow with
        // the classes is worth a few percent
        best = t[1] <= 1.10f * t[0];
        P.use_multi = best;
        st = build_warp_launches(P);
        if (st == AMFRW_OK) st = upload_warp_launches(P);
        if (st != AMFRW_OK) return st;
    }
    // 2. warp groups: their natural width against twice the lanes per grid
    //    (one more PCR level per line, half the nodes per lane)
    bool narrow = false;
    for (const LaunchClass& c : P.classes) narrow |= c.warp && c.glog < 5;
    if (narrow) {
        float t[2] = {0.f, 0.f};
        for (int d = 0; d < 2 && st == AMFRW_OK; ++d) {
            P.glog_delta = d;
            st = build_warp_launches(P);
            if (st == AMFRW_OK) st = upload_warp_launches(P);
            if (st == AMFRW_OK) st = timed(t[d], nullptr);
        }
        if (st != AMFRW_OK) return st;
        P.glog_delta = t[1] < t[0] ? 1 : 0;
        st = build_warp_launches(P);
        if (st == AMFRW_OK) st = upload_warp_launches(P);
        if (st != AMFRW_OK) return st;
    }
    // 3. CTA classes: grid state in shared memory against global memory, class by class
    int choice = (best ? 1 : 0) | (P.glog_delta << kChoiceWidthShift);
    std::vector<int> cta;
    for (size_t c = 0; c < P.classes.size(); ++c)
        if (P.classes[c].kind == kCtaGroup) cta.push_back((int)c);
    if (!cta.empty()) {
        // launch record of each CTA class
        std::vector<size_t> at;
        {
            const std::vector<std::pair<int, int>> recs = launch_records(P);
            for (int c : cta)
                for (size_t r = 0; r < recs.size(); ++r)
                    if (recs[r].second == c) at.push_back(r);
        }
        float tot[2];
        std::vector<float> rec[2];
        st = timed(tot[0], &rec[0]);
        for (int c : cta)
            if (st == AMFRW_OK) st = class_to_global(P, c);
        if (st == AMFRW_OK) st = relayout_scratch(P);
        if (st == AMFRW_OK) st = timed(tot[1], &rec[1]);
        if (st != AMFRW_OK) return st;
        P.classes = base;  // back to shared memory, then move the classes that were faster
        for (size_t k = 0; k < cta.size(); ++k) {
            if (rec[1][at[k]] < rec[0][at[k]]) {
                choice |= 1 << (1 + (int)k);
                st = class_to_global(P, cta[k]);
                if (st != AMFRW_OK) return st;
            }
        }
        st = relayout_scratch(P);
        if (st != AMFRW_OK) return st;
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[sig] = choice;
        save_tune_entry(sig, choice);
    }
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (use_multi_out) *use_multi_out = best ? 1 : 0;
    return AMFRW_OK;
}

int amfrw_batch_set_kappa_max(amfrw_batch* b, double kappa_max)
{
    if (!b || !std::isfinite(kappa_max)) return fail(AMFRW_EINVAL, "NULL argument or kappa_max not finite");
    if (kappa_max != b->kappa_max && b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->kappa_max = b->promo ? kappa_max : 0.0;
    return AMFRW_OK;
}

int amfrw_batch_promoted(amfrw_batch* b, int32_t* n_promoted, double* kappa_out)
{
    if (!b || !n_promoted) return fail(AMFRW_EINVAL, "NULL argument");
    Plan& P = b->plan;
    int32_t c = 0;
    if (b->d_pcount && b->kappa_max > 0.0) {
        CUDA_TRY(cudaMemcpyAsync(&c, b->d_pcount, sizeof(int32_t), cudaMemcpyDeviceToHost, P.stream));
        if (kappa_out)
            CUDA_TRY(cudaMemcpyAsync(kappa_out, b->d_kappa, sizeof(double) * P.n_inst, cudaMemcpyDeviceToHost,
                                     P.stream));
        CUDA_TRY(cudaStreamSynchronize(P.stream));
    } else if (kappa_out) {
        for (int i = 0; i < P.n_inst; ++i) kappa_out[i] = 0.0;
    }
    *n_promoted = c;
    return AMFRW_OK;
}

int amfrw_batch_classes(const amfrw_batch* b, int32_t* n_warp, int32_t* n_cta, int32_t* n_global)
{
    if (!b) return fail(AMFRW_EINVAL, "NULL argument");
    int32_t c[3] = {0, 0, 0};
    for (const LaunchClass& L : b->plan.classes) ++c[L.kind];
    if (n_warp) *n_warp = c[kWarpGroup];
    if (n_cta) *n_cta = c[kCtaGroup];
    if (n_global) *n_global = c[kMemGroup];
    return AMFRW_OK;
}

int amfrw_batch_enable_timing(amfrw_batch* b, int32_t on)
{
    if (!b) return fail(AMFRW_EINVAL, "NULL argument");
    if (on) {
        int st = ensure_events(b);
        if (st != AMFRW_OK) return st;
    }
    b->timing = on != 0;
    return AMFRW_OK;
}

int amfrw_batch_kernel_times(amfrw_batch* b, float* ms_out, double* node_steps_out, int32_t* dims_out,
                             int32_t cap, int32_t* n_out)
{
    if (!b || !ms_out || !n_out) return fail(AMFRW_EINVAL, "NULL argument");
    if (b->ev.empty()) return fail(AMFRW_EINVAL, "timing is not enabled");
    const Plan& P = b->plan;
    const std::vector<std::pair<int, int>> recs = launch_records(P);
    const int n = std::min<int>(cap, (int)recs.size());
    for (int r = 0; r < n; ++r) {
        CUDA_TRY(cudaEventSynchronize(b->ev[2 * r + 1]));
        CUDA_TRY(cudaEventElapsedTime(&ms_out[r], b->ev[2 * r], b->ev[2 * r + 1]));
        std::vector<int> cls;
        if (recs[r].first >= 0) cls = P.wl[recs[r].first].covers;
        else cls.push_back(recs[r].second);
        double s = 0.0;
        int dim = 0;
        for (int c : cls) {
            const LaunchClass& L = P.classes[c];
            for (int k = L.item_begin; k < L.item_begin + L.item_count; ++k)
                s += (double)P.items[k].L * (double)P.insts[P.items[k].inst].n_steps;
            dim = L.N;  // a launch's classes share N
        }
        if (node_steps_out) node_steps_out[r] = s;
        if (dims_out) dims_out[r] = dim;
    }
    *n_out = n;
    return AMFRW_OK;
}

int amfrw_batch_io_bytes(const amfrw_batch* b, int64_t* h2d_bytes, int64_t* d2h_bytes)
{
    if (!b || !h2d_bytes || !d2h_bytes) return fail(AMFRW_EINVAL, "NULL argument");
    const Plan& P = b->plan;
    *h2d_bytes = (int64_t)(sizeof(InstDev) * P.insts.size() + sizeof(Item) * P.items.size() +
                           sizeof(double) * P.coefs.size());
    *d2h_bytes = (int64_t)(sizeof(double) * P.n_inst + sizeof(int32_t));
    return AMFRW_OK;
}

int amfrw_batch_launches(const amfrw_batch* b, int32_t* n_launches)
{
    if (!b || !n_launches) return fail(AMFRW_EINVAL, "NULL argument");
    *n_launches = (int32_t)launch_records(b->plan).size() + 1;
    return AMFRW_OK;
}

void amfrw_batch_destroy(amfrw_batch* b) { delete b; }

}  // extern "C"

namespace {

// amfrw_solve_batch keeps, per calling thread, the batch of its last call:
// grid list, device buffers and captured graph depend only on the instances'
// shapes, the stream and the device, so a following call with the same
// shapes validates and uploads the new parameter records and replays the
// graph.  Released by amfrw_solve_batch_release, by a call with other
// shapes, or at thread exit.
struct SolveKey {
    int32_t n_rates, payoff, n_steps, level, psi, full_grid, precision, flags;
    bool operator==(const SolveKey& o) const { return memcmp(this, &o, sizeof(SolveKey)) == 0; }
};

struct SolveCache {
    amfrw_batch* b = nullptr;
    int dev = -1;
    void* stream = nullptr;
    std::vector<SolveKey> key;
    InstDev* stage = nullptr;  // pinned copy of the instance records (both plans)
    int64_t h2d = 0, d2h = 0;  // bytes the last call copied
    void drop()
    {
        if (b) amfrw_batch_destroy(b);
        if (stage) cudaFreeHost(stage);
        b = nullptr;
        stage = nullptr;
        key.clear();
    }
    ~SolveCache() { drop(); }
};
thread_local SolveCache g_solve_cache;

SolveKey solve_key(const amfrw_params& p)
{
    SolveKey k;
    memset(&k, 0, sizeof(k));
    k.n_rates = p.n_rates;
    k.payoff = p.payoff;
    k.n_steps = p.n_steps;
    k.level = p.level;
    k.psi = p.psi;
    k.full_grid = p.full_grid != 0;
    k.precision = p.precision;
    k.flags = p.flags;
    return k;
}

// New parameter records into a plan whose grids are those of `ps`
// (precision forced to FP64 for the re-solve plan), copied to the device
// from the pinned array `stage` [n].
int refresh_insts(Plan& P, const amfrw_params* ps, int n, bool fp64, InstDev* stage, int64_t& bytes)
{
    for (int i = 0; i < n; ++i) {
        amfrw_params q = ps[i];
        if (fp64) q.precision = AMFRW_FP64;
        InstDev I = to_device(&q);
        I.grid_begin = P.insts[(size_t)i].grid_begin;
        I.grid_count = P.insts[(size_t)i].grid_count;
        P.insts[(size_t)i] = I;
        stage[i] = I;
    }
    CUDA_TRY(cudaMemcpyAsync(P.d_insts, stage, sizeof(InstDev) * (size_t)n, cudaMemcpyHostToDevice, P.stream));
    bytes += (int64_t)(sizeof(InstDev) * (size_t)n);
    return AMFRW_OK;
}

}  // namespace

extern "C" {

int amfrw_solve_batch(const amfrw_params* ps, int32_t n, double* prices_out, void* cuda_stream)
{
    if (!prices_out) return fail(AMFRW_EINVAL, "prices_out is NULL");
    if (n < 1 || !ps) return fail(AMFRW_EINVAL, "need at least one instance and a params array");
    SolveCache& C = g_solve_cache;
    std::vector<SolveKey> key((size_t)n);
    for (int i = 0; i < n; ++i) key[(size_t)i] = solve_key(ps[i]);
    int64_t h2d = 0;
    int st = AMFRW_OK;
    // (no CUDA call before the parameters are validated: a fresh plan
    // validates first, and a kept plan exists only after a CUDA device did)
    int dev = -1;
    if (C.b) CUDA_TRY(cudaGetDevice(&dev));
    const bool hit = C.b && C.dev == dev && C.stream == cuda_stream && C.key == key;
    if (hit) {
        for (int i = 0; i < n && st == AMFRW_OK; ++i) {
            st = validate(ps + i);
            if (st != AMFRW_OK) g_last_error = "instance " + std::to_string(i) + ": " + g_last_error;
        }
        if (st != AMFRW_OK) return st;
        if (!C.stage && cudaMallocHost(&C.stage, 2 * sizeof(InstDev) * (size_t)n) != cudaSuccess) {
            C.stage = nullptr;
            C.drop();
            return fail(AMFRW_ENOMEM, "pinned host allocation failed");
        }
        st = refresh_insts(C.b->plan, ps, n, false, C.stage, h2d);
        if (st == AMFRW_OK && C.b->promo) st = refresh_insts(*C.b->promo, ps, n, true, C.stage + n, h2d);
        if (st != AMFRW_OK) {
            C.drop();
            return st;
        }
    } else {
        C.drop();
        st = amfrw_batch_create(ps, n, cuda_stream, &C.b);
        if (st != AMFRW_OK) return st;
        CUDA_TRY(cudaGetDevice(&dev));
        C.dev = dev;
        C.stream = cuda_stream;
        C.key = std::move(key);
        int64_t d2h_unused = 0;
        amfrw_batch_io_bytes(C.b, &h2d, &d2h_unused);
    }
    Plan& P = C.b->plan;
    st = amfrw_batch_run(C.b, P.d_prices);
    if (st == AMFRW_OK) {
        int32_t flag = 0;
        cudaError_t e1 = cudaMemcpyAsync(prices_out, P.d_prices, sizeof(double) * n, cudaMemcpyDeviceToHost, P.stream);
        cudaError_t e2 = cudaMemcpyAsync(&flag, P.d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, P.stream);
        cudaError_t e3 = cudaStreamSynchronize(P.stream);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
            st = fail(AMFRW_ECUDA, std::string("download: ") + cudaGetErrorString(e3 != cudaSuccess ? e3 : (e1 != cudaSuccess ? e1 : e2)));
        else if (flag)
            st = fail(AMFRW_ENONFINITE, "a combined price is not finite");
    }
    C.h2d = h2d;
    C.d2h = (int64_t)(sizeof(double) * (size_t)n + sizeof(int32_t));
    if (st == AMFRW_ECUDA) C.drop();  // keep nothing whose state is unknown
    return st;
}

int amfrw_solve_batch_io(int64_t* h2d_bytes, int64_t* d2h_bytes)
{
    if (!h2d_bytes || !d2h_bytes) return fail(AMFRW_EINVAL, "NULL argument");
    *h2d_bytes = g_solve_cache.h2d;
    *d2h_bytes = g_solve_cache.d2h;
    return AMFRW_OK;
}

void amfrw_solve_batch_release(void) { g_solve_cache.drop(); }

}  // extern "C"

// ------------------------------------------------------------------------
// Entry point that allocates no device memory (amfrw_solve_noalloc).
//
// Every other entry point gets its device buffers from cudaMalloc.  Some
// callers cannot do that: a host program whose device memory is owned by
// another allocator (a framework's caching pool or a fixed budget reserved
// at start-up), or a latency-sensitive loop that must not pay for
// cudaMalloc/cudaFree, whose frees synchronise the whole device and stall
// every other stream.  This entry point takes its working memory from one
// fixed device array declared below, so it never allocates.  That array is
// reserved by every GPU that loads the library, for the life of the
// process.
namespace {

// Scratch of amfrw_solve_noalloc: instance records, grid list, combination
// coefficients, per-grid values, work counters and the Thomas factors of
// the grids solved by whole blocks.
static __device__ __align__(256) unsigned char g_noalloc_scratch[AMFRW_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name only stands in for the symbol, so the address is asked
// from the runtime, with the calling thread's device current, on every call:
// the lookup is cheap once the module is loaded, and an address cached past a
// device reset (which unloads the module) would point at unmapped memory.
int noalloc_scratch(unsigned char** out)
{
    void* p = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    *out = static_cast<unsigned char*>(p);
    return AMFRW_OK;
}

int64_t align256(int64_t x) { return (x + 255) & ~(int64_t)255; }

// Releases the host vectors of a plan built in place for amfrw_solve_noalloc.
// The plan's destructor is never run on that path because it would call
// cudaFree (on null pointers).
void noalloc_release_host(Plan& P)
{
    std::vector<InstDev>().swap(P.insts);
    std::vector<Item>().swap(P.items);
    std::vector<double>().swap(P.coefs);
    std::vector<int8_t>().swap(P.levels);
    std::vector<LaunchClass>().swap(P.classes);
    std::vector<Plan::WarpLaunch>().swap(P.wl);
    P.d_insts = nullptr; P.d_items = nullptr; P.d_coefs = nullptr; P.d_u = nullptr;
    P.d_prices = nullptr; P.d_queue = nullptr; P.d_flag = nullptr; P.d_state = nullptr;
    P.d_lu = nullptr;
    P.d_cdesc = nullptr;
}

int noalloc_run(const amfrw_params* ps, int n, double* d_prices_out, cudaStream_t stream, Plan& P)
{
    int st = plan_host(ps, n, false, P);
    if (st == AMFRW_OK) st = build_warp_launches(P);
    if (st != AMFRW_OK) return st;
    const int s0 = P.insts[0].n_steps;
    for (const InstDev& I : P.insts)
        if (I.n_steps != s0) return fail(AMFRW_EINVAL, "all instances must use the same n_steps");
    // carve the fixed array: records, grid list, coefficients, values, counters, factors
    const int64_t o_inst = 0;
    const int64_t o_item = align256(o_inst + (int64_t)(sizeof(InstDev) * P.insts.size()));
    const int64_t o_coef = align256(o_item + (int64_t)(sizeof(Item) * P.items.size()));
    const int64_t o_u = align256(o_coef + (int64_t)(sizeof(double) * P.coefs.size()));
    const int64_t o_queue = align256(o_u + (int64_t)(sizeof(double) * P.coefs.size()));
    const int64_t o_flag = align256(o_queue + (int64_t)(sizeof(int32_t) * P.classes.size()));
    const int64_t o_desc = align256(o_flag + (int64_t)sizeof(int32_t));
    const int64_t o_lu = align256(o_desc + (int64_t)(sizeof(ClassDesc) * P.n_cdesc));
    // the per-block slices of the CTA and global-memory classes (factors,
    // states) take what the array has left: a class that wants more blocks
    // than fit runs fewer (each block pulls grids from the class's queue
    // until it is empty), down to one block per class
    const int64_t room = (int64_t)AMFRW_NOALLOC_SCRATCH_BYTES - o_lu;
    if (P.lu_scratch_len > room && room > 0) {
        int64_t off = 0;
        for (LaunchClass& c : P.classes) {
            if (c.lu_stride > 0) {
                const int64_t fit = (int64_t)((double)c.grid * (double)room / (double)P.lu_scratch_len);
                c.grid = (int)std::max<int64_t>(1, std::min<int64_t>(c.grid, fit));
            }
            c.lu_offset = off;
            off += c.lu_stride * c.grid;
        }
        P.lu_scratch_len = off;
    }
    const int64_t total = o_lu + P.lu_scratch_len;
    if (total > (int64_t)AMFRW_NOALLOC_SCRATCH_BYTES)
        return fail(AMFRW_ETOOBIG, "problem needs " + std::to_string(total) +
                                       " bytes of scratch; amfrw_solve_noalloc is limited to " +
                                       std::to_string((long long)AMFRW_NOALLOC_SCRATCH_BYTES));
    unsigned char* base = nullptr;
    st = noalloc_scratch(&base);
    if (st != AMFRW_OK) return st;
    P.stream = stream;
    P.d_insts = reinterpret_cast<InstDev*>(base + o_inst);
    P.d_items = reinterpret_cast<Item*>(base + o_item);
    P.d_coefs = reinterpret_cast<double*>(base + o_coef);
    P.d_u = reinterpret_cast<double*>(base + o_u);
    P.d_queue = reinterpret_cast<int32_t*>(base + o_queue);
    P.d_flag = reinterpret_cast<int32_t*>(base + o_flag);
    P.d_lu = P.lu_scratch_len > 0 ? base + o_lu : nullptr;
    P.d_cdesc = reinterpret_cast<ClassDesc*>(base + o_desc);
    std::vector<ClassDesc> descs;
    for (const Plan::WarpLaunch& w : P.wl) descs.insert(descs.end(), w.cls.begin(), w.cls.end());
    if (!descs.empty())
        CUDA_TRY(cudaMemcpyAsync(P.d_cdesc, descs.data(), sizeof(ClassDesc) * descs.size(),
                                 cudaMemcpyHostToDevice, stream));
    // the array keeps the previous call's contents: the records are rewritten,
    // the per-grid values cleared, and run_solve / run_combine zero the counters
    CUDA_TRY(cudaMemcpyAsync(P.d_insts, P.insts.data(), sizeof(InstDev) * P.insts.size(),
                             cudaMemcpyHostToDevice, stream));
    CUDA_TRY(cudaMemcpyAsync(P.d_items, P.items.data(), sizeof(Item) * P.items.size(),
                             cudaMemcpyHostToDevice, stream));
    CUDA_TRY(cudaMemcpyAsync(P.d_coefs, P.coefs.data(), sizeof(double) * P.coefs.size(),
                             cudaMemcpyHostToDevice, stream));
    CUDA_TRY(cudaMemsetAsync(P.d_u, 0, sizeof(double) * P.coefs.size(), stream));
    st = run_solve(P, s0, 0);
    if (st != AMFRW_OK) return st;
    return run_combine(P, d_prices_out);
}

}  // namespace

extern "C" int amfrw_solve_noalloc(const amfrw_params* ps, int32_t n, double* d_prices_out,
                                   void* cuda_stream)
{
    if (!d_prices_out) return fail(AMFRW_EINVAL, "d_prices_out is NULL");
    if (n < 1) return fail(AMFRW_EINVAL, "need at least one instance");
    if (!ps) return fail(AMFRW_EINVAL, "params is NULL");
    // The host records are copied from temporary host buffers that are freed
    // on return, so the call cannot be recorded into a CUDA graph: a replay
    // would read freed host memory.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing((cudaStream_t)cuda_stream, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(AMFRW_EINVAL, "amfrw_solve_noalloc must not be called while its stream is being captured");
    alignas(Plan) unsigned char buf[sizeof(Plan)];
    Plan* P = new (buf) Plan();
    const int st = noalloc_run(ps, n, d_prices_out, (cudaStream_t)cuda_stream, *P);
    noalloc_release_host(*P);
    return st;
}
