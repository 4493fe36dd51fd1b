// Library-internal records shared by the host launcher and the kernels.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define AMFRW_HD __host__ __device__ __forceinline__
#else
#define AMFRW_HD inline
#endif

namespace amfrw {

constexpr int kMaxDim = 8;

// Per-instance parameters on the device (one per pricing problem).
struct InstDev {
    int32_t N, payoff, n_steps, precision;
    int32_t grid_begin, grid_count, pad0, pad1;
    double alpha[kMaxDim], phi[kMaxDim], tau[kMaxDim], F0[kMaxDim];
    double Fmax[kMaxDim];          // Fmax[N-1] = V^max
    double rho[kMaxDim * kMaxDim];  // rate correlations, leading dimension 8
    double sigma, beta, V0, K, T, discount, theta, nu, dt;
    double pad2;
};

// One component grid of one instance: the unit of work of the solver.
struct Item {
    int32_t inst;        // instance index
    int32_t out_idx;     // slot of u_l(x*) in the per-grid output array
    int32_t L;           // Inner nodes prod_i M_i
    int32_t pad0;
    int8_t lv[kMaxDim];  // log2 M_i per axis
    int64_t state_off;   // offset (doubles) of the grid's Inner values in the
                         // state pool, or -1 when the state is not kept
};

// Shared-memory layout of one grid inside its work group.  The host uses it
// to size dynamic shared memory, the device to place the arrays; both call
// this one function so they cannot disagree.
struct Layout {
    int32_t cd, cf, tabd, tabf, pay, lu, Z, ZZ, H, FY, K1, K0, Kw, total;
    int32_t L, Lp, Lr, ntab, npay, nlu;
};

template <typename T>
struct Consts {
    T cV;                 // sigma^2 / (2 h_V^2)
    T dt, thdt, nudt;     // dt, theta*dt, nu*dt
    T rm[kMaxDim][kMaxDim];   // rho_ik / (4 h_i h_k), rate pairs i < k
    T rh[kMaxDim][kMaxDim];   // rho_ij for the drift sums (j <= i)
    T sm[kMaxDim];            // sigma phi_i / (4 h_i h_V)
    T g2[kMaxDim];            // 1 / (2 h_i)
};

AMFRW_HD int32_t align16(int32_t x) { return (x + 15) & ~15; }

// lu_smem: whether the Thomas factors live in shared memory (warp groups) or
// in the group's slice of a global scratch array (CTA groups, large grids).
AMFRW_HD Layout make_layout(int N, const int8_t* lv, bool mixed, bool lu_smem)
{
    Layout y{};
    int L = 1, sumM = 0, npay = 0;
    for (int i = 0; i < N; ++i) L <<= lv[i];
    for (int i = 0; i < N - 1; ++i) {
        sumM += 1 << lv[i];
        npay += (1 << lv[i]) + 1;
    }
    const int MV = 1 << lv[N - 1];
    const int M0 = 1 << lv[0];
    const int pad = M0 > 1 ? 1 : 0;
    y.L = L;
    y.Lp = L + (pad ? (L >> lv[0]) : 0);
    y.Lr = L >> lv[N - 1];
    y.ntab = 3 * sumM + MV;
    y.npay = 2 * npay;
    y.nlu = 3 * (MV * sumM + MV);
    const int sk = mixed ? 4 : 8;  // bytes of an increment / table value
    int o = 0;
    y.cd = o;   o = align16(o + (int)sizeof(Consts<double>));
    y.cf = o;   o = align16(o + (mixed ? (int)sizeof(Consts<float>) : 0));
    y.tabd = o; o = align16(o + 8 * y.ntab);
    y.tabf = o; o = align16(o + (mixed ? 4 * y.ntab : 0));
    y.pay = o;  o = align16(o + 8 * y.npay);
    y.lu = o;   o = align16(o + (lu_smem ? sk * y.nlu : 0));
    y.Z = o;    o = align16(o + 8 * y.Lp);
    y.ZZ = o;   o = align16(o + (mixed ? 8 * y.Lp : 0));
    y.H = o;    o = align16(o + sk * y.Lr);
    y.FY = o;   o = align16(o + (mixed ? 4 * y.Lp : 0));
    y.K1 = o;   o = align16(o + sk * y.Lp);
    y.K0 = o;   o = align16(o + sk * y.Lp);
    y.Kw = o;   o = align16(o + sk * y.Lp);
    y.total = o;
    return y;
}

// Launch-time arguments of the solver kernels.
struct SolveArgs {
    const Item* items;
    int32_t n_items;
    int32_t steps;        // steps to take in this launch
    int32_t flags;        // kLoadState | kStoreState
    int32_t smem_group;   // dynamic shared bytes per work group
    const InstDev* insts;
    double* u_out;        // [n grids] u_l(x*)
    double* state;        // state pool (Inner values of Y), may be null
    int32_t* queue;       // work counter, zero before the launch
    unsigned char* lu_scratch;  // CTA groups: Thomas factors, lu_stride bytes per block
    int64_t lu_stride;
};

constexpr int kLoadState = 1;
constexpr int kStoreState = 2;

// Host-side launchers, one translation unit per dimension N.
using LaunchFn = int (*)(const SolveArgs&, bool mixed, bool warp, int block, int grid,
                         size_t smem, void* stream);
int launch_n2(const SolveArgs&, bool, bool, int, int, size_t, void*);
int launch_n3(const SolveArgs&, bool, bool, int, int, size_t, void*);
int launch_n4(const SolveArgs&, bool, bool, int, int, size_t, void*);
int launch_n5(const SolveArgs&, bool, bool, int, int, size_t, void*);
int launch_n6(const SolveArgs&, bool, bool, int, int, size_t, void*);
int launch_n7(const SolveArgs&, bool, bool, int, int, size_t, void*);
int launch_n8(const SolveArgs&, bool, bool, int, int, size_t, void*);
// Occupancy query for the same instantiation (blocks per SM).
int occupancy(int N, bool mixed, bool warp, int block, size_t smem);
using OccFn = int (*)(bool mixed, bool warp, int block, size_t smem);
int occupancy_n2(bool, bool, int, size_t);
int occupancy_n3(bool, bool, int, size_t);
int occupancy_n4(bool, bool, int, size_t);
int occupancy_n5(bool, bool, int, size_t);
int occupancy_n6(bool, bool, int, size_t);
int occupancy_n7(bool, bool, int, size_t);
int occupancy_n8(bool, bool, int, size_t);

}  // namespace amfrw
