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
constexpr int kCtaMaxThreads = 256;  // CTA work groups (grids of more than 64 Inner nodes)

// Per-instance parameters on the device (one per pricing problem).
struct InstDev {
    int32_t N, payoff, n_steps, precision;
    int32_t grid_begin, grid_count;
    int32_t bc;          // 0: Neumann upper faces (Sketch 1); 1: Dirichlet rate faces (eq. bound1_0)
    int32_t pad1;
    double alpha[kMaxDim], phi[kMaxDim], tau[kMaxDim], F0[kMaxDim];
    double Fmax[kMaxDim];          // Fmax[N-1] = V^max
    double rho[kMaxDim * kMaxDim];  // rate correlations, leading dimension 8
    double sigma, beta, V0, K, T, discount, theta, nu, dt;
    double pad2;
    // The level-free factors of a grid's constants, computed once per
    // instance: h_i = Fmax_i 2^-l_i exactly, so every constant of a grid is
    // one of these times an exact power of two (the same FP64 value as
    // dividing by the grid's h directly).
    double cVb;                                // sigma^2 / (2 Vmax^2), times 4^l_V
    double dcb[kMaxDim];                       // alpha_a^2 rho_aa / (2 Fmax_a^2), times 4^l_a
    double rmb[kMaxDim * (kMaxDim - 1) / 2];   // rho_ik / (4 Fmax_i Fmax_k), times 2^(l_i + l_k)
    double smb[kMaxDim];                       // sigma phi_i / (4 Fmax_i Vmax), times 2^(l_i + l_V)
    double g2b[kMaxDim];                       // 1 / (2 Fmax_i), times 2^l_i
    double xs[kMaxDim];                        // spot over Fmax: F_i(0) / Fmax_i, V0 / Vmax (times M_i: x*/h_i)
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
    int32_t meta, cd, cf, tabd, tabf, pay, lu, Z, ZZ, H, DR, FY, K1, K0, Kw, D, C, scr, total;
    // CTA groups: bytes of the block's slice of global scratch (line-solve
    // factors, and in mixed precision Z and dt F(Y_n) at offsets gZ, gFY)
    int32_t gbytes, gZ, gFY;
    int32_t L, Lp, Lr, ntab, npay, nlu, ncoef;
};

// Per-node coefficients of the difference-array stencil (FP64 warp groups):
// N diagonal, 1 centre, N(N-1)/2 cross, N-2 drift, 1 for dt F(payoff).
AMFRW_HD int node_coefs(int N) { return N + 1 + N * (N - 1) / 2 + (N - 2) + 1; }

// Packed index of the pair (i, k), i < k < 8, and of (i, r), r <= i < 8.
AMFRW_HD int upair(int i, int k) { return i * (2 * kMaxDim - i - 1) / 2 + (k - i - 1); }
AMFRW_HD int ltri(int i, int r) { return i * (i + 1) / 2 + r; }

template <typename T>
struct Consts {
    T cV;                 // sigma^2 / (2 h_V^2)
    T dt, thdt, nudt;     // dt, theta*dt, nu*dt
    T rm[kMaxDim * (kMaxDim - 1) / 2];  // rho_ik / (4 h_i h_k), rate pairs i < k (upair)
    T rh[kMaxDim * (kMaxDim + 1) / 2];  // rho_ir for the drift sums, r <= i (ltri)
    T sm[kMaxDim];                      // sigma phi_i / (4 h_i h_V)
    T g2[kMaxDim];                      // 1 / (2 h_i)
};

// Active axes of a grid (those with more than one Inner row) for the
// mixed-precision stencil, built once per grid in shared memory.
// One active axis: read by the stencil as two 16-byte loads.
struct alignas(16) ActAxis {
    int sh;       // bit offset of j - 1 in the node index t
    int msk;      // M - 1
    int nfm;      // j - 1 of the Neumann face, or -2 (Dirichlet data on the upper face)
    int Sp;       // padded stride
    int toff;     // rate axes: offset of their coefficient tables (d, pw, drift)
    int M;        // rows
    int drift;    // 1: rate axis with a drift term (rates 2..N-1)
    int dslot;    // warp groups: its slot in the per-node drift coefficients
};

struct ActAxes {
    int n;                      // active axes, ascending axis order
    int nr;                     // active rate axes (the first nr of them; V, if active, is last)
    float cinact;               // second-difference coefficients of the inactive axes, summed
    int ns;                     // directional solves of a stage (the axes not folded into another)
    ActAxis rec[kMaxDim];
    int ax[kMaxDim];            // the axis index
    float g2[kMaxDim];          // 1 / (2 h) (drift gradient)
    float sconst[kMaxDim];      // drift sum: the part of the inactive rates
    float cx[kMaxDim][kMaxDim]; // pair (q, r), q < r: rho/(4 h h) (two rates) or sigma phi/(4 h h_V)
    float drh[kMaxDim][kMaxDim];// drift of active rate q: rho for the active rates r <= q
    // the solves in ascending axis order, read as one 8-byte load each:
    // [2q] offset of the axis's factors; [2q + 1] sh | M << 8 | axis << 16 |
    // (rate axis) << 24 | (solved by its explicit inverse) << 25
    alignas(8) int sv[2 * kMaxDim];
};

// Per-grid descriptors the mixed-precision solver keeps in shared memory:
// the grid's shape (10 per-axis arrays and 8 scalars of int) and its active
// axes.  Warp groups hold them in their layout; whole-block groups in a
// static shared array of the kernel.
AMFRW_HD constexpr int32_t align16(int32_t x) { return (x + 15) & ~15; }
AMFRW_HD constexpr int shape_bytes(int N) { return align16(4 * (10 * N + 8)); }
AMFRW_HD constexpr int meta_bytes(int N) { return shape_bytes(N) + align16((int)sizeof(ActAxes)); }
constexpr int kMetaBytesMax = meta_bytes(kMaxDim);

// Work-group kinds.  kWarpGroup: a grid of at most 64 Inner nodes on (part
// of) one warp, everything in shared memory.  kCtaGroup: one CTA per grid,
// the grid in shared memory, line-solve factors in a global scratch slice.
// kMemGroup: one CTA per grid with the whole grid state in its block's slice
// of global scratch (L2/HBM resident): grids too large for shared memory or
// with lines of more than 256 rows.
constexpr int kWarpGroup = 0;
constexpr int kCtaGroup = 1;
constexpr int kMemGroup = 2;

// Rows of a line per lane in a line solve: at most 2 for warp groups (grids of
// at most 64 Inner nodes), at most 8 for FP64 CTA groups and 4 for
// mixed-precision ones (rows held in registers; mixed-precision CTA groups
// run two blocks per SM, so 128 registers a thread), hence lines of at most
// 256 / 128 rows there; unbounded for global-memory groups (rows streamed
// from memory).
constexpr int kRowsLogWarp = 1;
constexpr int kRowsLogCta = 3;
constexpr int kRowsLogCtaMixed = 2;
constexpr int kRowsLogMem = 24;
AMFRW_HD int rows_log(int kind, bool mixed = false)
{
    return kind == kWarpGroup ? kRowsLogWarp
                              : (kind == kCtaGroup ? (mixed ? kRowsLogCtaMixed : kRowsLogCta) : kRowsLogMem);
}

// Lanes per line (as log2) for the directional solves along an axis with
// 2^mlog rows, on a grid of 2^llog Inner nodes solved by a group of 2^tlog
// threads: enough lanes that the whole group is busy, at most 2^rlog rows per
// lane, at most 32 lanes (one warp) and at most one row per lane.
AMFRW_HD int lanes_log(int mlog, int llog, int tlog, int rlog)
{
    int p = tlog + mlog - llog;
    if (p < mlog - rlog) p = mlog - rlog;
    if (p < 0) p = 0;
    if (p > mlog) p = mlog;
    if (p > 5) p = 5;
    return p;
}

// Values stored per matrix row for an axis solved with 2^plog lanes per line:
// PCR multipliers (alpha, gamma) of each level, then the Thomas factors
// (lower, 1/pivot, upper/pivot) of the reduced interleaved systems.
AMFRW_HD int lu_row_values(int plog) { return 2 * plog + 3; }

// Mixed-precision warp groups hold a grid's values in registers (at most two
// nodes per lane) and solve the lines of an axis of 2..8 rows by the explicit
// inverse of its directional matrix: M values per matrix row, the rows of a
// line exchanged by shuffles.  Their offsets are kept 16-byte aligned for
// vector loads.
constexpr int kDenseMaxRows = 8;
AMFRW_HD bool dense_axis(int kind, bool mixed, int M)
{
    return mixed && kind == kWarpGroup && M >= 2 && M <= kDenseMaxRows;
}

// Rows of axis 0 get one padding slot each (lines along axis 0 then start in
// different banks) when they have at least this many nodes.  Mixed-precision
// CTA groups pad only rows of 4 or more, which keeps a 4096-node grid within
// half an SM's shared memory (two resident CTAs); the others pad every row of
// 2 or more.
AMFRW_HD int pad_rows_min(bool lean) { return lean ? 4 : 2; }

// kind: the work-group kind.  Warp and global-memory groups keep the
// line-solve factors inside the layout; CTA groups in the group's slice of a
// global scratch array.  Global-memory groups also get FP64 scratch for the
// factorisation (three values per matrix row of the largest axis).  tlog:
// log2 of the group's thread count.
AMFRW_HD Layout make_layout(int N, const int8_t* lv, bool mixed, int kind, int tlog)
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
    const bool lean = mixed && kind == kCtaGroup;
    const int pad = M0 >= pad_rows_min(lean) ? 1 : 0;
    y.L = L;
    y.Lp = L + (pad ? (L >> lv[0]) : 0);
    y.Lr = L >> lv[N - 1];
    y.ntab = 3 * sumM + MV;
    y.npay = 2 * npay;
    int llog = 0;
    for (int i = 0; i < N; ++i) llog += lv[i];
    // Mixed-precision warp groups fold the single-row axes into another
    // axis's solve (all rate axes of one row; the V axis of one row when a
    // rate axis has more) and store no factors for them.
    const bool dense = mixed && kind == kWarpGroup;
    bool rate_rows = false;
    for (int i = 0; i < N - 1; ++i) rate_rows |= lv[i] > 0;
    int nlu = 0;
    for (int i = 0; i < N; ++i) {
        const int rows = (i < N - 1 ? MV : 1) << lv[i];  // classes x rows
        if (dense && lv[i] == 0 && (i < N - 1 || rate_rows)) continue;
        if (dense_axis(kind, mixed, 1 << lv[i])) {
            nlu = (nlu + 3) & ~3;
            nlu += rows << lv[i];
        } else {
            nlu += rows * lu_row_values(lanes_log(lv[i], llog, tlog, rows_log(kind, mixed)));
        }
    }
    const bool lu_in = kind != kCtaGroup;
    y.nlu = nlu;
    const int sk = mixed ? 4 : 8;  // bytes of a factor value
    int o = 0;
    if (mixed) {
        // The FP64 constants and tables serve the per-grid setup only (tables,
        // line-solve factors, F of the payoff); the time loop reads their FP32
        // copies.  They share one region with the time loop's vectors.
        y.meta = o; o = align16(o + (kind == kWarpGroup ? meta_bytes(N) : 0));
        y.cf = o;   o = align16(o + (int)sizeof(Consts<float>));
        y.tabf = o; o = align16(o + 4 * y.ntab);
        y.pay = o;  o = align16(o + 8 * y.npay);
        y.lu = o;   o = align16(o + (lu_in ? 4 * y.nlu : 0));
        y.Z = o;    o = align16(o + (lean ? 0 : 8 * y.Lp));
        y.ZZ = o;   o = align16(o + 8 * y.Lp);
        y.H = o;    o = align16(o + 4 * y.Lr);
        // warp groups: per node, the drift coefficient of every refined rate
        // axis 2..N-1 (it depends on the node only, and the time loop would
        // otherwise re-sum it at every F evaluation)
        int ndrift = 0;
        for (int i = 1; i < N - 1; ++i) ndrift += lv[i] > 0 ? 1 : 0;
        y.DR = o;   o = align16(o + (kind == kWarpGroup ? 4 * ndrift * y.Lp : 0));
        int a = o, b = o;
        y.cd = a;   a = align16(a + (int)sizeof(Consts<double>));
        y.tabd = a; a = align16(a + 8 * y.ntab);
        y.FY = b;   b = align16(b + (lean ? 0 : 4 * y.Lp));
        y.K1 = b;   b = align16(b + 4 * y.Lp);
        y.K0 = b;   b = align16(b + 4 * y.Lp);
        y.Kw = b;   b = align16(b + 4 * y.Lp);
        o = a > b ? a : b;
        y.ncoef = 0;
        y.D = o;
        y.C = o;
    } else {
        y.meta = o;
        y.cd = o;   o = align16(o + (int)sizeof(Consts<double>));
        y.cf = o;
        y.tabd = o; o = align16(o + 8 * y.ntab);
        y.tabf = o;
        y.pay = o;  o = align16(o + 8 * y.npay);
        y.lu = o;   o = align16(o + (lu_in ? 8 * y.nlu : 0));
        y.Z = o;    o = align16(o + 8 * y.Lp);
        y.ZZ = o;
        y.H = o;    o = align16(o + 8 * y.Lr);
        y.DR = o;
        y.FY = o;
        y.K1 = o;   o = align16(o + 8 * y.Lp);
        y.K0 = o;   o = align16(o + 8 * y.Lp);
        y.Kw = o;   o = align16(o + 8 * y.Lp);
        // FP64 warp groups: central differences per axis and per-node coefficients
        const bool diff = kind == kWarpGroup;
        y.ncoef = diff ? node_coefs(N) : 0;
        y.D = o;    o = align16(o + (diff ? 8 * N * y.Lp : 0));
        y.C = o;    o = align16(o + 8 * y.ncoef * y.Lp);
    }
    int rmax = 0;
    for (int i = 0; i < N; ++i) {
        const int rows = (i < N - 1 ? MV : 1) << lv[i];
        rmax = rows > rmax ? rows : rmax;
    }
    y.scr = o;  o = align16(o + (kind == kMemGroup ? 3 * 8 * rmax : 0));
    y.total = o;
    // the global slice of a CTA group: factors, then (mixed) Z and dt F(Y_n)
    y.gbytes = y.gZ = y.gFY = 0;
    if (kind == kCtaGroup) {
        int g = (nlu * sk + 255) & ~255;
        if (lean) {
            y.gZ = g;   g += (8 * y.Lp + 255) & ~255;
            y.gFY = g;  g += (4 * y.Lp + 255) & ~255;
        }
        y.gbytes = g;
    }
    return y;
}

// One grid class of a warp-group launch: grids of one size solved by work
// groups of 2^glog lanes (several groups per warp when glog < 5).
struct ClassDesc {
    int32_t glog, item_begin, item_count, smem_group, qidx, pad;  // qidx: its work counter
};

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
    // warp groups: the classes of this launch, walked in order by every warp
    const ClassDesc* classes;
    int32_t n_classes;
    int32_t smem_warp;    // dynamic shared bytes per warp
    // instances to solve (nonzero entries), or null for all: the FP64
    // re-solve of ill-conditioned mixed-precision instances skips the others
    const int32_t* inst_mask;
};

constexpr int kLoadState = 1;
constexpr int kStoreState = 2;

// Host-side launchers, one translation unit per dimension N.
using LaunchFn = int (*)(const SolveArgs&, bool mixed, int kind, int block, int grid,
                         size_t smem, void* stream);
int launch_n2(const SolveArgs&, bool, int, int, int, size_t, void*);
int launch_n3(const SolveArgs&, bool, int, int, int, size_t, void*);
int launch_n4(const SolveArgs&, bool, int, int, int, size_t, void*);
int launch_n5(const SolveArgs&, bool, int, int, int, size_t, void*);
int launch_n6(const SolveArgs&, bool, int, int, int, size_t, void*);
int launch_n7(const SolveArgs&, bool, int, int, int, size_t, void*);
int launch_n8(const SolveArgs&, bool, int, int, int, size_t, void*);
// Occupancy query for the same instantiation (blocks per SM).
int occupancy(int N, bool mixed, int kind, int block, size_t smem);
using OccFn = int (*)(bool mixed, int kind, int block, size_t smem);
int occupancy_n2(bool, int, int, size_t);
int occupancy_n3(bool, int, int, size_t);
int occupancy_n4(bool, int, int, size_t);
int occupancy_n5(bool, int, int, size_t);
int occupancy_n6(bool, int, int, size_t);
int occupancy_n7(bool, int, int, size_t);
int occupancy_n8(bool, int, int, size_t);

}  // namespace amfrw
