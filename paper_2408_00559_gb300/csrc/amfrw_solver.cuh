// AMFR-W2 solver for one sparse-grid component grid, resident in shared
// memory for the whole time integration.
//
// A work group (one warp, or a whole CTA for large grids) takes a component
// grid from a queue, builds its coefficient and line-solve tables, sets the
// grid to the payoff, runs every AMFR-W2 step on chip and writes the value
// interpolated at the spot.  HBM traffic per grid is the parameter record in
// and one double out.
//
// Storage.  Only the Inner nodes (all j_i >= 1, Sec. 3) are stored, in the
// paper's lexicographic order with axis 0 fastest, plus one padding slot per
// axis-0 row so that lines along axis 0 handled by consecutive lanes fall in
// different shared-memory banks.  The grid function is split as Y = G + Z,
// where G is the payoff on every node (Inner and Outer) and Z vanishes on the
// Outer nodes (they keep the Dirichlet data, Y' = 0 there).  Because F is
// linear (end of Sec. 4.1), F(Y) = F(G) + F_0(Z), where F_0 is Sketch 1 with
// zero Outer values, and F(G) is computed once per grid in FP64.  The payoff
// does not depend on V and every coefficient carries the factor V^2, so
// F(G) = V^2 H(F_1..F_{N-1}) and only H is stored.
//
// Time stepping follows eq. (amfrw) with the AMFR-W2 coefficients of eq.
// (coef_W2):  per stage an F evaluation, N directional solves (Lemma ls),
// the refinement Khat = 2K^(0) - K^(N) + theta dt F(K^(N)), and N solves.
// The directional matrices (I - nu dt A_i) do not change in time, so their
// Thomas factors are computed once per grid: for a rate axis they depend on
// the V index only (d_i = 1/2 alpha_i^2 F_i^{2 beta} V^2), for the V axis on
// nothing else.
//
// Precision.  FP64 mode: every operation in double.  Mixed mode: the stencil
// and the line solves run in FP32 on the increments K; Z is accumulated in
// FP64 (Y_{n+1} = Y_n + b1 K1 + b2 K2) and the stencil of F(Y_n) reads Z as
// an unevaluated pair of floats (hi + lo), so its differences keep ~48 bits;
// F(G) (through H), the interpolation and the combination sum are FP64.  The
// stage-2 argument uses linearity, F(Y_n + a21 K1) = F(Y_n) + a21 F_0(K1), so
// that F is applied to Y only once per step.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "amfrw_internal.h"

namespace amfrw {

// Resident blocks of 128 threads per SM the mixed-precision warp kernels are
// compiled for (it caps their registers).
constexpr int kWarpBlocksMixed = 4;
constexpr double kA21 = 2.0 / 3.0;   // eq. (coef_W2)
constexpr double kQ21 = -4.0 / 3.0;
constexpr double kB1 = 5.0 / 4.0;
constexpr double kB2 = 3.0 / 4.0;

template <int N>
struct Shape {
    int lv[N], M[N], sh[N], Sp[N];
    int nf[N];     // j of the Neumann face of the axis (Sketch 1), or -1 where eq. bound1_0
                   // puts Dirichlet data on the upper face (rate axes)
    int dmask;     // rate axes with Dirichlet data on their upper face
    int toff[N];   // coefficient tables: rate axis a -> [dI | pw | ph] of M_a each; V -> v2
    int poff[N];   // payoff tables: rate axis a -> M_a + 1 entries (Outer node included)
    int luoff[N];  // line-solve factors: rate axis -> M_V classes x M_a rows; V -> M_V rows
    int plog[N];   // log2 lanes per line in the directional solves
    int luS[N];    // factor values per matrix row (2 plog + 3)
    int L, Lr, pad, phalf;
    int skip;      // axes whose single-row solves are folded into the solve along `last`
    int last;      // the last axis solved in a stage (carries the stage's epilogue)
    int dense;     // axes solved by the explicit inverse of their directional matrix
    __device__ __forceinline__ int padded(int t) const { return t + pad * (t >> lv[0]); }
};

template <int N>
__device__ __forceinline__ void make_shape(Shape<N>& s, const int8_t* lv, int tlog, int rlog, bool fold,
                                           bool fold_v, bool dirichlet, bool dense = false, int padmin = 2)
{
    int sh = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        s.lv[i] = lv[i];
        s.M[i] = 1 << lv[i];
        s.sh[i] = sh;
        s.nf[i] = (dirichlet && i < N - 1) ? -1 : s.M[i];
        sh += lv[i];
    }
    s.dmask = dirichlet ? (1 << (N - 1)) - 1 : 0;
    s.L = 1 << sh;
    s.Lr = s.L >> s.lv[N - 1];
    s.pad = s.M[0] >= padmin ? 1 : 0;  // (make_layout's rule: pad_rows_min)
    int r = s.M[0] + s.pad;
    s.Sp[0] = 1;
#pragma unroll
    for (int i = 1; i < N; ++i) {
        s.Sp[i] = r;
        r *= s.M[i];
    }
    int o = 0, po = 0, lo = 0;
#pragma unroll
    for (int i = 0; i < N - 1; ++i) {
        s.toff[i] = o;
        o += 3 * s.M[i];
        s.poff[i] = po;
        po += s.M[i] + 1;
    }
    s.toff[N - 1] = o;
    s.poff[N - 1] = po;
    s.phalf = po;
    s.skip = 0;
    s.last = N - 1;
    int lastr = -1;  // the last rate axis with more than one row
#pragma unroll
    for (int i = 0; i < N - 1; ++i) {
        if (fold && s.M[i] == 1) s.skip |= 1 << i;
        if (s.M[i] > 1) lastr = i;
    }
    if (fold && fold_v && s.M[N - 1] == 1 && lastr >= 0) {
        s.skip |= 1 << (N - 1);
        s.last = lastr;
    }
    s.dense = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        // (the same sizes as make_layout's line-solve region; with `dense`
        // the folded single-row axes, never solved on their own, get none)
        const bool dn = dense && s.M[i] >= 2 && s.M[i] <= kDenseMaxRows;
        s.plog[i] = lanes_log(s.lv[i], sh, tlog, rlog);
        s.luS[i] = dn ? s.M[i] : lu_row_values(s.plog[i]);
        if (dn) {
            s.dense |= 1 << i;
            lo = (lo + 3) & ~3;
        }
        s.luoff[i] = lo;
        if (!(dense && ((s.skip >> i) & 1))) lo += ((i < N - 1 ? s.M[N - 1] : 1) << s.lv[i]) * s.luS[i];
    }
}

// Under eq. bound1_0 the nodes on the upper face of a rate axis hold
// Dirichlet data: they are stored (Z = 0 there, as on the lower faces) but
// are not Inner nodes, so every increment is 0 on them.
template <int N>
__device__ __forceinline__ bool dirichlet_node(const Shape<N>& s, int t)
{
    bool out = false;
    if (s.dmask) {
#pragma unroll
        for (int i = 0; i < N - 1; ++i) out |= ((t >> s.sh[i]) & (s.M[i] - 1)) == s.M[i] - 1;
    }
    return out;
}

template <int N>
__device__ __forceinline__ void decode(const Shape<N>& s, int t, int (&j)[N])
{
#pragma unroll
    for (int i = 0; i < N; ++i) j[i] = ((t >> s.sh[i]) & (s.M[i] - 1)) + 1;
}

// ------------------------------------------------------------------ sources
// A source supplies the grid values the stencil reads.  nb() gets both the
// shared-memory offset of the neighbour and its multi-index displacement;
// each source uses what it needs.

template <typename T>
struct ArrSrc {  // stored increments or Z: zero on Outer nodes
    using V = T;
    const T* X;
    __device__ __forceinline__ V ctr(int J) const { return X[J]; }
    __device__ __forceinline__ V nb(int J, int off, bool valid, int, int, int, int) const
    {
        return valid ? X[J + off] : T(0);
    }
    __device__ static __forceinline__ T diff(V a, V b) { return a - b; }
    __device__ static __forceinline__ T val(V a) { return a; }
};

struct DFSrc {  // Z as an unevaluated float pair hi + lo
    using V = float2;
    const float2* X;
    __device__ __forceinline__ V ctr(int J) const { return X[J]; }
    __device__ __forceinline__ V nb(int J, int off, bool valid, int, int, int, int) const
    {
        return valid ? X[J + off] : make_float2(0.f, 0.f);
    }
    // hi parts of nearby values are close, so hi_a - hi_b is (nearly) exact
    __device__ static __forceinline__ float diff(V a, V b) { return (a.x - b.x) + (a.y - b.y); }
    __device__ static __forceinline__ float val(V a) { return a.x + a.y; }
};

// Payoff g at rate multi-index jj (Sec. 2).  Caplet: (F_1 - K)^+.
// Swaption: max{ sum_i tau_i (F_i - K) prod_{l<=i} 1/(1 + tau_l F_l), 0 }.
template <int N>
__device__ __forceinline__ double payoff_at(const int (&poff)[N], int phalf, const double* pay,
                                            int payoff, const int (&jj)[N])
{
    if (payoff == 0) return fmax(pay[poff[0] + jj[0]], 0.0);
    double sum = 0.0, P = 1.0;
#pragma unroll
    for (int r = 0; r < N - 1; ++r) {
        P *= pay[phalf + poff[r] + jj[r]];
        sum = fma(pay[poff[r] + jj[r]], P, sum);
    }
    return fmax(sum, 0.0);
}

template <int N>
__device__ __forceinline__ double payoff_at(const Shape<N>& s, const double* pay, int payoff,
                                            const int (&jj)[N])
{
    return payoff_at<N>(s.poff, s.phalf, pay, payoff, jj);
}

// -------------------------------------------------------------- the stencil
// Sketch 1 at the Inner node with multi-index j, divided by V^2 (every
// coefficient of eqs. coef_diff, coef_mix, coef_adv carries F_N^2 = V^2):
//   sum_i d_i/V^2 Delta^(i) + sum_{i<k} m_ik/V^2 Delta^(ik) + sum_i a_i/V^2 nabla^(i)
// with the Neumann rules of Sketch 1 on the upper faces (ghost node
// Y_{J+E_i} = Y_{J-E_i}, zero first and mixed differences).  The 1/h factors
// are folded into the tables.
template <int N, typename TC, class Src>
__device__ __forceinline__ TC stencil_acc(const Shape<N>& s, const int (&j)[N], int J,
                                          const Src& src, const TC* __restrict__ tab,
                                          const Consts<TC>& c)
{
    using V = typename Src::V;
    const V x0 = src.ctr(J);
    TC lap[N], grad[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const bool has_lo = j[i] > 1;
        const bool top = j[i] == s.nf[i];
        const V m = src.nb(J, -s.Sp[i], has_lo, i, -1, -1, 0);
        const V p = top ? m : src.nb(J, s.Sp[i], true, i, 1, -1, 0);
        const TC dp = Src::diff(p, x0);
        const TC dm = Src::diff(x0, m);
        lap[i] = dp - dm;
        grad[i] = top ? TC(0) : dp + dm;
    }
    TC acc = c.cV * lap[N - 1];
#pragma unroll
    for (int i = 0; i < N - 1; ++i) acc += tab[s.toff[i] + j[i] - 1] * lap[i];
#pragma unroll
    for (int i = 0; i < N - 1; ++i) {
        // cross and drift terms of rate i: zero on its upper (Neumann) face
        if (j[i] != s.nf[i]) {
            TC inner = TC(0);
            const bool li = j[i] > 1;
#pragma unroll
            for (int k = i + 1; k < N; ++k) {
                if (j[k] != s.nf[k]) {
                    const bool lk = j[k] > 1;
                    const V pp = src.nb(J, s.Sp[i] + s.Sp[k], true, i, 1, k, 1);
                    const V pm = src.nb(J, s.Sp[i] - s.Sp[k], lk, i, 1, k, -1);
                    const V mp = src.nb(J, -s.Sp[i] + s.Sp[k], li, i, -1, k, 1);
                    const V mm = src.nb(J, -s.Sp[i] - s.Sp[k], li && lk, i, -1, k, -1);
                    const TC mix = Src::diff(pp, pm) - Src::diff(mp, mm);
                    const TC ck = (k < N - 1) ? c.rm[upair(i, k)] * tab[s.toff[k] + s.M[k] + j[k] - 1]
                                              : c.sm[i];
                    inner += ck * mix;
                }
            }
            if (i >= 1) {  // drift of rates 2..N-1 (eq. coef_adv), sum over rates 2..i
                TC S = TC(0);
#pragma unroll
                for (int r = 1; r <= i; ++r) S += c.rh[ltri(i, r)] * tab[s.toff[r] + 2 * s.M[r] + j[r] - 1];
                inner += S * c.g2[i] * grad[i];
            }
            acc += tab[s.toff[i] + s.M[i] + j[i] - 1] * inner;
        }
    }
    return acc;
}

// ------------------------------------------------- the stencil of the payoff
// H = F(G)/V^2 at the rate multi-index j: Sketch 1 applied to the payoff G,
// computed once per grid in FP64.  G does not depend on V, so every term that
// differentiates along V vanishes and is skipped; the remaining terms use the
// same coefficients, Neumann reflections and upper-face rules as stencil_acc.
// A neighbour differs from the centre in one or two rates, so its swaption
// payoff sum_r a_r prod_{l<=r} b_l (a_r = tau_r (F_r - K),
// b_r = 1/(1 + tau_r F_r)) starts from the centre's partial product and sum
// just before the first changed rate and finishes the same forward loop as
// payoff_at: every value is bitwise the one payoff_at gives (second
// differences over fine axes amplify any rounding difference by 1/h^2), at a
// fraction of the cost.
template <int N>
__device__ __noinline__ double payoff_H(const Shape<N>& s, const double* pay, int payoff, const int (&j)[N],
                                        const double* __restrict__ tab, const Consts<double>& c)
{
    constexpr int n = N - 1;  // rate axes
    const double* A = pay;
    const double* Bv = pay + s.phalf;
    if (payoff == 0) {  // caplet: G = (F_1 - K)^+ depends on rate 1 only
        const int o = s.poff[0] + j[0];
        const double x0 = fmax(A[o], 0.0);
        const double m = fmax(A[o - 1], 0.0);
        const double p = (j[0] == s.nf[0]) ? m : fmax(A[o + 1], 0.0);
        return tab[s.toff[0] + j[0] - 1] * ((p - x0) - (x0 - m));
    }
    double a[n], b[n], P0[n], S0[n];  // P0[r], S0[r]: product and sum before rate r
    double P = 1.0, S = 0.0;
#pragma unroll
    for (int r = 0; r < n; ++r) {
        a[r] = A[s.poff[r] + j[r]];
        b[r] = Bv[s.poff[r] + j[r]];
        P0[r] = P;
        S0[r] = S;
        P *= b[r];
        S = fma(a[r], P, S);
    }
    const double x0 = fmax(S, 0.0);
    // payoff with rate i at table offset oi (and rate k > i at ok; k < 0: none)
    auto g = [&](int i, int oi, int k, int ok) {
        double p = P0[i] * Bv[oi];
        double q = fma(A[oi], p, S0[i]);
#pragma unroll
        for (int r = 0; r < n; ++r) {
            if (r <= i) continue;
            const bool ch = r == k;
            p *= ch ? Bv[ok] : b[r];
            q = fma(ch ? A[ok] : a[r], p, q);
        }
        return fmax(q, 0.0);
    };
    double lap[n], grad[n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const int o = s.poff[i] + j[i];
        const bool top = j[i] == s.nf[i];
        const double m = g(i, o - 1, -1, 0);
        const double p = top ? m : g(i, o + 1, -1, 0);
        const double dp = p - x0;
        const double dm = x0 - m;
        lap[i] = dp - dm;
        grad[i] = top ? 0.0 : dp + dm;
    }
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < n; ++i) acc += tab[s.toff[i] + j[i] - 1] * lap[i];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        double inner = 0.0;
        if (j[i] != s.nf[i]) {
            const int oi = s.poff[i] + j[i];
#pragma unroll
            for (int k = i + 1; k < n; ++k) {
                if (j[k] != s.nf[k]) {
                    const int ok = s.poff[k] + j[k];
                    const double pp = g(i, oi + 1, k, ok + 1);
                    const double pm = g(i, oi + 1, k, ok - 1);
                    const double mp = g(i, oi - 1, k, ok + 1);
                    const double mm = g(i, oi - 1, k, ok - 1);
                    const double mix = (pp - pm) - (mp - mm);
                    inner += c.rm[upair(i, k)] * tab[s.toff[k] + s.M[k] + j[k] - 1] * mix;
                }
            }
        }
        if (i >= 1) {  // drift of rates 2..N-1 (eq. coef_adv), sum over rates 2..i
            double Sd = 0.0;
#pragma unroll
            for (int r = 1; r <= i; ++r) Sd += c.rh[ltri(i, r)] * tab[s.toff[r] + 2 * s.M[r] + j[r] - 1];
            inner += Sd * c.g2[i] * grad[i];
        }
        acc += tab[s.toff[i] + s.M[i] + j[i] - 1] * inner;
    }
    return acc;
}

// The same H for the mixed-precision mode, with every neighbour's payoff in
// O(1) instead of resuming the forward loop: with the centre's prefix
// P0[r] = prod_{l<r} b_l, S0[r] = sum_{m<r} a_m prod_{l<=m} b_l and suffix
// T[r] = b_r (a_r + T[r+1]) (so that S = S0[r] + P0[r] T[r] for every r), a
// neighbour that changes rate i to (a', b') has S' = S0[i] + P0[i] b' (a' +
// T[i+1]); one that also changes rate k > i has T[i+1] replaced by
// U_ik + Q_ik b_k' (a_k' + T[k+1]), with Q_ik = prod_{i<l<k} b_l and
// U_ik = sum_{i<m<k} a_m prod_{i<l<=m} b_l built up as k grows.  The sums are
// associated differently from payoff_at, which moves H by a few ulps: far
// below the FP32 rounding of the mode, and not used by the FP64 mode.
template <int N>
__device__ __noinline__ float payoff_H_fast(const Shape<N>& s, const double* pay, int payoff, const int (&j)[N],
                                            const float* __restrict__ tab, const Consts<float>& c)
{
    constexpr int n = N - 1;  // rate axes
    const double* A = pay;
    if (payoff == 0) {  // caplet: G = (F_1 - K)^+ depends on rate 1 only
        const int o = s.poff[0] + j[0];
        const double x0 = fmax(A[o], 0.0);
        const double m = fmax(A[o - 1], 0.0);
        const double p = (j[0] == s.nf[0]) ? m : fmax(A[o + 1], 0.0);
        return tab[s.toff[0] + j[0] - 1] * (float)((p - x0) - (x0 - m));
    }
    const double* Bv = pay + s.phalf;
    double a[n], b[n], P0[n], S0[n], T[n + 1];
    double P = 1.0, S = 0.0;
#pragma unroll
    for (int r = 0; r < n; ++r) {
        a[r] = A[s.poff[r] + j[r]];
        b[r] = Bv[s.poff[r] + j[r]];
        P0[r] = P;
        S0[r] = S;
        P *= b[r];
        S = fma(a[r], P, S);
    }
    T[n] = 0.0;
#pragma unroll
    for (int r = n - 1; r >= 0; --r) T[r] = b[r] * (a[r] + T[r + 1]);
    const double x0 = fmax(S, 0.0);
    // differences of payoffs in FP64 (they cancel), their coefficients in FP32
    float lap[n], grad[n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const int o = s.poff[i] + j[i];
        const bool top = j[i] == s.nf[i];
        const double m = fmax(fma(P0[i] * Bv[o - 1], A[o - 1] + T[i + 1], S0[i]), 0.0);
        const double p = top ? m : fmax(fma(P0[i] * Bv[o + 1], A[o + 1] + T[i + 1], S0[i]), 0.0);
        const double dp = p - x0;
        const double dm = x0 - m;
        lap[i] = (float)(dp - dm);
        grad[i] = top ? 0.f : (float)(dp + dm);
    }
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < n; ++i) acc += tab[s.toff[i] + j[i] - 1] * lap[i];
    int kend = -1;  // the last rate off its upper face: no cross term lies beyond it
#pragma unroll
    for (int k = 0; k < n; ++k)
        if (j[k] != s.nf[k]) kend = k;
#pragma unroll
    for (int i = 0; i < n; ++i) {
        float inner = 0.f;
        if (j[i] != s.nf[i]) {
            const int oi = s.poff[i] + j[i];
            // a corner's payoff is S0[i] + c (a_i' + w) with c = P0[i] b_i' of
            // rate i's neighbour row: S0[i] + c a_i' is formed once per rate i
            const double cp = P0[i] * Bv[oi + 1], cm = P0[i] * Bv[oi - 1];
            const double sp = fma(cp, A[oi + 1], S0[i]), sm = fma(cm, A[oi - 1], S0[i]);
            double Q = 1.0, U = 0.0;  // Q_ik, U_ik for the current k
#pragma unroll
            for (int k = i + 1; k < n; ++k) {
                if (k > kend) break;
                if (j[k] != s.nf[k]) {
                    const int ok = s.poff[k] + j[k];
                    const double wp = U + Q * Bv[ok + 1] * (A[ok + 1] + T[k + 1]);
                    const double wm = U + Q * Bv[ok - 1] * (A[ok - 1] + T[k + 1]);
                    const double pp = fmax(fma(cp, wp, sp), 0.0);
                    const double pm = fmax(fma(cp, wm, sp), 0.0);
                    const double mp = fmax(fma(cm, wp, sm), 0.0);
                    const double mm = fmax(fma(cm, wm, sm), 0.0);
                    const float mix = (float)((pp - pm) - (mp - mm));
                    inner += c.rm[upair(i, k)] * tab[s.toff[k] + s.M[k] + j[k] - 1] * mix;
                }
                Q *= b[k];
                U = fma(a[k], Q, U);
            }
        }
        if (i >= 1) {  // drift of rates 2..N-1 (eq. coef_adv), sum over rates 2..i
            float Sd = 0.f;
#pragma unroll
            for (int r = 1; r <= i; ++r) Sd += c.rh[ltri(i, r)] * tab[s.toff[r] + 2 * s.M[r] + j[r] - 1];
            inner += Sd * c.g2[i] * grad[i];
        }
        acc += tab[s.toff[i] + s.M[i] + j[i] - 1] * inner;
    }
    return acc;
}

// ------------------------------------------- difference-array stencil
// FP64 warp groups evaluate Sketch 1 in two passes.  Pass 1 stores, per
// axis k, the central difference D_k = X(J+E_k) - X(J-E_k) (zero on Outer
// nodes and, by the ghost node Y_{J+E_k} = Y_{J-E_k}, zero on the upper face
// of axis k).  Pass 2 combines, with per-node coefficients computed once per
// grid (every coefficient of eqs. coef_diff/mix/adv carries V^2, folded in,
// and so is the time step, so that pass 2 gives dt F_0 and can start from the
// stage's other terms):
//   F_0(X)_J = sum_i d_i/h_i^2 (X+_i + X-_i) - 2 sum_i d_i/h_i^2 X_J
//            + sum_{i<k} m_ik/(4 h_i h_k) (D_k(J+E_i) - D_k(J-E_i))
//            + sum_i a_i/(2 h_i) D_i(J)
// with the same ghost reflection on X and D.  This reproduces every rule of
// Sketch 1 (zero cross and first differences on upper faces, the doubled
// Neumann second difference, Outer values) with about half the FP64
// operations of the direct form.
template <int N>
struct CIdx {
    static constexpr int diag = 0;                           // N
    static constexpr int ctr = N;                            // 1
    static constexpr int cross = N + 1;                      // N(N-1)/2, (i,k) i<k row by row
    static constexpr int drift = N + 1 + N * (N - 1) / 2;    // N-2, axes 1..N-2
    static constexpr int fg = drift + N - 2;                 // dt * F(payoff)
    __device__ static constexpr int pair(int i, int k) { return cross + i * (2 * N - i - 1) / 2 + (k - i - 1); }
};

template <int N>
__device__ void build_node_coefs(const Shape<N>& s, const double* tabd, const Consts<double>& c,
                                 const double* H, double* C, int Lp, int rank, int gsize)
{
    using I = CIdx<N>;
    for (int t = rank; t < s.L; t += gsize) {
        int j[N];
        decode<N>(s, t, j);
        const int J = s.padded(t);
        const double v2 = tabd[s.toff[N - 1] + j[N - 1] - 1] * c.dt;  // dt V^2
        double sum = 0.0;
#pragma unroll
        for (int i = 0; i < N - 1; ++i) {
            const double cdi = tabd[s.toff[i] + j[i] - 1] * v2;
            C[(I::diag + i) * Lp + J] = cdi;
            sum += cdi;
        }
        const double cdv = c.cV * v2;
        C[(I::diag + N - 1) * Lp + J] = cdv;
        sum += cdv;
        C[I::ctr * Lp + J] = -2.0 * sum;
#pragma unroll
        for (int i = 0; i < N - 1; ++i) {
            const double pwi = tabd[s.toff[i] + s.M[i] + j[i] - 1];
#pragma unroll
            for (int k = i + 1; k < N; ++k) {
                const double m = (k < N - 1) ? c.rm[upair(i, k)] * pwi * tabd[s.toff[k] + s.M[k] + j[k] - 1] * v2
                                             : c.sm[i] * pwi * v2;
                C[I::pair(i, k) * Lp + J] = m;
            }
            if (i >= 1) {
                double S = 0.0;
#pragma unroll
                for (int r = 1; r <= i; ++r) S += c.rh[ltri(i, r)] * tabd[s.toff[r] + 2 * s.M[r] + j[r] - 1];
                C[(I::drift + i - 1) * Lp + J] = pwi * S * c.g2[i] * v2;
            }
        }
        C[I::fg * Lp + J] = v2 * H[t & (s.Lr - 1)];
    }
}

// Central differences D_k = X[J + E_k] - X[J - E_k] for axes k >= 1, off
// the upper face of axis k.  The cross terms read D_k for k > i >= 0 and the
// drift terms D_i for i >= 1, both only off that face (where Sketch 1 sets
// them to zero), so axis 0 and the upper-face entries are never read.  On an
// axis with a single Inner row (M_k = 1) every node is on the upper face, and
// the whole pass along it is skipped alike by every lane of the grid.
template <int N>
__device__ __forceinline__ void diff_pass(const Shape<N>& s, const double* X, double* D, int Lp,
                                          int rank, int gsize)
{
    for (int t = rank; t < s.L; t += gsize) {
        int j[N];
        decode<N>(s, t, j);
        const int J = s.padded(t);
#pragma unroll
        for (int k = 1; k < N; ++k) {
            if (j[k] != s.M[k]) {  // (also not on a Dirichlet face: never read there)
                const double xm = (j[k] > 1) ? X[J - s.Sp[k]] : 0.0;
                D[k * Lp + J] = X[J + s.Sp[k]] - xm;
            }
        }
    }
}

// dt F_0(X) at the Inner node J, plus init.  Terms that vanish are skipped:
// the neighbour sum along an axis with one Inner row (both neighbours are
// zero: an Outer node and its ghost reflection; the centre term keeps its
// part), and the cross and drift terms on the upper face of their axes.
template <int N>
__device__ __forceinline__ double diff_F(const Shape<N>& s, const int (&j)[N], int J,
                                         const double* X, const double* D, const double* C, int Lp,
                                         double init)
{
    using I = CIdx<N>;
    double f = fma(C[I::ctr * Lp + J], X[J], init);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (s.M[i] > 1) {
            const double xm = (j[i] > 1) ? X[J - s.Sp[i]] : 0.0;
            const double xp = (j[i] == s.nf[i]) ? xm : X[J + s.Sp[i]];
            f += C[(I::diag + i) * Lp + J] * (xp + xm);
        }
    }
#pragma unroll
    for (int i = 0; i < N - 1; ++i) {
        if (j[i] != s.nf[i]) {
            const bool li = j[i] > 1;
#pragma unroll
            for (int k = i + 1; k < N; ++k) {
                if (j[k] != s.nf[k]) {
                    const double dp = D[k * Lp + J + s.Sp[i]];
                    const double dm = li ? D[k * Lp + J - s.Sp[i]] : 0.0;
                    f += C[I::pair(i, k) * Lp + J] * (dp - dm);
                }
            }
        }
    }
#pragma unroll
    for (int i = 1; i < N - 1; ++i)
        if (j[i] != s.nf[i]) f += C[(I::drift + i - 1) * Lp + J] * D[i * Lp + J];
    return f;
}

// ----------------------------------------------------------- line solves
// (I - nu dt A_axis) X = G on every line along `axis` (Lemma ls, eq.
// decomp1).  A line of M rows is shared by P = 2^plog lanes of one warp; lane
// p holds rows p, p+P, p+2P, ... (R = M/P <= kMaxRows of them).  plog levels
// of parallel cyclic reduction over warp shuffles decouple the line into P
// interleaved tridiagonal systems, which each lane then solves by Thomas
// elimination.  The matrices do not change in time, so every multiplier and
// Thomas factor comes from tables built once per grid (pcr_setup).  At a
// wrap-around (row p+Pq's neighbour at distance d lives in the previous or
// next row slot of another lane) the sending lane picks the slot, so each
// level costs one shuffle per direction.

// Lanes of the calling thread's work group inside its warp: the whole warp
// for CTA groups and 32-lane warp groups, 2^glog lanes for smaller groups.
__device__ __forceinline__ unsigned group_mask(int glog)
{
    if (glog >= 5) return 0xffffffffu;
    const unsigned lanes = (1u << (1 << glog)) - 1u;
    return lanes << ((threadIdx.x & 31) & ~((1 << glog) - 1));
}

template <typename T>
__device__ __forceinline__ T shfl(T v, int src, int width, unsigned mask)
{
    return __shfl_sync(mask, v, src, width);
}

// Row r of (I - nu dt A_axis) for line class cls: lower a, diagonal b, upper c.
template <int N>
__device__ __forceinline__ void matrix_row(const Shape<N>& s, const double* tabd,
                                           const Consts<double>& c, int axis, int cls, int r,
                                           double& a, double& b, double& u)
{
    const int M = s.M[axis];
    const double delta = (axis < N - 1) ? tabd[s.toff[axis] + r] * tabd[s.toff[N - 1] + cls]
                                        : c.cV * tabd[s.toff[N - 1] + r];
    const double nd = c.nudt * delta;
    if ((s.dmask >> axis) & 1) {
        // eq. bound1_0: rows 0..M-2 are the M-1 Inner nodes (no super-diagonal
        // in the last, whose upper neighbour holds Dirichlet data); row M-1 is
        // that Dirichlet node, an identity row
        const bool dir = r == M - 1;
        b = dir ? 1.0 : 1.0 + 2.0 * nd;
        u = (r < M - 2) ? -nd : 0.0;
        a = (r == 0 || dir) ? 0.0 : -nd;
        return;
    }
    b = 1.0 + 2.0 * nd;
    u = (r < M - 1) ? -nd : 0.0;
    a = (r == 0) ? 0.0 : ((r < M - 1) ? -nd : -2.0 * nd);
}

// An axis with one Inner row (M_i = 1) has a 1x1 directional matrix
// b_i = 1 + 2 nu dt delta_i, which for a rate axis depends on the V index
// only, so its solve is the scaling by 1/b_i(j_V).  These scalings commute
// with the solves along the other rate axes (which keep j_V), so they are
// applied together inside one other solve: solving (I - nu dt A_a) x = S g
// with S = prod 1/b_i is solving (S^-1 (I - nu dt A_a)) x = g, whose matrix
// rows are those of axis a times prod_i b_i.  The target a (`last`) is the V
// axis, or, when V has one row too (then every b_i is a constant), the last
// rate axis with more than one row.  This returns that product for row r of
// line class cls of the target axis.
template <int N>
__device__ __forceinline__ double fold_scale(const Shape<N>& s, const double* tabd,
                                             const Consts<double>& c, int axis, int cls, int r)
{
    const int v = (axis == N - 1) ? r : cls;  // V index of the row
    double f = 1.0;
#pragma unroll
    for (int i = 0; i < N - 1; ++i)  // (a Dirichlet axis of one row has no Inner node: identity)
        if (((s.skip & ~s.dmask) >> i) & 1) f *= 1.0 + 2.0 * (c.nudt * (tabd[s.toff[i]] * tabd[s.toff[N - 1] + v]));
    if ((s.skip >> (N - 1)) & 1) f *= 1.0 + 2.0 * (c.nudt * (c.cV * tabd[s.toff[N - 1]]));
    return f;
}

// The PCR multipliers and Thomas factors of every line class: the same
// reduction as the solve, applied to the matrix coefficients (FP64).  Rows
// are updated in ascending order; each lane keeps the pre-update values of
// its previous row, which is the wrap-around neighbour the next row needs.
// TC: the precision of the reduction (FP64 for the FP64 mode; the
// mixed-precision mode solves its lines in FP32 and factors them in FP32 as
// well, from matrix rows formed in FP64).
template <int N, typename T, int RMAX, typename TC = double>
__device__ void pcr_setup(const Shape<N>& s, const double* tabd, const Consts<double>& c, T* lu,
                          int rank, int gsize, unsigned gm)
{
    for (int axis = 0; axis < N; ++axis) {
        // axes folded into another solve have no factors; dense_setup factors the dense ones
        if (((s.skip | s.dense) >> axis) & 1) continue;
        const int M = s.M[axis];
        const int plog = s.plog[axis];
        const int P = 1 << plog;
        const int R = M >> plog;
        const int S = s.luS[axis];
        const int ncls = (axis < N - 1) ? s.M[N - 1] : 1;
        const int lpr = gsize >> plog;
        const int p = rank & (P - 1);
        const int slot = rank >> plog;
        for (int base = 0; base < ncls; base += lpr) {  // uniform across the group
            const int cls = base + slot;
            const bool act = cls < ncls;
            const int cl = act ? cls : 0;
            T* tb = lu + s.luoff[axis] + (cl * M + p) * S;
            TC a[RMAX], b[RMAX], u[RMAX];
#pragma unroll
            for (int q = 0; q < RMAX; ++q) {
                if (q < R) {
                    double ad, bd, ud;
                    matrix_row<N>(s, tabd, c, axis, cl, p + P * q, ad, bd, ud);
                    if (axis == s.last && s.skip) {  // the folded single-row solves
                        const double f = fold_scale<N>(s, tabd, c, axis, cl, p + P * q);
                        ad *= f;
                        bd *= f;
                        ud *= f;
                    }
                    a[q] = (TC)ad;
                    b[q] = (TC)bd;
                    u[q] = (TC)ud;
                }
            }
            for (int k = 0; k < plog; ++k) {
                const int d = 1 << k;
                const int sm = (p - d) & (P - 1), sp = (p + d) & (P - 1);
                const bool wm = p < d, wp = p + d >= P;      // this lane receives across a wrap
                const bool send_prev = p >= P - d;          // my receiver (p + d) wraps
                const bool send_next = p < d;               // my receiver (p - d) wraps
                // reciprocals of this level's diagonals (one division per row;
                // the neighbours' reciprocals arrive by shuffle)
                TC rb[RMAX];
#pragma unroll
                for (int q = 0; q < RMAX; ++q) rb[q] = (q < R) ? TC(1) / b[q] : TC(1);
                TC pa = TC(0), prb = TC(1), pu = TC(0);      // pre-update values of row q-1
#pragma unroll
                for (int q = 0; q < RMAX; ++q) {
                    if (q < R) {
                        const int qn = (q + 1 < RMAX) ? q + 1 : q;  // static after unrolling
                        const bool nx = q + 1 < R;
                        // to the lane above (p + d): my row q, or my row q-1 across the wrap
                        const TC a_m = shfl(send_prev ? pa : a[q], sm, P, gm);
                        const TC rb_m = shfl(send_prev ? prb : rb[q], sm, P, gm);
                        const TC u_m = shfl(send_prev ? pu : u[q], sm, P, gm);
                        // to the lane below (p - d): my row q, or my row q+1 across the wrap
                        const TC a_p = shfl(send_next ? (nx ? a[qn] : TC(0)) : a[q], sp, P, gm);
                        const TC rb_p = shfl(send_next ? (nx ? rb[qn] : TC(1)) : rb[q], sp, P, gm);
                        const TC u_p = shfl(send_next ? (nx ? u[qn] : TC(0)) : u[q], sp, P, gm);
                        const bool hm = !wm || q >= 1;
                        const TC al = hm ? a[q] * rb_m : TC(0);
                        const TC ga = u[q] * rb_p;  // identity row sent past the end
                        if (act) {
                            tb[q * P * S + 2 * k] = (T)al;
                            tb[q * P * S + 2 * k + 1] = (T)(wp && !nx ? TC(0) : ga);
                        }
                        pa = a[q];
                        prb = rb[q];
                        pu = u[q];
                        const TC gg = (wp && !nx) ? TC(0) : ga;
                        b[q] = b[q] - al * u_m - gg * a_p;
                        a[q] = -al * a_m;
                        u[q] = -gg * u_p;
                    }
                }
            }
            // Thomas factors of the lane's interleaved system (rows coupled at distance P)
            TC gam = TC(0);
#pragma unroll
            for (int q = 0; q < RMAX; ++q) {
                if (q < R) {
                    const TC inv = TC(1) / (b[q] - a[q] * gam);
                    gam = u[q] * inv;
                    if (act) {
                        T* row = tb + q * P * S + 2 * plog;
                        row[0] = (T)a[q];
                        row[1] = (T)inv;
                        row[2] = (T)gam;
                    }
                }
            }
        }
    }
}

template <int N, typename T, int RMAX, class Epi>
__device__ __forceinline__ void sweep(const Shape<N>& s, int axis, const T* __restrict__ lu,
                                      const T* src, T* dst, int rank, int gsize, unsigned gm,
                                      Epi epi)
{
    const int M = s.M[axis];
    const int plog = s.plog[axis];
    const int P = 1 << plog;
    const int R = M >> plog;
    const int S = s.luS[axis];
    const int lvA = s.lv[axis];
    const int sh = s.sh[axis];
    const int Spa = s.Sp[axis];
    const int nl = s.L >> lvA;
    const int lo_mask = (1 << sh) - 1;
    const int MV1 = s.M[N - 1] - 1;
    const int shV = s.sh[N - 1];
    const int lpr = gsize >> plog;
    const int p = rank & (P - 1);
    const int slot = rank >> plog;
    for (int base = 0; base < nl; base += lpr) {  // uniform across the group
        const int line = base + slot;
        const bool act = line < nl;
        const int ln = act ? line : 0;
        const int t0 = (ln & lo_mask) | ((ln >> sh) << (sh + lvA));
        const int J0 = s.padded(t0) + p * Spa;
        const int cls = (axis == N - 1) ? 0 : ((t0 >> shV) & MV1);
        const T* tb = lu + s.luoff[axis] + (cls * M + p) * S;  // row p of the line
        const int PS = P * S, PSp = P * Spa;
        T x[RMAX];
#pragma unroll
        for (int q = 0; q < RMAX; ++q)
            if (q < R) x[q] = act ? src[J0 + q * PSp] : T(0);
        for (int k = 0; k < plog; ++k) {
            const int d = 1 << k;
            const int sm = (p - d) & (P - 1), sp = (p + d) & (P - 1);
            const bool send_prev = p >= P - d;
            const bool send_next = p < d;
            T prev = T(0);  // pre-update value of this lane's row q-1
#pragma unroll
            for (int q = 0; q < RMAX; ++q) {
                if (q < R) {
                    const int qn = (q + 1 < RMAX) ? q + 1 : q;  // static after unrolling
                    const T vm = shfl(send_prev ? prev : x[q], sm, P, gm);
                    const T vp = shfl(send_next ? ((q + 1 < R) ? x[qn] : T(0)) : x[q], sp, P, gm);
                    const T* row = tb + q * PS;
                    prev = x[q];
                    // multipliers are zero where the neighbour lies outside the line
                    x[q] = x[q] - row[2 * k] * vm - row[2 * k + 1] * vp;
                }
            }
        }
        // forward elimination; the lane's first row has no predecessor, so its
        // lower factor drops out (x - l * 0 = x)
        T y = T(0);
#pragma unroll
        for (int q = 0; q < RMAX; ++q) {
            if (q < R) {
                const T* row = tb + q * PS + 2 * plog;
                y = (q == 0) ? x[q] * row[1] : (x[q] - row[0] * y) * row[1];
                x[q] = y;
            }
        }
#pragma unroll
        for (int q = RMAX - 2; q >= 0; --q)
            if (q < R - 1) x[q] = x[q] - tb[q * PS + 2 * plog + 2] * x[q + 1];
        if (act) {
#pragma unroll
            for (int q = 0; q < RMAX; ++q) {
                if (q < R) {
                    const int J = J0 + q * PSp;
                    dst[J] = x[q];
                    epi(J, x[q]);
                }
            }
        }
    }
}

struct NoEpi {
    template <typename T>
    __device__ __forceinline__ void operator()(int, T) const {}
};

// ------------------------------------------ explicit inverses of short lines
// For an axis of M = 2..8 rows (mixed-precision warp groups), the inverse of
// every line class's directional matrix (I - nu dt A_axis), with the folded
// single-row scalings when the axis is `last`.  One lane per (axis, class)
// forms the M matrix rows in FP64 (as the line-solve factors are formed),
// factors them by Thomas elimination in FP32, the precision of the mode's line
// solves (the matrix is diagonally dominant, its inverse non-negative with row
// sums at most 1), and solves for the M unit vectors.  Entry (q, col) is
// stored in row q at position q XOR col, the order in which dense_mix meets
// the rows of a line.
template <int N>
__device__ __noinline__ void dense_setup(const Shape<N>& s, const double* tabd, const Consts<double>& c, float* lu,
                            int rank, int gsize)
{
    int total = 0;  // (axis, class) pairs of the dense axes
#pragma unroll
    for (int axis = 0; axis < N; ++axis)
        if ((s.dense >> axis) & 1) total += (axis < N - 1) ? s.M[N - 1] : 1;
    for (int w = rank; w < total; w += gsize) {
        int axis = 0, cls = w;
        for (; axis < N; ++axis) {
            if (!((s.dense >> axis) & 1)) continue;
            const int nc = (axis < N - 1) ? s.M[N - 1] : 1;
            if (cls < nc) break;
            cls -= nc;
        }
        const int M = s.M[axis];
        const bool fold = axis == s.last && s.skip;
        // a rate axis's fold product depends on its class (the V index) only
        const double fr = (fold && axis < N - 1) ? fold_scale<N>(s, tabd, c, axis, cls, 0) : 1.0;
        float lo[kDenseMaxRows], inv[kDenseMaxRows], gam[kDenseMaxRows];
        float gp = 0.f;
#pragma unroll
        for (int q = 0; q < kDenseMaxRows; ++q) {
            if (q < M) {
                double ad, bd, ud;
                matrix_row<N>(s, tabd, c, axis, cls, q, ad, bd, ud);
                if (fold) {
                    const double f = (axis < N - 1) ? fr : fold_scale<N>(s, tabd, c, axis, cls, q);
                    ad *= f;
                    bd *= f;
                    ud *= f;
                }
                lo[q] = (float)ad;
                inv[q] = 1.f / ((float)bd - lo[q] * gp);
                gp = (float)ud * inv[q];
                gam[q] = gp;
            }
        }
        float* out = lu + s.luoff[axis] + cls * M * M;
#pragma unroll 1
        for (int col = 0; col < M; ++col) {
            // forward elimination into the output slots, then back substitution there
            float yp = 0.f;
#pragma unroll
            for (int q = 0; q < kDenseMaxRows; ++q) {
                if (q < M) {
                    yp = ((q == col ? 1.f : 0.f) - lo[q] * yp) * inv[q];
                    out[q * M + (q ^ col)] = yp;
                }
            }
            float x = 0.f;  // the last row has no upper neighbour (gam = 0 there)
#pragma unroll
            for (int q = kDenseMaxRows - 1; q >= 0; --q) {
                if (q < M) {
                    float& o = out[q * M + (q ^ col)];
                    x = o - gam[q] * x;
                    o = x;
                }
            }
        }
    }
}

// Coefficient row of MM floats (16-byte aligned for MM >= 4, 8-byte for 2).
template <int MM>
__device__ __forceinline__ void load_row(const float* p, float (&r)[MM])
{
    if constexpr (MM == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        r[0] = v.x;
        r[1] = v.y;
    } else {
#pragma unroll
        for (int q = 0; q < MM; q += 4) {
            const float4 v = *reinterpret_cast<const float4*>(p + q);
            r[q] = v.x;
            r[q + 1] = v.y;
            r[q + 2] = v.z;
            r[q + 3] = v.w;
        }
    }
}

// The directional solves along an axis of MM rows for the group's values in
// registers: lane `rank` holds nodes t = rank (x[0]) and, when the grid has
// more nodes than the group has lanes, t = rank + gsize (x[1]).  Node t gets
// sum_s Cinv[j][j ^ s] x(t ^ (s << sh)), j its row on the line; the node at
// XOR distance s << sh sits in lane rank ^ ((s << sh) mod gsize), in the
// other slot when s << sh reaches gsize.  Every lane of the group takes part
// (the shuffles); the values of lanes without a node are never read by one
// that has a node (the XOR of two node indices below L stays below L).
template <int MM>
__device__ __forceinline__ void dense_mix(const float* __restrict__ C, int sh, int shV, int mV, bool rate,
                                          int rank, int gsize, int tlog, bool two, unsigned gm, float (&x)[2])
{
    float y[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (k == 1 && !two) break;
        const int t = rank + (k << tlog);
        const int j = (t >> sh) & (MM - 1);
        const int cls = rate ? ((t >> shV) & mV) : 0;
        float r[MM];
        load_row<MM>(C + (cls * MM + j) * MM, r);
        float acc = r[0] * x[k];
#pragma unroll
        for (int q = 1; q < MM; ++q) {
            const int d = q << sh;
            const int lm = d & (gsize - 1);
            const float mine = (d >> tlog) ? x[k ^ 1] : x[k];
            const float v = lm ? __shfl_xor_sync(gm, mine, lm, gsize) : mine;
            acc = fmaf(r[q], v, acc);
        }
        y[k] = acc;
    }
    x[0] = y[0];
    if (two) x[1] = y[1];
}

// ------------------------------------- line solves on grids in global memory
// The same reduction and elimination as pcr_setup / sweep, for grids whose
// state lives in global memory and whose lines may have any length: a lane's
// rows are not held in registers but streamed from memory, one pass per PCR
// level (ascending rows; the lane keeps the pre-update value of its previous
// row and reads the next row before it is overwritten) and one pass each for
// the Thomas forward and backward sweeps.  Lanes of a line step through their
// rows together, so the shuffles pair the same rows as in the register
// version and the arithmetic is the same.

// PCR multipliers and Thomas factors; scr holds the running (lower, diagonal,
// upper) of every row of the axis being factored (3 x rows doubles).
template <int N, typename T>
__device__ void pcr_setup_mem(const Shape<N>& s, const double* tabd, const Consts<double>& c, T* lu,
                              double* scr, int rank, int gsize, unsigned gm)
{
    for (int axis = 0; axis < N; ++axis) {
        const int M = s.M[axis];
        const int plog = s.plog[axis];
        const int P = 1 << plog;
        const int R = M >> plog;
        const int S = s.luS[axis];
        const int ncls = (axis < N - 1) ? s.M[N - 1] : 1;
        const int rows = ncls * M;
        double* sa = scr;
        double* sb = scr + rows;
        double* su = scr + 2 * rows;
        const int lpr = gsize >> plog;
        const int p = rank & (P - 1);
        const int slot = rank >> plog;
        for (int base = 0; base < ncls; base += lpr) {  // uniform across the group
            const int cls = base + slot;
            const bool act = cls < ncls;
            const int cl = act ? cls : 0;
            T* tb = lu + s.luoff[axis] + (cl * M + p) * S;
            const int r0 = cl * M + p;  // this lane's row q lives at r0 + P q
            if (act)
                for (int q = 0; q < R; ++q) {
                    double a, b, u;
                    matrix_row<N>(s, tabd, c, axis, cl, p + P * q, a, b, u);
                    sa[r0 + P * q] = a;
                    sb[r0 + P * q] = b;
                    su[r0 + P * q] = u;
                }
            for (int k = 0; k < plog; ++k) {
                const int d = 1 << k;
                const int sm = (p - d) & (P - 1), sp = (p + d) & (P - 1);
                const bool wm = p < d, wp = p + d >= P;
                const bool send_prev = p >= P - d;
                const bool send_next = p < d;
                double pa = 0.0, pb = 1.0, pu = 0.0;  // pre-update values of row q-1
                double ca = act ? sa[r0] : 0.0, cb = act ? sb[r0] : 1.0, cu = act ? su[r0] : 0.0;
                for (int q = 0; q < R; ++q) {
                    const bool nx = q + 1 < R;
                    const int rn = r0 + P * (q + 1);
                    const double na = (act && nx) ? sa[rn] : 0.0;
                    const double nb = (act && nx) ? sb[rn] : 1.0;
                    const double nu = (act && nx) ? su[rn] : 0.0;
                    const double a_m = shfl(send_prev ? pa : ca, sm, P, gm);
                    const double b_m = shfl(send_prev ? pb : cb, sm, P, gm);
                    const double u_m = shfl(send_prev ? pu : cu, sm, P, gm);
                    const double a_p = shfl(send_next ? na : ca, sp, P, gm);
                    const double b_p = shfl(send_next ? nb : cb, sp, P, gm);
                    const double u_p = shfl(send_next ? nu : cu, sp, P, gm);
                    const bool hm = !wm || q >= 1;
                    const double al = hm ? ca / b_m : 0.0;
                    const double ga = cu / b_p;  // identity row sent past the end
                    const double gg = (wp && !nx) ? 0.0 : ga;
                    if (act) {
                        tb[q * P * S + 2 * k] = (T)al;
                        tb[q * P * S + 2 * k + 1] = (T)gg;
                        const int rq = r0 + P * q;
                        sb[rq] = cb - al * u_m - gg * a_p;
                        sa[rq] = -al * a_m;
                        su[rq] = -gg * u_p;
                    }
                    pa = ca;
                    pb = cb;
                    pu = cu;
                    ca = na;
                    cb = nb;
                    cu = nu;
                }
            }
            // Thomas factors of the lane's interleaved system
            double gam = 0.0;
            if (act)
                for (int q = 0; q < R; ++q) {
                    const int rq = r0 + P * q;
                    const double inv = 1.0 / (sb[rq] - sa[rq] * gam);
                    gam = su[rq] * inv;
                    T* row = tb + q * P * S + 2 * plog;
                    row[0] = (T)sa[rq];
                    row[1] = (T)inv;
                    row[2] = (T)gam;
                }
        }
        __syncthreads();  // the next axis reuses scr
    }
}

template <int N, typename T, class Epi>
__device__ __forceinline__ void sweep_mem(const Shape<N>& s, int axis, const T* __restrict__ lu,
                                          const T* src, T* dst, int rank, int gsize, unsigned gm,
                                          Epi epi)
{
    const int M = s.M[axis];
    const int plog = s.plog[axis];
    const int P = 1 << plog;
    const int R = M >> plog;
    const int S = s.luS[axis];
    const int lvA = s.lv[axis];
    const int sh = s.sh[axis];
    const int Spa = s.Sp[axis];
    const int nl = s.L >> lvA;
    const int lo_mask = (1 << sh) - 1;
    const int MV1 = s.M[N - 1] - 1;
    const int shV = s.sh[N - 1];
    const int lpr = gsize >> plog;
    const int p = rank & (P - 1);
    const int slot = rank >> plog;
    for (int base = 0; base < nl; base += lpr) {  // uniform across the group
        const int line = base + slot;
        const bool act = line < nl;
        const int ln = act ? line : 0;
        const int t0 = (ln & lo_mask) | ((ln >> sh) << (sh + lvA));
        const int J0 = s.padded(t0) + p * Spa;
        const int cls = (axis == N - 1) ? 0 : ((t0 >> shV) & MV1);
        const T* tb = lu + s.luoff[axis] + (cls * M + p) * S;
        const int PS = P * S, PSp = P * Spa;
        // Loads run ahead of their use (rows two ahead, factors one ahead) so
        // that a lane does not wait a full memory round trip per row; every
        // load of a row precedes, in program order, the store that replaces it.
        const T* in = src;
        for (int k = 0; k < plog; ++k) {
            const int d = 1 << k;
            const int sm = (p - d) & (P - 1), sp = (p + d) & (P - 1);
            const bool send_prev = p >= P - d;
            const bool send_next = p < d;
            T prev = T(0);
            T cur = act ? in[J0] : T(0);
            T nxt = (act && R > 1) ? in[J0 + PSp] : T(0);
            T al = act ? tb[2 * k] : T(0), ga = act ? tb[2 * k + 1] : T(0);
            for (int q = 0; q < R; ++q) {
                const T nn = (act && q + 2 < R) ? in[J0 + (q + 2) * PSp] : T(0);
                const bool more = act && q + 1 < R;
                const T al_n = more ? tb[(q + 1) * PS + 2 * k] : T(0);
                const T ga_n = more ? tb[(q + 1) * PS + 2 * k + 1] : T(0);
                const T vm = shfl(send_prev ? prev : cur, sm, P, gm);
                const T vp = shfl(send_next ? nxt : cur, sp, P, gm);
                if (act) dst[J0 + q * PSp] = cur - al * vm - ga * vp;
                prev = cur;
                cur = nxt;
                nxt = nn;
                al = al_n;
                ga = ga_n;
            }
            in = dst;  // later levels in place
        }
        if (act) {
            const T* th = tb + 2 * plog;  // Thomas factors (lower, 1/pivot, upper/pivot) of row q at q PS
            // the first row has no predecessor: its lower factor drops out
            T y = in[J0] * th[1];
            dst[J0] = y;
            T x = R > 1 ? in[J0 + PSp] : T(0);
            T lo = R > 1 ? th[PS] : T(0), iv = R > 1 ? th[PS + 1] : T(0);
            T x1 = R > 2 ? in[J0 + 2 * PSp] : T(0);
            for (int q = 1; q < R; ++q) {
                const T x2 = q + 2 < R ? in[J0 + (q + 2) * PSp] : T(0);
                const T lo_n = q + 1 < R ? th[(q + 1) * PS] : T(0);
                const T iv_n = q + 1 < R ? th[(q + 1) * PS + 1] : T(0);
                y = (x - lo * y) * iv;
                dst[J0 + q * PSp] = y;
                x = x1;
                x1 = x2;
                lo = lo_n;
                iv = iv_n;
            }
            int J = J0 + (R - 1) * PSp;
            epi(J, y);
            T b = R > 1 ? dst[J0 + (R - 2) * PSp] : T(0), g = R > 1 ? th[(R - 2) * PS + 2] : T(0);
            for (int q = R - 2; q >= 0; --q) {
                const T b_n = q > 0 ? dst[J0 + (q - 1) * PSp] : T(0);
                const T g_n = q > 0 ? th[(q - 1) * PS + 2] : T(0);
                J = J0 + q * PSp;
                y = b - g * y;
                dst[J] = y;
                epi(J, y);
                b = b_n;
                g = g_n;
            }
        }
    }
}

// One out-of-line copy of the register sweep per epilogue type.
template <int N, typename T, int RMAX, class Epi>
__device__ __noinline__ void sweep_outlined(const Shape<N>& s, int axis, const T* __restrict__ lu,
                                            const T* src, T* dst, int rank, int gsize, unsigned gm,
                                            Epi epi)
{
    sweep<N, T, RMAX>(s, axis, lu, src, dst, rank, gsize, gm, epi);
}

// Line sweep of a work-group kind: rows in registers (warp and CTA groups)
// or streamed from memory (global-memory groups).  For N <= 4 the register
// sweep is called out of line (one copy instead of one per call site), which
// measured faster there; for larger N inlining measured faster.
template <int N, typename T, int KIND, class Epi>
__device__ __forceinline__ void lsweep(const Shape<N>& s, int axis, const T* __restrict__ lu,
                                       const T* src, T* dst, int rank, int gsize, unsigned gm,
                                       Epi epi)
{
    constexpr int RM = 1 << (KIND == kWarpGroup ? kRowsLogWarp
                                                : (std::is_same<T, float>::value ? kRowsLogCtaMixed : kRowsLogCta));
    if constexpr (KIND == kMemGroup)
        sweep_mem<N, T>(s, axis, lu, src, dst, rank, gsize, gm, epi);
    else if constexpr (N <= 4)
        sweep_outlined<N, T, RM>(s, axis, lu, src, dst, rank, gsize, gm, epi);
    else
        sweep<N, T, RM>(s, axis, lu, src, dst, rank, gsize, gm, epi);
}

template <bool WARP>
__device__ __forceinline__ void gsync(unsigned gm)
{
    if (WARP)
        __syncwarp(gm);
    else
        __syncthreads();
}

// --------------------------------------------------------- table building
// Exact power of two 2^e (|e| < 1023).
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// Coefficient and payoff tables of the grid and its constants.  The table
// entries of all axes are spread over the group's lanes at once (an entry
// divides once and takes a square root), and each constant is the instance's
// level-free factor times an exact power of two (no division per grid).
// F32ROOT: F^beta (beta = 1/2) by an FP32 square root, for the mixed
// precision mode, whose coefficient tables feed FP32 arithmetic only (the
// stencil, the drift and the line-solve factors, formed from FP32-accurate
// rows); the payoff tables stay FP64.
template <int N, bool F32ROOT = false>
__device__ void build_tables(const Shape<N>& s, const InstDev& P, double* tabd, double* pay,
                             Consts<double>* cd, int rank, int gsize)
{
    const double beta = P.beta;
    const bool half = beta == 0.5;  // F^beta by a square root (the usual SABR choice)
    int nrate = 0;                  // rate entries: j = 0..M_a per axis
#pragma unroll
    for (int a = 0; a < N - 1; ++a) nrate += s.M[a] + 1;
    const int MV = s.M[N - 1];
    for (int w = rank; w < nrate + MV; w += gsize) {
        if (w >= nrate) {
            const int jj = w - nrate + 1;
            const double V = (double)jj * (P.Fmax[N - 1] * pow2(-s.lv[N - 1]));  // h_V = Vmax / M_V exactly
            tabd[s.toff[N - 1] + jj - 1] = V * V;
            continue;
        }
        int a = 0, jj = w;
        while (jj > s.M[a]) {
            jj -= s.M[a] + 1;
            ++a;
        }
        const int M = s.M[a];
        const double h = P.Fmax[a] * pow2(-s.lv[a]);  // Fmax / M exactly (M = 2^lv)
        const double al = P.alpha[a], ta = P.tau[a];
        const double F = (double)jj * h;
        const double bF = 1.0 / (1.0 + ta * F);  // discount factor of the accrual period
        pay[s.poff[a] + jj] = (P.payoff == 0) ? (F - P.K) : ta * (F - P.K);
        pay[s.phalf + s.poff[a] + jj] = bF;
        if (jj >= 1) {
            const double dcoef = P.dcb[a] * pow2(2 * s.lv[a]);  // alpha^2 rho_aa / (2 h^2)
            const double Fb = half ? (F32ROOT ? (double)sqrtf((float)F) : sqrt(F)) : pow(F, beta);
            const double F2b = half ? F : pow(F, 2.0 * beta);
            tabd[s.toff[a] + jj - 1] = dcoef * F2b;
            tabd[s.toff[a] + M + jj - 1] = al * Fb;
            tabd[s.toff[a] + 2 * M + jj - 1] = al * ta * Fb * bF;
        }
    }
    // the constants, one entry per lane at a time
    constexpr int kPairs = kMaxDim * (kMaxDim - 1) / 2, kTri = kMaxDim * (kMaxDim + 1) / 2;
    constexpr int kConsts = 1 + kPairs + kTri + 2 * kMaxDim;
    for (int q = rank; q < kConsts; q += gsize) {
        if (q == 0) {
            cd->cV = P.cVb * pow2(2 * s.lv[N - 1]);  // sigma^2 / (2 h_V^2)
            cd->dt = P.dt;
            cd->thdt = P.theta * P.dt;
            cd->nudt = P.nu * P.dt;
        } else if (q <= kPairs) {  // rm[upair(i, k)] = rho_ik / (4 h_i h_k), i < k
            int i = 0, r = q - 1;
            while (r >= kMaxDim - 1 - i) {
                r -= kMaxDim - 1 - i;
                ++i;
            }
            const int k = i + 1 + r;
            const bool ok = i < N - 1 && k < N - 1;
            cd->rm[upair(i, k)] = ok ? P.rmb[upair(i, k)] * pow2(s.lv[i] + s.lv[k]) : 0.0;
        } else if (q <= kPairs + kTri) {  // rh[ltri(i, r)], r <= i
            int i = 0, r = q - 1 - kPairs;
            while (r > i) {
                r -= i + 1;
                ++i;
            }
            cd->rh[ltri(i, r)] = (i < N - 1) ? P.rho[i * kMaxDim + r] : 0.0;
        } else if (q <= kPairs + kTri + kMaxDim) {  // sigma phi_i / (4 h_i h_V)
            const int i = q - 1 - kPairs - kTri;
            cd->sm[i] = (i < N - 1) ? P.smb[i] * pow2(s.lv[i] + s.lv[N - 1]) : 0.0;
        } else {  // 1 / (2 h_i)
            const int i = q - 1 - kPairs - kTri - kMaxDim;
            cd->g2[i] = (i < N) ? P.g2b[i] * pow2(s.lv[i]) : 0.0;
        }
    }
}

// The FP32 (or FP64) copy of the constants, one entry per lane at a time.
template <typename T>
__device__ void convert_consts(const Consts<double>& a, Consts<T>* b, int rank, int gsize)
{
    constexpr int kP = kMaxDim * (kMaxDim - 1) / 2, kT = kMaxDim * (kMaxDim + 1) / 2;
    for (int q = rank; q < 4 + kP + kT + 2 * kMaxDim; q += gsize) {
        if (q < 4) {
            const double v = q == 0 ? a.cV : (q == 1 ? a.dt : (q == 2 ? a.thdt : a.nudt));
            T& o = q == 0 ? b->cV : (q == 1 ? b->dt : (q == 2 ? b->thdt : b->nudt));
            o = (T)v;
        } else if (q < 4 + kP) {
            b->rm[q - 4] = (T)a.rm[q - 4];
        } else if (q < 4 + kP + kT) {
            b->rh[q - 4 - kP] = (T)a.rh[q - 4 - kP];
        } else if (q < 4 + kP + kT + kMaxDim) {
            b->sm[q - 4 - kP - kT] = (T)a.sm[q - 4 - kP - kT];
        } else {
            b->g2[q - 4 - kP - kT - kMaxDim] = (T)a.g2[q - 4 - kP - kT - kMaxDim];
        }
    }
}

// Mixed mode keeps, beside the FP64 accumulation of Z, the unevaluated pair
// hi + lo that the stencil of F(Y_n) reads.  It is advanced with the same two
// increments by error-free transformations in FP32 (Knuth's TwoSum; the
// product error c*x - fl(c*x) by one FMA), so it follows Z to the pair's
// precision without converting Z every step.  The _rn intrinsics keep the
// compiler from contracting the products into the sums.
__device__ __forceinline__ float2 ff_axpy(float2 z, float c, float x)
{
    const float p = __fmul_rn(c, x);
    const float pe = __fmaf_rn(c, x, -p);
    const float s = __fadd_rn(z.x, p);
    const float bb = __fsub_rn(s, z.x);
    const float e = __fadd_rn(__fadd_rn(__fsub_rn(z.x, __fsub_rn(s, bb)), __fsub_rn(p, bb)), __fadd_rn(z.y, pe));
    const float hi = __fadd_rn(s, e);
    return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

__device__ __forceinline__ float2 split_df(double z)
{
    const float hi = __double2float_rn(z);
    const float lo = __double2float_rn(z - (double)hi);
    return make_float2(hi, lo);
}

// N directional solves: the first from `from` into `to`, the rest in place.
template <int N, typename TK, int KIND>
__device__ __forceinline__ void sweeps_into(const Shape<N>& s, const TK* lu, const TK* from, TK* to,
                                            int rank, int gsize, unsigned gm)
{
    constexpr bool WARP = KIND == kWarpGroup;
    const TK* src = from;
#pragma unroll
    for (int ax = 0; ax < N; ++ax) {
        if ((s.skip >> ax) & 1) continue;  // folded into the solve along s.last
        lsweep<N, TK, KIND>(s, ax, lu, src, to, rank, gsize, gm, NoEpi());
        gsync<WARP>(gm);
        src = to;
    }
}

// Multilinear interpolation at the spot x* = (F_1(0), ..., V0) of Y = G + Z
// (Sec. 5.1).  The 2^N corners of the containing cell are shared among up to
// 32 lanes of the group (a whole warp group, or the first warp of a CTA),
// which sum them by a shuffle reduction.  Z, zero on Outer nodes, is read
// only at corners of nonzero weight whose every index is Inner.
template <int N, bool WARP>
__device__ __forceinline__ void interp_spot(const Shape<N>& s, const InstDev& P, const double* pay,
                                            const double* Z, double* u_out, int rank, int gsize, unsigned gm)
{
    const int il = gsize < 32 ? gsize : 32;
    if (rank < il) {
        int c[N];
        double w[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const double sx = P.xs[i] * (double)s.M[i];  // x / h_i, h_i = Fmax_i / M_i
            int ci = (int)floor(sx);
            ci = ci > s.M[i] - 1 ? s.M[i] - 1 : ci;
            ci = ci < 0 ? 0 : ci;
            c[i] = ci;
            w[i] = sx - (double)ci;
        }
        // Corner `corner` goes to lane corner mod il, so a lane's corners
        // share their lowest lb bits: the weight product, the payoff's
        // running discount product and sum, and the node offset over those
        // axes are formed once per lane, in the same order as per corner.
        const int lb = 31 - __clz(il);
        double wl = 1.0, Pl = 1.0, Sl = 0.0;
        int tl = 0;
        bool ol = false;
        const double* Bv = pay + s.phalf;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (i < lb) {
                const int bit = (rank >> i) & 1;
                const int jj = c[i] + bit;
                wl *= bit ? w[i] : 1.0 - w[i];
                ol |= jj == 0;
                tl += (jj - 1) << s.sh[i];
                if (i < N - 1) {
                    Pl *= Bv[s.poff[i] + jj];
                    Sl = fma(pay[s.poff[i] + jj], Pl, Sl);
                }
            }
        }
        const int j0l = c[0] + (rank & 1);  // the caplet's rate index when axis 0 is a lane bit
        // When V's bit is one the lane loops over, the two V corners of a
        // rate corner share its payoff (g does not depend on V): the loop
        // runs over the rate bits and visits both V corners inside.
        const bool vloop = N - 1 >= lb;
        const int nbits = vloop ? N - 1 : N;
        double u = 0.0;
        for (int corner = rank; corner < (1 << nbits); corner += il) {
            double wt = wl, Pc = Pl, Sc = Sl;
            int t = tl;
            bool outer = ol;
            int j0 = j0l;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                if (i >= lb && i < nbits) {
                    const int bit = (corner >> i) & 1;
                    const int jj = c[i] + bit;
                    wt *= bit ? w[i] : 1.0 - w[i];
                    outer |= jj == 0;
                    t += (jj - 1) << s.sh[i];
                    if (i == 0) j0 = jj;
                    if (i < N - 1) {
                        Pc *= Bv[s.poff[i] + jj];
                        Sc = fma(pay[s.poff[i] + jj], Pc, Sc);
                    }
                }
            }
            const double g = (P.payoff == 0) ? fmax(pay[s.poff[0] + j0], 0.0) : fmax(Sc, 0.0);
            if (!vloop) {
                if (wt == 0.0) continue;
                const double zv = outer ? 0.0 : Z[s.padded(t)];
                u += wt * (g + zv);
                continue;
            }
            // the V weights of a rate corner sum to its weight wt; Z is 0 on
            // Outer nodes, so only a corner whose rate indices are all Inner
            // reads it
            u = fma(wt, g, u);
            if (outer) continue;
#pragma unroll
            for (int bit = 0; bit < 2; ++bit) {
                const int jj = c[N - 1] + bit;
                const double wv = wt * (bit ? w[N - 1] : 1.0 - w[N - 1]);
                if (wv == 0.0 || jj == 0) continue;
                u = fma(wv, Z[s.padded(t + ((jj - 1) << s.sh[N - 1]))], u);
            }
        }
        const unsigned im = WARP ? gm : 0xffffffffu;
        for (int off = il >> 1; off > 0; off >>= 1) u += __shfl_xor_sync(im, u, off, il);
        if (rank == 0) *u_out = u;
    }
}

// ------------------------------------------------------------- one grid
template <int N, bool MIXED, int KIND>
__device__ void solve_item(const SolveArgs& a, const Item& it, unsigned char* base, int rank,
                           int gsize)
{
    using TK = typename std::conditional<MIXED, float, double>::type;
    constexpr bool WARP = KIND == kWarpGroup;
    const InstDev& P = a.insts[it.inst];
    constexpr int RMAX = 1 << (WARP ? kRowsLogWarp : (MIXED ? kRowsLogCtaMixed : kRowsLogCta));
    const int tlog = 31 - __clz(gsize);
    const unsigned gm = WARP ? group_mask(tlog) : 0xffffffffu;
    Shape<N> s;
    // single-row solves are folded into another solve (not for global-memory
    // groups); into a rate-axis solve only where the register sweep is called
    // out of line (N <= 4), since the epilogue then moves to a runtime axis
    constexpr bool kFoldV = N <= 4 && KIND != kMemGroup;
    // mixed-precision CTA groups keep Z and dt F(Y_n) in their block's global
    // slice and pad fewer rows, so that two CTAs fit an SM's shared memory
    constexpr bool LEAN = MIXED && KIND == kCtaGroup;
    make_shape<N>(s, it.lv, tlog, rows_log(KIND, MIXED), KIND != kMemGroup, kFoldV, P.bc != 0, false,
                  pad_rows_min(LEAN));
    const int last = kFoldV ? s.last : N - 1;  // the axis whose solve carries the epilogues
    const Layout lay = make_layout(N, it.lv, MIXED, KIND, tlog);
    Consts<double>* cd = reinterpret_cast<Consts<double>*>(base + lay.cd);
    Consts<TK>* ck = MIXED ? reinterpret_cast<Consts<TK>*>(base + lay.cf)
                           : reinterpret_cast<Consts<TK>*>(base + lay.cd);
    double* tabd = reinterpret_cast<double*>(base + lay.tabd);
    TK* tabk = MIXED ? reinterpret_cast<TK*>(base + lay.tabf) : reinterpret_cast<TK*>(tabd);
    double* pay = reinterpret_cast<double*>(base + lay.pay);
    // warp groups keep the Thomas factors on chip; a CTA group (grids of more
    // than 64 Inner nodes) keeps them in its block's slice of global scratch,
    // read through L1; a global-memory group has them in its layout
    unsigned char* gslice = a.lu_scratch + (size_t)blockIdx.x * (size_t)a.lu_stride;
    TK* lu = KIND != kCtaGroup ? reinterpret_cast<TK*>(base + lay.lu) : reinterpret_cast<TK*>(gslice);
    double* Z = LEAN ? reinterpret_cast<double*>(gslice + lay.gZ) : reinterpret_cast<double*>(base + lay.Z);
    float2* ZZ = reinterpret_cast<float2*>(base + lay.ZZ);
    TK* H = reinterpret_cast<TK*>(base + lay.H);
    float* FY = LEAN ? reinterpret_cast<float*>(gslice + lay.gFY) : reinterpret_cast<float*>(base + lay.FY);
    TK* K1 = reinterpret_cast<TK*>(base + lay.K1);
    TK* K0 = reinterpret_cast<TK*>(base + lay.K0);
    TK* Kw = reinterpret_cast<TK*>(base + lay.Kw);
    // FP64 warp groups use the difference-array stencil
    constexpr bool DIFF = !MIXED && WARP;
    double* Dd = reinterpret_cast<double*>(base + lay.D);
    double* Cc = reinterpret_cast<double*>(base + lay.C);
    const int Lp = lay.Lp;

    // 1. coefficient and payoff tables, constants
    build_tables<N>(s, P, tabd, pay, cd, rank, gsize);
    gsync<WARP>(gm);
    if constexpr (MIXED) {
        for (int q = rank; q < lay.ntab; q += gsize) tabk[q] = (TK)tabd[q];
        convert_consts<TK>(*cd, ck, rank, gsize);
    }
    if constexpr (KIND == kMemGroup) {
        gsync<WARP>(gm);
        pcr_setup_mem<N, TK>(s, tabd, *cd, lu, reinterpret_cast<double*>(base + lay.scr), rank, gsize, gm);
    } else {
        pcr_setup<N, TK, RMAX>(s, tabd, *cd, lu, rank, gsize, gm);
    }
    if constexpr (MIXED) gsync<WARP>(gm);  // the FP32 tables and constants are complete

    // 2. H = F(G)/V^2 on the rate grid (FP64), Z from the state or zero
    for (int tr = rank; tr < s.Lr; tr += gsize) {
        int j[N];
        decode<N>(s, tr, j);
        if (dirichlet_node(s, tr)) H[tr] = TK(0);
        else if constexpr (MIXED) H[tr] = (TK)payoff_H_fast<N>(s, pay, P.payoff, j, (const float*)tabk,
                                                               *(const Consts<float>*)ck);
        else H[tr] = (TK)payoff_H<N>(s, pay, P.payoff, j, tabd, *cd);
    }
    for (int t = rank; t < s.L; t += gsize) {
        const int J = s.padded(t);
        double z = 0.0;
        if (a.flags & kLoadState) {
            int j[N];
            decode<N>(s, t, j);
            z = a.state[it.state_off + t] - payoff_at<N>(s, pay, P.payoff, j);
        }
        Z[J] = z;
        if constexpr (MIXED) ZZ[J] = split_df(z);
    }
    gsync<WARP>(gm);
    if constexpr (DIFF) {
        build_node_coefs<N>(s, tabd, *cd, (const double*)H, Cc, Lp, rank, gsize);
        gsync<WARP>(gm);
    }

    const int Lr1 = s.Lr - 1;
    const TK* v2 = tabk + s.toff[N - 1] - 1;  // v2[j_V], 1-based
    const TK* luc = lu;
    const double theta = P.theta;

    using CI = CIdx<N>;
    for (int n = 0; n < a.steps; ++n) {
        // ---- stage 1: K^(0) = dt F(Y_n)
        if constexpr (DIFF) {
            diff_pass<N>(s, Z, Dd, Lp, rank, gsize);
            gsync<WARP>(gm);
            for (int t = rank; t < s.L; t += gsize) {
                int j[N];
                decode<N>(s, t, j);
                const int J = s.padded(t);
                if (dirichlet_node(s, t)) K0[J] = TK(0);
                else K0[J] = (TK)diff_F<N>(s, j, J, Z, Dd, Cc, Lp, Cc[CI::fg * Lp + J]);
            }
        } else for (int t = rank; t < s.L; t += gsize) {
            int j[N];
            decode<N>(s, t, j);
            const int J = s.padded(t);
            if (dirichlet_node(s, t)) {  // no stencil on a Dirichlet face (its far neighbour is not stored)
                K0[J] = TK(0);
                if constexpr (MIXED) FY[J] = 0.f;
                continue;
            }
            TK k0;
            if constexpr (MIXED) {
                const float acc = stencil_acc<N, float>(s, j, J, DFSrc{ZZ}, (const float*)tabk,
                                                        *(const Consts<float>*)ck);
                k0 = (TK)(ck->dt * v2[j[N - 1]] * ((float)H[t & Lr1] + acc));
                FY[J] = (float)k0;
            } else {
                const double acc = stencil_acc<N, double>(s, j, J, ArrSrc<double>{Z},
                                                          (const double*)tabk,
                                                          *(const Consts<double>*)ck);
                k0 = (TK)(cd->dt * (double)v2[j[N - 1]] * ((double)H[t & Lr1] + acc));
            }
            K0[J] = k0;
        }
        gsync<WARP>(gm);
        sweeps_into<N, TK, KIND>(s, luc, K0, Kw, rank, gsize, gm);
        // refinement: Khat = 2 K^(0) - K^(N) + theta dt F(K^(N))
        if constexpr (DIFF) {
            diff_pass<N>(s, (const double*)Kw, Dd, Lp, rank, gsize);
            gsync<WARP>(gm);
            for (int t = rank; t < s.L; t += gsize) {
                int j[N];
                decode<N>(s, t, j);
                const int J = s.padded(t);
                if (dirichlet_node(s, t)) {
                    K0[J] = TK(0);
                    continue;
                }
                const double f = diff_F<N>(s, j, J, (const double*)Kw, Dd, Cc, Lp, 0.0);
                K0[J] = (TK)(2.0 * (double)K0[J] - (double)Kw[J] + theta * f);
            }
        } else for (int t = rank; t < s.L; t += gsize) {
            int j[N];
            decode<N>(s, t, j);
            const int J = s.padded(t);
            if (dirichlet_node(s, t)) {
                K0[J] = TK(0);
                continue;
            }
            const TK acc = stencil_acc<N, TK>(s, j, J, ArrSrc<TK>{Kw}, tabk, *ck);
            K0[J] = TK(2) * K0[J] - Kw[J] + ck->thdt * v2[j[N - 1]] * acc;
        }
        gsync<WARP>(gm);
        // N solves into K1 (single-row axes folded into the solve along
        // `last`); the last one also forms the stage-2 argument
        {
            const TK* src = K0;
            for (int ax = 0; ax < N; ++ax) {
                if ((s.skip >> ax) & 1) continue;
                if (!MIXED && ax == last) {  // FP64: Kw = Z + a21 K1
                    lsweep<N, TK, KIND>(s, ax, luc, src, K1, rank, gsize, gm, [=](int J, TK x) {
                        Kw[J] = (TK)(Z[J] + kA21 * (double)x);
                    });
                } else {
                    lsweep<N, TK, KIND>(s, ax, luc, src, K1, rank, gsize, gm, NoEpi());
                }
                gsync<WARP>(gm);
                src = K1;
            }
        }
        // ---- stage 2: K^(0) = dt F(Y_n + a21 K1) + q21 K1
        if constexpr (DIFF) {
            diff_pass<N>(s, (const double*)Kw, Dd, Lp, rank, gsize);
            gsync<WARP>(gm);
            for (int t = rank; t < s.L; t += gsize) {
                int j[N];
                decode<N>(s, t, j);
                const int J = s.padded(t);
                if (dirichlet_node(s, t)) K0[J] = TK(0);
                else K0[J] = (TK)diff_F<N>(s, j, J, (const double*)Kw, Dd, Cc, Lp,
                                           fma(kQ21, (double)K1[J], Cc[CI::fg * Lp + J]));
            }
        } else for (int t = rank; t < s.L; t += gsize) {
            int j[N];
            decode<N>(s, t, j);
            const int J = s.padded(t);
            if (dirichlet_node(s, t)) {
                K0[J] = TK(0);
                continue;
            }
            if constexpr (MIXED) {
                const float acc = stencil_acc<N, float>(s, j, J, ArrSrc<float>{(const float*)K1},
                                                        (const float*)tabk,
                                                        *(const Consts<float>*)ck);
                const float a21dt = (float)kA21 * (float)ck->dt;
                K0[J] = (TK)(FY[J] + a21dt * (float)v2[j[N - 1]] * acc + (float)kQ21 * (float)K1[J]);
            } else {
                const double acc = stencil_acc<N, double>(s, j, J, ArrSrc<double>{(const double*)Kw},
                                                          (const double*)tabk,
                                                          *(const Consts<double>*)ck);
                K0[J] = (TK)(cd->dt * (double)v2[j[N - 1]] * ((double)H[t & Lr1] + acc) +
                             kQ21 * (double)K1[J]);
            }
        }
        gsync<WARP>(gm);
        sweeps_into<N, TK, KIND>(s, luc, K0, Kw, rank, gsize, gm);
        if constexpr (DIFF) {
            diff_pass<N>(s, (const double*)Kw, Dd, Lp, rank, gsize);
            gsync<WARP>(gm);
            for (int t = rank; t < s.L; t += gsize) {
                int j[N];
                decode<N>(s, t, j);
                const int J = s.padded(t);
                if (dirichlet_node(s, t)) {
                    K0[J] = TK(0);
                    continue;
                }
                const double f = diff_F<N>(s, j, J, (const double*)Kw, Dd, Cc, Lp, 0.0);
                K0[J] = (TK)(2.0 * (double)K0[J] - (double)Kw[J] + theta * f);
            }
        } else for (int t = rank; t < s.L; t += gsize) {
            int j[N];
            decode<N>(s, t, j);
            const int J = s.padded(t);
            if (dirichlet_node(s, t)) {
                K0[J] = TK(0);
                continue;
            }
            const TK acc = stencil_acc<N, TK>(s, j, J, ArrSrc<TK>{Kw}, tabk, *ck);
            K0[J] = TK(2) * K0[J] - Kw[J] + ck->thdt * v2[j[N - 1]] * acc;
        }
        gsync<WARP>(gm);
        // N solves in place; the last one accumulates Y_{n+1} = Y_n + b1 K1 + b2 K2
        for (int ax = 0; ax < N; ++ax) {
            if ((s.skip >> ax) & 1) continue;
            if (ax == last) {
                lsweep<N, TK, KIND>(s, ax, luc, K0, K0, rank, gsize, gm, [=](int J, TK x) {
                    const double z = fma(kB2, (double)x, fma(kB1, (double)K1[J], Z[J]));
                    Z[J] = z;
                    if constexpr (MIXED)
                        ZZ[J] = ff_axpy(ff_axpy(ZZ[J], (float)kB1, (float)K1[J]), (float)kB2, (float)x);
                });
            } else {
                lsweep<N, TK, KIND>(s, ax, luc, K0, K0, rank, gsize, gm, NoEpi());
            }
            gsync<WARP>(gm);
        }
    }

    // 3. keep the state (Y on Inner nodes) if asked
    if (a.flags & kStoreState) {
        for (int t = rank; t < s.L; t += gsize) {
            int j[N];
            decode<N>(s, t, j);
            a.state[it.state_off + t] = payoff_at<N>(s, pay, P.payoff, j) + Z[s.padded(t)];
        }
    }
    // 4. multilinear interpolation at the spot
    interp_spot<N, WARP>(s, P, pay, Z, a.u_out + it.out_idx, rank, gsize, gm);
    gsync<WARP>(gm);  // the group's shared memory is reused by its next grid
}

// ---------------------------------------------- mixed precision, any N
// The mixed-precision solver keeps the grid's shape and a table of its
// active axes (those with more than one Inner row) in shared memory and walks
// that table with run-time loops, so one copy of the stencil and of each line
// sweep serves every grid of every dimension: the code stays small enough for
// the instruction cache and no per-thread copy of the shape spills to local
// memory.  An axis with one Inner row contributes only its second difference
// -2 x0 (both neighbours are zero: the Outer node and its ghost reflection),
// and no cross or drift term (every node lies on its upper face); those
// contributions are summed into one coefficient per grid.

static_assert(sizeof(Shape<2>) <= shape_bytes(2) && sizeof(Shape<8>) <= shape_bytes(8),
              "Shape exceeds its reserved shared memory");

template <int N>
__device__ void build_act(const Shape<N>& s, const Consts<float>& c, const float* tab, ActAxes& A)
{
    int n = 0;
    float cin = 0.f;
    for (int i = 0; i < N; ++i) {
        if (s.M[i] > 1) {
            A.rec[n].sh = s.sh[i];
            A.rec[n].msk = s.M[i] - 1;
            A.rec[n].nfm = s.nf[i] - 1;
            A.rec[n].M = s.M[i];
            A.rec[n].Sp = s.Sp[i];
            A.rec[n].toff = s.toff[i];
            A.ax[n] = i;
            A.g2[n] = c.g2[i];
            A.rec[n].drift = (i >= 1 && i < N - 1) ? 1 : 0;
            ++n;
        } else {
            cin += (i < N - 1) ? tab[s.toff[i]] : c.cV;  // the coefficient at j = 1
        }
    }
    A.n = n;
    A.nr = (s.M[N - 1] > 1) ? n - 1 : n;
    A.cinact = cin;
    int slot = 0;
    for (int q = 0; q < n; ++q) A.rec[q].dslot = A.rec[q].drift ? slot++ : -1;
    for (int q = 0; q < n; ++q) {
        const int i = A.ax[q];
        for (int r = 0; r < kMaxDim; ++r) {
            A.cx[q][r] = 0.f;
            A.drh[q][r] = 0.f;
        }
        if (i >= N - 1) continue;
        for (int r = q + 1; r < n; ++r) {
            const int k = A.ax[r];
            A.cx[q][r] = (k < N - 1) ? c.rm[upair(i, k)] : c.sm[i];
        }
        float sc = 0.f;
        if (A.rec[q].drift) {
            for (int r = 1; r <= i; ++r)
                if (s.M[r] == 1) sc += c.rh[ltri(i, r)] * tab[s.toff[r] + 2];  // j_r = 1
            for (int r = 0; r <= q; ++r)
                if (A.ax[r] >= 1) A.drh[q][r] = c.rh[ltri(i, A.ax[r])];
        }
        A.sconst[q] = sc;
    }
    int ns = 0;
    for (int i = 0; i < N; ++i) {
        if ((s.skip >> i) & 1) continue;  // folded into the solve along s.last
        A.sv[2 * ns] = s.luoff[i];
        A.sv[2 * ns + 1] = s.sh[i] | (s.M[i] << 8) | (i << 16) | ((i < N - 1 ? 1 : 0) << 24) |
                           (((s.dense >> i) & 1) << 25);
        ++ns;
    }
    A.ns = ns;
}

// Sketch 1 divided by V^2 at two nodes of a lane at once (t[0], t[1];
// padded indices J), from the active-axis table: the same terms as
// stencil_acc (second differences with the Neumann ghost, cross differences
// and drift off the upper faces, zero Outer values), with the inactive axes'
// second differences folded into one coefficient and the drift coefficients
// taken per node from DR.  The table entries of an axis or a pair are loaded
// once for both nodes, and the two accumulations are independent chains.
// Both nodes must be Inner (a caller substitutes an Inner node for an unused
// one and discards its result).
template <class Src>
__device__ __forceinline__ void stencil_act2(const ActAxes& A, const float* __restrict__ tab, float cV,
                                             const int (&t)[2], const int (&J)[2], const Src& src, float (&acc)[2],
                                             const float* __restrict__ DR, int Lp)
{
    using V = typename Src::V;
    V x0[2];
    float xv[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        x0[k] = src.ctr(J[k]);
        xv[k] = Src::val(x0[k]);
        acc[k] = A.cinact * (-2.f * xv[k]);
    }
    const int n = A.n, nr = A.nr;
#pragma unroll 1
    for (int q = 0; q < n; ++q) {
        const int4 q0 = reinterpret_cast<const int4*>(&A.rec[q])[0];  // sh, msk, nfm, Sp
        const int4 q1 = reinterpret_cast<const int4*>(&A.rec[q])[1];  // toff, M, drift, dslot
        const int sh = q0.x, msk = q0.y, nfm = q0.z, Sp = q0.w, to = q1.x;
        const bool rate = q < nr;
        int jm[2];
        bool lo[2], top[2];
        float dp[2], dm[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            jm[k] = (t[k] >> sh) & msk;  // j - 1
            lo[k] = jm[k] > 0;
            top[k] = jm[k] == nfm;
            const V m = src.nb(J[k], -Sp, lo[k], 0, 0, 0, 0);
            const V p = top[k] ? m : src.nb(J[k], Sp, true, 0, 0, 0, 0);
            dp[k] = Src::diff(p, x0[k]);
            dm[k] = Src::diff(x0[k], m);
            acc[k] += (rate ? tab[to + jm[k]] : cV) * (dp[k] - dm[k]);
        }
        if (rate && !(top[0] && top[1])) {
            const int Mq = q1.y;
            float inner[2] = {0.f, 0.f};
#pragma unroll 1
            for (int r = q + 1; r < n; ++r) {
                const int4 r0 = reinterpret_cast<const int4*>(&A.rec[r])[0];
                const int mr = r0.y, shr = r0.x, nfr = r0.z, Sr = r0.w;
                const float cx = A.cx[q][r];
                const bool vr = r >= nr;
                int pw = 0;
                if (!vr) {
                    const int2 r1 = reinterpret_cast<const int2*>(&A.rec[r])[2];  // toff, M
                    pw = r1.x + r1.y;
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int jr = (t[k] >> shr) & mr;
                    if (!top[k] && jr != nfr) {
                        const bool lr = jr > 0;
                        const V pp = src.nb(J[k], Sp + Sr, true, 0, 0, 0, 0);
                        const V pm = src.nb(J[k], Sp - Sr, lr, 0, 0, 0, 0);
                        const V mp = src.nb(J[k], -Sp + Sr, lo[k], 0, 0, 0, 0);
                        const V mm = src.nb(J[k], -Sp - Sr, lo[k] && lr, 0, 0, 0, 0);
                        const float mix = Src::diff(pp, pm) - Src::diff(mp, mm);
                        inner[k] += (vr ? cx : cx * tab[pw + jr]) * mix;
                    }
                }
            }
            if (q1.z) {  // drift of rates 2..N-1 (eq. coef_adv): its per-node coefficient
                const float* dr = DR + q1.w * Lp;
#pragma unroll
                for (int k = 0; k < 2; ++k) inner[k] += dr[J[k]] * (dp[k] + dm[k]);
            }
#pragma unroll
            for (int k = 0; k < 2; ++k)
                if (!top[k]) acc[k] += tab[to + Mq + jm[k]] * inner[k];
        }
    }
}


// One grid of a mixed-precision warp group: the F evaluations and line
// solves in FP32 on the increments, Z accumulated in FP64 beside its hi/lo
// float pair, F of the payoff (H), the interpolation and the state in FP64.
// Each step runs four phases, each one F evaluation (right-hand side r)
// followed by the directional solves of r:
//   0: r = dt F(Y_n) (kept as FY),              solved into Kw
//   1: r = 2 FY - Kw + theta dt F_0(Kw),        solved into K1
//   2: r = FY + a21 dt F_0(K1) + q21 K1 (kept in K0), solved into Kw
//   3: r = 2 K0 - Kw + theta dt F_0(Kw),        solved into K0, then
//      Y_{n+1} = Y_n + b1 K1 + b2 K2 (eq. coef_W2).
template <int N, int KIND>
__device__ void solve_item_mixed(const SolveArgs& a, const Item& it, unsigned char* base, unsigned char* meta,
                                 int rank, int gsize)
{
    static_assert(KIND == kWarpGroup, "the register-resident phases need at most two nodes per lane");
    constexpr bool WARP = true;
    const InstDev& P = a.insts[it.inst];
    constexpr int RMAX = 1 << (WARP ? kRowsLogWarp : kRowsLogCtaMixed);
    const int tlog = 31 - __clz(gsize);
    const unsigned gm = WARP ? group_mask(tlog) : 0xffffffffu;
    Shape<N>& s = *reinterpret_cast<Shape<N>*>(meta);
    ActAxes& A = *reinterpret_cast<ActAxes*>(meta + shape_bytes(N));
    // single-row solves are folded into another solve
    if (rank == 0) make_shape<N>(s, it.lv, tlog, rows_log(KIND, true), true, true, P.bc != 0, true);
    gsync<WARP>(gm);
    const Layout lay = make_layout(N, it.lv, true, KIND, tlog);
    Consts<double>* cd = reinterpret_cast<Consts<double>*>(base + lay.cd);
    Consts<float>* ck = reinterpret_cast<Consts<float>*>(base + lay.cf);
    double* tabd = reinterpret_cast<double*>(base + lay.tabd);
    float* tabk = reinterpret_cast<float*>(base + lay.tabf);
    double* pay = reinterpret_cast<double*>(base + lay.pay);
    float* lu = reinterpret_cast<float*>(base + lay.lu);
    double* Z = reinterpret_cast<double*>(base + lay.Z);
    float2* ZZ = reinterpret_cast<float2*>(base + lay.ZZ);
    float* H = reinterpret_cast<float*>(base + lay.H);
    float* FY = reinterpret_cast<float*>(base + lay.FY);
    float* K1 = reinterpret_cast<float*>(base + lay.K1);
    float* K0 = reinterpret_cast<float*>(base + lay.K0);
    float* Kw = reinterpret_cast<float*>(base + lay.Kw);

    // 1. coefficient and payoff tables, constants, line-solve factors
    build_tables<N, true>(s, P, tabd, pay, cd, rank, gsize);
    gsync<WARP>(gm);
    for (int q = rank; q < lay.ntab; q += gsize) tabk[q] = (float)tabd[q];
    convert_consts<float>(*cd, ck, rank, gsize);
    pcr_setup<N, float, RMAX, float>(s, tabd, *cd, lu, rank, gsize, gm);
    dense_setup<N>(s, tabd, *cd, lu, rank, gsize);
    gsync<WARP>(gm);  // the FP32 tables and constants are complete
    // 2. H = F(G)/V^2 on the rate grid (payoff differences in FP64), Z from the state or zero
    for (int tr = rank; tr < s.Lr; tr += gsize) {
        int j[N];
        decode<N>(s, tr, j);
        H[tr] = dirichlet_node(s, tr) ? 0.f : payoff_H_fast<N>(s, pay, P.payoff, j, tabk, *ck);
    }
    for (int t = rank; t < s.L; t += gsize) {
        const int J = s.padded(t);
        double z = 0.0;
        if (a.flags & kLoadState) {
            int j[N];
            decode<N>(s, t, j);
            z = a.state[it.state_off + t] - payoff_at<N>(s, pay, P.payoff, j);
        }
        Z[J] = z;
        ZZ[J] = split_df(z);
    }
    gsync<WARP>(gm);
    if (rank == 0) build_act<N>(s, *ck, tabk, A);
    gsync<WARP>(gm);
    // per-node drift coefficients S_i g2_i, S_i = sum over rates 2..i of
    // rho_ir alpha_r tau_r F_r^beta / (1 + tau_r F_r) (eq. coef_adv)
    float* DR = reinterpret_cast<float*>(base + lay.DR);
    const int Lp = lay.Lp;
    if constexpr (WARP) {
        for (int t = rank; t < s.L; t += gsize) {
            const int J = s.padded(t);
            for (int q = 0; q < A.n; ++q) {
                if (!A.rec[q].drift) continue;
                float S = A.sconst[q];
                for (int r = 0; r <= q; ++r) {
                    const float w = A.drh[q][r];
                    if (w != 0.f) S += w * tabk[A.rec[r].toff + 2 * A.rec[r].M + ((t >> A.rec[r].sh) & A.rec[r].msk)];
                }
                DR[A.rec[q].dslot * Lp + J] = S * A.g2[q];
            }
        }
        gsync<WARP>(gm);
    }

    const int Lr1 = s.Lr - 1;
    const int shV = s.sh[N - 1], mV = s.M[N - 1] - 1;
    const float* v2 = tabk + s.toff[N - 1];  // v2[j_V - 1]
    const float cV = ck->cV, dt = ck->dt, thdt = ck->thdt;
    const float a21dt = (float)kA21 * dt;
    const int last = s.last;
    const int L = s.L;
    // a Dirichlet rate axis of one row leaves no Inner node: F is 0 everywhere
    bool all_dir = false;
    for (int i = 0; i < N - 1; ++i) all_dir |= ((s.dmask >> i) & 1) && s.M[i] == 1;
    // The group's nodes stay in registers through a phase: lane `rank` holds
    // t = rank and, when the grid has more nodes than the group has lanes,
    // t = rank + gsize (a warp group has at least half as many lanes as its
    // grid has nodes: the host sizes it so).
    const bool two = L > gsize;
    // The lane's nodes are fixed for the whole time loop: slot k holds node
    // rank + k gsize when that is below L (its padded index Jo[k], else -1).
    // The stencil evaluates a slot that is unused or holds Dirichlet data
    // (eq. bound1_0: its far neighbour is not stored) as node 0 (always Inner
    // when any node is) and discards the result.
    int t[2], J[2], Jo[2];
    bool use[2];
    float vv[2];  // V^2 of the slot's node
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int tk = rank + k * gsize;
        const bool in = tk < L;
        use[k] = in && !dirichlet_node(s, tk);
        t[k] = use[k] ? tk : 0;
        J[k] = s.padded(t[k]);
        Jo[k] = in ? s.padded(tk) : -1;
        vv[k] = in ? v2[(tk >> shV) & mV] : 0.f;
    }
    const bool eval = (use[0] || use[1]) && !all_dir;
    for (int n = 0; n < a.steps; ++n) {
#pragma unroll 1
        for (int ph = 0; ph < 4; ++ph) {
            float acc[2];
            acc[0] = acc[1] = 0.f;
            if (eval) {
                if (ph == 0) stencil_act2(A, tabk, cV, t, J, DFSrc{ZZ}, acc, DR, Lp);
                else stencil_act2(A, tabk, cV, t, J, ArrSrc<float>{ph == 2 ? K1 : Kw}, acc, DR, Lp);
            }
            // the right-hand side of the phase's solves (its own node only):
            // ph 0: dt F(Y_n); ph 1 and 3: the refinement 2 k - k_prev + theta dt A k;
            // ph 2: the second stage's right-hand side (kept in K0 for ph 3)
            float x[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                x[k] = 0.f;
                if (!use[k]) continue;
                const int Jk = J[k];
                if (ph == 0) {
                    x[k] = dt * vv[k] * (H[t[k] & Lr1] + acc[k]);
                    FY[Jk] = x[k];
                } else if (ph == 1) {
                    x[k] = 2.f * FY[Jk] - Kw[Jk] + thdt * vv[k] * acc[k];
                } else if (ph == 2) {
                    x[k] = FY[Jk] + a21dt * vv[k] * acc[k] + (float)kQ21 * K1[Jk];
                    K0[Jk] = x[k];
                } else {
                    x[k] = 2.f * K0[Jk] - Kw[Jk] + thdt * vv[k] * acc[k];
                }
            }
            // directional solves in ascending axis order (single-row axes
            // folded into the solve along `last`): axes of 2..8 rows by their
            // explicit inverses in registers, longer ones by the line solve
            // through shared memory, in place in the phase's target
            float* dst = (ph == 1) ? K1 : (ph == 3 ? K0 : Kw);
            bool in_smem = false;  // the values live in dst, not in x
            const int ns = A.ns;
#pragma unroll 1
            for (int q = 0; q < ns; ++q) {
                const int2 e = reinterpret_cast<const int2*>(A.sv)[q];
                if ((e.y >> 25) & 1) {
                    if (in_smem) {
#pragma unroll
                        for (int k = 0; k < 2; ++k)
                            if (Jo[k] >= 0) x[k] = dst[Jo[k]];
                        in_smem = false;
                    }
                    const float* C = lu + e.x;
                    const int sha = e.y & 0xff, Ma = (e.y >> 8) & 0xff;
                    const bool rate = (e.y >> 24) & 1;
                    if (Ma == 2) dense_mix<2>(C, sha, shV, mV, rate, rank, gsize, tlog, two, gm, x);
                    else if (Ma == 4) dense_mix<4>(C, sha, shV, mV, rate, rank, gsize, tlog, two, gm, x);
                    else dense_mix<8>(C, sha, shV, mV, rate, rank, gsize, tlog, two, gm, x);
                } else {
                    if (!in_smem) {
#pragma unroll
                        for (int k = 0; k < 2; ++k)
                            if (Jo[k] >= 0) dst[Jo[k]] = x[k];
                        gsync<WARP>(gm);
                        in_smem = true;
                    }
                    sweep<N, float, RMAX>(s, (e.y >> 16) & 0xff, lu, dst, dst, rank, gsize, gm, NoEpi());
                    gsync<WARP>(gm);
                }
            }
            // the phase's result, and at the end of a step the update
            // Z_{n+1} = Z_n + b1 k1 + b2 k2 (FP64 and its float-float copy)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int Jk = Jo[k];
                if (Jk < 0) continue;
                const float xk = in_smem ? dst[Jk] : x[k];
                if (!in_smem) dst[Jk] = xk;
                if (ph == 3) {
                    Z[Jk] = fma(kB2, (double)xk, fma(kB1, (double)K1[Jk], Z[Jk]));
                    ZZ[Jk] = ff_axpy(ff_axpy(ZZ[Jk], (float)kB1, K1[Jk]), (float)kB2, xk);
                }
            }
            gsync<WARP>(gm);
        }
    }

    // 3. keep the state (Y on Inner nodes) if asked
    if (a.flags & kStoreState) {
        for (int t = rank; t < s.L; t += gsize) {
            int j[N];
            decode<N>(s, t, j);
            a.state[it.state_off + t] = payoff_at<N>(s, pay, P.payoff, j) + Z[s.padded(t)];
        }
    }
    // 4. interpolation at the spot
    interp_spot<N, WARP>(s, P, pay, Z, a.u_out + it.out_idx, rank, gsize, gm);
    gsync<WARP>(gm);  // the group's shared memory is reused by its next grid
}

// The solver kernel.  CTA groups: one grid per block at a time from the
// launch's work counter.  Warp groups: a persistent multi-class launch -- every
// warp walks the launch's class list (ordered largest grids first) and takes
// chunks of 32 >> glog grids from each class's counter until it is exhausted,
// then moves on, so classes of uneven instances share one launch and no warp
// waits for another.
template <int N, bool MIXED, int KIND>
__global__ void __launch_bounds__(KIND == kWarpGroup ? 128 : kCtaMaxThreads, KIND == kWarpGroup ? (MIXED ? kWarpBlocksMixed : 3) : ((KIND == kMemGroup || MIXED) ? 2 : 1)) solve_kernel(SolveArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    if constexpr (KIND == kWarpGroup) {
        const int warp = threadIdx.x >> 5;
        const int lane = threadIdx.x & 31;
        unsigned char* wbase = smem + (size_t)warp * (size_t)a.smem_warp;
        int c = 0;
        while (c < a.n_classes) {
            const ClassDesc cd = a.classes[c];
            int chunk = 0;
            if (lane == 0) chunk = atomicAdd(a.queue + cd.qidx, 32 >> cd.glog);
            chunk = __shfl_sync(0xffffffffu, chunk, 0);
            if (chunk >= cd.item_count) {
                ++c;
                continue;
            }
            const int item = chunk + (lane >> cd.glog);
            bool take = item < cd.item_count;
            Item it{};
            if (take) {
                it = a.items[cd.item_begin + item];
                take = !a.inst_mask || a.inst_mask[it.inst] != 0;
            }
            if (take) {
                const int gsize = 1 << cd.glog;
                unsigned char* base = wbase + (size_t)(lane >> cd.glog) * (size_t)cd.smem_group;
                if constexpr (MIXED)
                    solve_item_mixed<N, kWarpGroup>(a, it, base, base, lane & (gsize - 1), gsize);
                else
                    solve_item<N, false, kWarpGroup>(a, it, base, lane & (gsize - 1), gsize);
            }
        }
    } else {
        // CTA groups: the grid in shared memory; global-memory groups: in the
        // block's slice of the scratch array
        unsigned char* base = KIND == kMemGroup ? a.lu_scratch + (size_t)blockIdx.x * (size_t)a.lu_stride : smem;
        __shared__ int s_item;
        for (;;) {
            if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
            __syncthreads();
            const int item = s_item;
            __syncthreads();
            if (item >= a.n_items) break;
            const Item it = a.items[item];
            if (a.inst_mask && a.inst_mask[it.inst] == 0) continue;  // uniform across the block
            // whole-block groups keep the unrolled stencil of solve_item in both
            // precisions: with up to 256 threads on one grid the per-node work
            // dominates, and the unrolled form, each axis's offsets in
            // registers, measured 30 % faster on the d=6 modified level-6
            // workload than the table-driven form of the warp groups
            solve_item<N, MIXED, KIND>(a, it, base, (int)threadIdx.x, (int)blockDim.x);
        }
    }
}

// Host launch / occupancy helpers, instantiated once per N.
template <int N>
const void* kernel_for(bool mixed, int kind)
{
    if (kind == kWarpGroup)
        return mixed ? (const void*)solve_kernel<N, true, kWarpGroup> : (const void*)solve_kernel<N, false, kWarpGroup>;
    if (kind == kCtaGroup)
        return mixed ? (const void*)solve_kernel<N, true, kCtaGroup> : (const void*)solve_kernel<N, false, kCtaGroup>;
    return mixed ? (const void*)solve_kernel<N, true, kMemGroup> : (const void*)solve_kernel<N, false, kMemGroup>;
}

template <int N>
int launch_impl(const SolveArgs& a, bool mixed, int kind, int block, int grid, size_t smem, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (kind == kWarpGroup) {
        if (mixed) solve_kernel<N, true, kWarpGroup><<<grid, block, smem, st>>>(a);
        else solve_kernel<N, false, kWarpGroup><<<grid, block, smem, st>>>(a);
    } else if (kind == kCtaGroup) {
        if (mixed) solve_kernel<N, true, kCtaGroup><<<grid, block, smem, st>>>(a);
        else solve_kernel<N, false, kCtaGroup><<<grid, block, smem, st>>>(a);
    } else {
        if (mixed) solve_kernel<N, true, kMemGroup><<<grid, block, smem, st>>>(a);
        else solve_kernel<N, false, kMemGroup><<<grid, block, smem, st>>>(a);
    }
    return (int)cudaGetLastError();
}

template <int N>
int occupancy_impl(bool mixed, int kind, int block, size_t smem)
{
    int nb = 0;
    const void* f = kernel_for<N>(mixed, kind);
    // The limit is an attribute of the kernel, shared by all its launches, and
    // launches of one kernel request different amounts: past the default
    // 48 KB, allow the device's opt-in maximum (less the kernel's static
    // shared memory), so that no launch depends on which query came last.
    if (smem > 48 * 1024) {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa{};
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, f) != cudaSuccess)
            return 0;
        const int lim = optin - (int)fa.sharedSizeBytes;
        if ((size_t)lim < smem ||
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess)
            return 0;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, block, smem) != cudaSuccess) return 0;
    return nb;
}

}  // namespace amfrw

#define AMFRW_INSTANTIATE(NN)                                                               \
    namespace amfrw {                                                                       \
    int launch_n##NN(const SolveArgs& a, bool m, int k, int b, int g, size_t s, void* st)   \
    {                                                                                       \
        return launch_impl<NN>(a, m, k, b, g, s, st);                                       \
    }                                                                                       \
    int occupancy_n##NN(bool m, int k, int b, size_t s) { return occupancy_impl<NN>(m, k, b, s); } \
    }
