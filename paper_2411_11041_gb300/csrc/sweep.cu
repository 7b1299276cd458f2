// Directional sweep kernels (the hot path).
//
//  k_curve_prep   once per (theta dt, sigma): assembles the substep systems
//                 (§6 eqs. SemiDiscrSplit1Dbeta / SemiDiscrSplit1Dgamma) and
//                 factors their partitioned elimination.
//  k_curve_solve  every substep: bilinear gather of the grid state onto the
//                 curve nodes (§6.1), right-hand side F - S u, the factored
//                 elimination, curve values u + dt d out; a block of BS threads
//                 holds BS/T curves of T threads each.
//  k_grid_map     one thread per grid node: curve -> grid interpolation through
//                 the nearest crossings on the node's row and column (§6), with
//                 the relative-update norms fused in.
//  k_check        one block: convergence test and the CUDA-graph loop condition.
//  *_batch        the same steps for many problems in one persistent launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kCmax = 16;      // most rows per thread of the curve solve (kept in shared memory)
constexpr int kGridThreads = 256;

// ---------------------------------------------------------------- curves
// The curve systems A = M + theta dt S are fixed for a given (theta, dt,
// sigma), so their partitioned elimination is factored once (k_curve_prep)
// and every split step only carries a right-hand side through it
// (k_curve_solve).
//
// One block of T threads per curve (T = 32..1024 chosen per curve so that a
// thread owns at most R <= kCmax rows).  Thread t owns rows [t c, t c + c) of
// the curve's m unknowns, c = ceil(m / T) (row q <-> curve node q+1).
// Downward elimination inside a chunk writes every row as
//     x_q + cp_q x_{q+1} + vp_q x_{s-1} = rp_q,   rp_q = r_q ip_q - lp_q rp_{q-1},
// an upward pass gives the chunk's first unknown in terms of the chunk ends,
// the chunk ends G_t = x_{e_t - 1} satisfy a T-equation tridiagonal system
// solved by cyclic reduction in shared memory (multipliers factored once),
// and back substitution gives every x_q.  The rows' rp values stay in shared
// memory between the passes.
//
// What is solved (§6 eqs. SemiDiscrSplit1Dbeta / SemiDiscrSplit1Dgamma, with
// the curve values carried as v = u + dt d):
//  * FP64 mode: the new curve values directly,
//        A v = dt F + (M - (1 - theta) dt S) u,
//    the same v as u + dt A^-1 (F - S u) without the update of every row;
//  * reduced-precision mode: one step of mixed-precision iterative refinement
//    of that system from the current curve values x0 = u: the residual
//    dt (F - S u) is formed in FP64, the correction A d = F - S u is solved in
//    FP32 with the factors rounded to FP32, and v = u + dt d is accumulated in
//    FP64;
//  * the steady start (eq. u0stationary): S v = F.
// Every right-hand-side row is stored times its row factor ip, so the rhs and
// the first elimination step are plain FMAs.
//
// Per-row data live in a chunk-interleaved "slot" layout: row (t, j) of a
// curve is stored at soff[curve] + j T + t, so that the j-th row of all
// threads is one coalesced access.

struct CurveArgs {
    int nx, ny;
    const double* u_even;  // grid state of the gather (by step parity)
    const double* u_odd;
    const IterState* state;
    const int* off;        // curve -> first node
    const int* soff;       // curve -> first slot
    const double* h;
    int* gcell;            // per slot: bilinear cell r*nx + i of the row's node
    double* gw;            // 4 planes per slot: the cell's corner weights of the row's node
    int* ncell;            // per node: the same cell (setup; -1 at the curves' ends)
    double* nw;            // 4 per node: the same weights (setup)
    const double* bnorm;   // per node
    const double* fval;    // per node
    const double* xi;      // per node (setup of the gather descriptors)
    const double* eta;
    const double* fextra;  // load kernel only
    double fx_scale;
    double* Fl;            // per slot: ip (dt F) in the FP64 form, ip F otherwise (B)
    double* srow;          // B: 3 planes per slot, ip (M - (1-theta) dt S) rows in the FP64
                           // form, -ip S rows otherwise; G: one plane, ip times the
                           // off-diagonal coefficient of the rhs stencil
    double* kap;           // G, per curve: diagonal / off-diagonal ratio of the rhs stencil
    int vform;             // 1: FP64 form (new values); 0: residual form or steady start
    double fscale;         // load scale of the right-hand side (dt in the FP64 form, else 1)
    int supg;              // B curves: SUPG-stabilised element forms (mass, S and load)
    double* fac;           // 4 planes per slot: cp, vp, ip, lp
    float* fac32;          // the same factors rounded to FP32 (reduced-precision mode)
    const double* lanecs[3];   // reduced-system constants of the item sets (batched launches)
    const float* lanec32s[3];
    double* v;             // per node: curve values
    double* pivmin;        // prep: the smallest |pivot| of the family (an ordered-int bit pattern)
    int n_slots;
    int R;                 // rows per thread of the launch (shared-memory stride)
    double mu, sig, td, dt;
    int paper;             // steady solve S v = F (no mass term, values out)
};

// Work items: a block of BS threads takes BS/T curves of the same block size
// T (a power of two, 32 <= T <= BS); sub-block k of the item owns curve
// item_curve[item*(BS/32) + k] (-1: empty).  T is uniform per block, so every
// __syncthreads below is reached by the whole block.
template <int BS>
struct Items {
    static constexpr int LMAX = BS == 256 ? 8 : BS == 512 ? 9 : 10;
    static constexpr int NF = 2 * LMAX + 2;  // per-thread constants: cpL, k1[LMAX], k2[LMAX], 1/B
    static constexpr int MAXC = BS / 32;
};

struct BlockChunk {
    int line, base, n, m, c, s, cnt, so, T, lt;
    bool active;
};

// chunk of the calling thread inside a work item of block size T whose curves
// are curves[0 .. BS/T-1]
__device__ __forceinline__ void item_chunk_of(const CurveArgs& a, int T, const int* curves,
                                              BlockChunk& b)
{
    b.T = T;
    int L = __ffs(b.T) - 1;
    int sb = threadIdx.x >> L;
    b.lt = threadIdx.x & (b.T - 1);
    b.line = curves[sb];
    b.active = b.line >= 0;
    b.base = b.n = b.m = b.c = b.s = b.cnt = b.so = 0;
    if (!b.active) return;
    b.base = a.off[b.line];
    b.n = a.off[b.line + 1] - b.base - 1;
    b.m = b.n - 1;
    b.c = b.m > 0 ? (b.m + b.T - 1) / b.T : 0;
    b.s = b.lt * b.c;
    b.cnt = b.m > 0 ? max(0, min(b.m, b.s + b.c) - b.s) : 0;
    b.so = a.soff[b.line];
}

template <int BS>
__device__ __forceinline__ void item_chunk(const CurveArgs& a, const int* item_T,
                                           const int* item_curve, BlockChunk& b)
{
    item_chunk_of(a, item_T[blockIdx.x], item_curve + blockIdx.x * Items<BS>::MAXC, b);
}

// bilinear gather at a row's node from its cell and corner weights (slot sl)
__device__ __forceinline__ double gather_w(const double* __restrict__ u, int nx, int cell,
                                           const double* __restrict__ w, size_t NS, int sl)
{
    const double* r0 = u + cell;
    double p11 = __ldg(r0), p12 = __ldg(r0 + 1), p21 = __ldg(r0 + nx), p22 = __ldg(r0 + nx + 1);
    double v = __ldg(w + sl) * p11;
    v = fma(__ldg(w + NS + sl), p12, v);
    v = fma(__ldg(w + 2 * NS + sl), p21, v);
    return fma(__ldg(w + 3 * NS + sl), p22, v);
}

__device__ __forceinline__ double gather_at(const double* __restrict__ u, int nx, int cell,
                                            double lx, double ly)
{
    const double* r0 = u + cell;
    double p11 = __ldg(r0), p12 = __ldg(r0 + 1), p21 = __ldg(r0 + nx), p22 = __ldg(r0 + nx + 1);
    double b = p11 + lx * (p12 - p11);
    double t = p21 + lx * (p22 - p21);
    return b + ly * (t - b);
}

// SUPG parameter of a B-curve element of length h with mean |beta| b:
// tau = h / (2 b) (coth Pe - 1 / Pe), Pe = b h / (2 mu), the value that makes
// the 1D solution of -mu u'' + b u' = f nodally exact (series below Pe = 1e-3)
__device__ __forceinline__ double supg_tau(double h, double b, double mu)
{
    if (!(b > 0.0)) return 0.0;
    const double pe = b * h / (2.0 * mu);
    const double xi = pe < 1e-3 ? pe / 3.0 - pe * pe * pe / 45.0 : 1.0 / tanh(pe) - 1.0 / pe;
    return h / (2.0 * b) * xi;
}

// gather descriptors of every row's node, in slot layout (setup)
template <int BS>
__global__ void __launch_bounds__(BS) k_curve_gdesc(CurveArgs a, const int* item_T,
                                                    const int* item_curve)
{
    BlockChunk b;
    item_chunk<BS>(a, item_T, item_curve, b);
    for (int j = 0; j < b.cnt; ++j) {
        int node = b.base + b.s + j + 1;
        double x = a.xi[node], y = a.eta[node];
        int i = (int)floor(x), r = (int)floor(y);
        i = i > a.nx - 2 ? a.nx - 2 : (i < 0 ? 0 : i);
        r = r > a.ny - 2 ? a.ny - 2 : (r < 0 ? 0 : r);
        size_t sl = b.so + (size_t)j * b.T + b.lt;
        const size_t NS = a.n_slots;
        const double lx = x - i, ly = y - r;
        const double w0 = (1.0 - lx) * (1.0 - ly), w1 = lx * (1.0 - ly), w2 = (1.0 - lx) * ly, w3 = lx * ly;
        a.gcell[sl] = r * a.nx + i;
        a.gw[sl] = w0;
        a.gw[NS + sl] = w1;
        a.gw[2 * NS + sl] = w2;
        a.gw[3 * NS + sl] = w3;
        if (a.ncell) {  // the same descriptor in node order (the separate gather pass)
            a.ncell[node] = r * a.nx + i;
            a.nw[4 * (size_t)node] = w0;
            a.nw[4 * (size_t)node + 1] = w1;
            a.nw[4 * (size_t)node + 2] = w2;
            a.nw[4 * (size_t)node + 3] = w3;
        }
    }
}

// the grid state at every node of a family from the node-order descriptors
// (the same corner products, in the same order, as the solve's own gather);
// 0 at the curves' ends.  The grid by the step's parity when state is given.
__global__ void __launch_bounds__(256) k_gather_grid(long long n, const int* __restrict__ ncell,
                                                     const double* __restrict__ nw, int nx,
                                                     const double* u_even, const double* u_odd,
                                                     const IterState* state, double* __restrict__ out)
{
    if (state && state->done) return;
    const double* __restrict__ u = (state && (state->iter & 1)) ? u_odd : u_even;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int c = __ldg(ncell + k);
        double v = 0.0;
        if (c >= 0) {
            const double2 wa = *reinterpret_cast<const double2*>(nw + 4 * k);
            const double2 wb = *reinterpret_cast<const double2*>(nw + 4 * k + 2);
            const double* r0 = u + c;
            const double p11 = __ldg(r0), p12 = __ldg(r0 + 1), p21 = __ldg(r0 + nx), p22 = __ldg(r0 + nx + 1);
            v = wa.x * p11;
            v = fma(wa.y, p12, v);
            v = fma(wb.x, p21, v);
            v = fma(wb.y, p22, v);
        }
        out[k] = v;
    }
}

// load F = M f on the B curves (f + fx_scale * fextra when an extra load is given),
// stored times the row factor ip and the form's scale
template <int BS>
__global__ void __launch_bounds__(BS) k_curve_load(CurveArgs a, const int* item_T,
                                                   const int* item_curve)
{
    BlockChunk b;
    item_chunk<BS>(a, item_T, item_curve, b);
    if (b.cnt == 0) return;
    const double Mo = a.h[b.line] / 6.0;
    auto fat = [&](int k) {
        int g = b.base + k;
        double f = a.fval[g];
        if (a.fextra) {
            double x = a.xi[g], y = a.eta[g];
            int i = (int)floor(x), r = (int)floor(y);
            i = i > a.nx - 2 ? a.nx - 2 : (i < 0 ? 0 : i);
            r = r > a.ny - 2 ? a.ny - 2 : (r < 0 ? 0 : r);
            f += a.fx_scale * gather_at(a.fextra, a.nx, r * a.nx + i, x - i, y - r);
        }
        return f;
    };
    double f0 = fat(b.s), f1 = fat(b.s + 1);
    for (int j = 0; j < b.cnt; ++j) {
        double f2 = fat(b.s + j + 2);
        const size_t sl = b.so + (size_t)j * b.T + b.lt;
        double F = Mo * (f0 + 4.0 * f1 + f2);
        if (a.supg) {  // + tau int f |beta| phi' over the two elements of the row's node
            const int g = b.base + b.s + j;
            const double h = a.h[b.line];
            const double bm = a.bnorm[g], b0 = a.bnorm[g + 1], bp = a.bnorm[g + 2];
            const double tl = supg_tau(h, 0.5 * (bm + b0), a.mu), tr = supg_tau(h, 0.5 * (b0 + bp), a.mu);
            F += tl * (2.0 * f0 * bm + f0 * b0 + f1 * bm + 2.0 * f1 * b0) / 6.0 -
                 tr * (2.0 * f1 * b0 + f1 * bp + f2 * b0 + 2.0 * f2 * bp) / 6.0;
        }
        a.Fl[sl] = F * (a.fac[2 * a.n_slots + sl] * a.fscale);  // times ip (k_curve_prep) and dt or 1
        f0 = f1;
        f1 = f2;
    }
}

// 2 x 2 projective map [[a b][c d]] (the Thomas pivot recurrence); products
// are rescaled by a power of two so that long chains stay finite
struct Mob {
    double a, b, c, d;
};
__device__ __forceinline__ Mob mob_mul(const Mob& X, const Mob& Y)
{
    Mob Z{fma(X.a, Y.a, X.b * Y.c), fma(X.a, Y.b, X.b * Y.d), fma(X.c, Y.a, X.d * Y.c),
          fma(X.c, Y.b, X.d * Y.d)};
    const double s = fmax(fmax(fabs(Z.a), fabs(Z.b)), fmax(fabs(Z.c), fabs(Z.d)));
    if (s > 0.0 && isfinite(s)) {
        const int e = ilogb(s);
        Z.a = scalbn(Z.a, -e);
        Z.b = scalbn(Z.b, -e);
        Z.c = scalbn(Z.c, -e);
        Z.d = scalbn(Z.d, -e);
    }
    return Z;
}

template <int BS, int FAM>
__global__ void __launch_bounds__(BS) k_curve_prep(CurveArgs a, const int* item_T,
                                                   const int* item_curve, double* lanec,
                                                   float* lanec32)
{
    constexpr int LMAX = Items<BS>::LMAX, NF = Items<BS>::NF;
    __shared__ double sA[BS], sB[BS], sC[BS], sD[BS];
    BlockChunk b;
    item_chunk<BS>(a, item_T, item_curve, b);
    const int tid = threadIdx.x, lt = b.lt, T = b.T, L = __ffs(T) - 1, m = b.m, base = b.base;
    const bool has = b.cnt > 0;
    const size_t NS = a.n_slots;
    const double h = b.active ? a.h[b.line] : 1.0;
    const double Mo = h / 6.0, Md = 2.0 * h / 3.0, Ko = -1.0 / h, Kd = 2.0 / h;
    const double mw = a.paper ? 0.0 : 1.0, td = a.td;
    const double dd = a.dt - a.td;  // (1 - theta) dt of the FP64 form's right-hand side
    // element rows of node q + 1: mass M and operator S (sub, diag, super)
    auto rowcoef = [&](int q, double* Mr, double* Sr) {
        Mr[0] = Mo;
        Mr[1] = Md;
        Mr[2] = Mo;
        if (FAM == 0) {
            const double b0 = a.bnorm[base + q], b1 = a.bnorm[base + q + 1], b2 = a.bnorm[base + q + 2];
            const double Csub = -(b0 * (1.0 / 6.0) + b1 * (1.0 / 3.0));
            const double Cdia = (b0 - b2) * (1.0 / 6.0);
            const double Csup = b1 * (1.0 / 3.0) + b2 * (1.0 / 6.0);
            Sr[0] = a.mu * Ko + Csub + a.sig * Mo;
            Sr[1] = a.mu * Kd + Cdia + a.sig * Md;
            Sr[2] = a.mu * Ko + Csup + a.sig * Mo;
            if (a.supg) {  // SUPG terms of the two elements of node q + 1
                const double tl = supg_tau(h, 0.5 * (b0 + b1), a.mu);
                const double tr = supg_tau(h, 0.5 * (b1 + b2), a.mu);
                const double mbs = tl * (2.0 * b0 + b1) / 6.0;
                const double mbd = tl * (b0 + 2.0 * b1) / 6.0 - tr * (2.0 * b1 + b2) / 6.0;
                const double mbp = -tr * (b1 + 2.0 * b2) / 6.0;
                const double al = tl * (b0 * b0 + b0 * b1 + b1 * b1) / (3.0 * h);
                const double ar = tr * (b1 * b1 + b1 * b2 + b2 * b2) / (3.0 * h);
                Mr[0] += mbs;
                Mr[1] += mbd;
                Mr[2] += mbp;
                Sr[0] += -al + a.sig * mbs;
                Sr[1] += al + ar + a.sig * mbd;
                Sr[2] += -ar + a.sig * mbp;
            }
        } else {
            Sr[0] = a.mu * Ko;
            Sr[1] = a.mu * Kd;
            Sr[2] = Sr[0];
        }
    };
    // row q of A = mw M + td S (Dirichlet couplings dropped)
    auto sysrow = [&](int q, const double* Mr, const double* Sr, double& A, double& B, double& C) {
        A = (q == 0) ? 0.0 : mw * Mr[0] + td * Sr[0];
        B = mw * Mr[1] + td * Sr[1];
        C = (q == m - 1) ? 0.0 : mw * Mr[2] + td * Sr[2];
    };
    double cpL = 0, vpL = 0, A0 = 0, B0 = 1, Clast = 0;
    Mob P{1.0, 0.0, 0.0, 1.0};  // pivot maps of the chunk's rows after its first
    if (has) {
        double cpp = 0, vpp = 0, Cprev = 0;
        for (int j = 0; j < b.cnt; ++j) {
            const int q = b.s + j;
            const size_t sl = b.so + (size_t)j * T + lt;
            double Mr[3], Sr[3], A, B, C;
            rowcoef(q, Mr, Sr);
            sysrow(q, Mr, Sr, A, B, C);
            double ip, cp, vp, lp;
            if (j == 0) {
                ip = 1.0 / B;
                cp = C * ip;
                vp = A * ip;
                lp = 0.0;
                A0 = A;
                B0 = B;
            } else {
                ip = 1.0 / (B - A * cpp);
                cp = C * ip;
                vp = -A * vpp * ip;
                lp = A * ip;
                P = mob_mul(Mob{B, -A * Cprev, 1.0, 0.0}, P);
            }
            a.fac[sl] = cp;
            a.fac[NS + sl] = vp;
            a.fac[2 * NS + sl] = ip;
            a.fac[3 * NS + sl] = lp;
            // right-hand-side rows times ip: (M - (1 - theta) dt S) in the FP64
            // form, -S in the residual form
            if (FAM == 0) {
                for (int k = 0; k < 3; ++k)
                    a.srow[k * NS + sl] = (a.vform ? Mr[k] - dd * Sr[k] : -Sr[k]) * ip;
            } else {
                a.srow[sl] = (a.vform ? Mr[0] - dd * Sr[0] : -Sr[0]) * ip;
            }
            if (a.fac32) {
                a.fac32[sl] = (float)cp;
                a.fac32[NS + sl] = (float)vp;
                a.fac32[2 * NS + sl] = (float)ip;
                a.fac32[3 * NS + sl] = (float)lp;
            }
            cpp = cp;
            vpp = vp;
            Cprev = C;
        }
        cpL = cpp;
        vpL = vpp;
        Clast = Cprev;
    }
    // G: ratio of the diagonal to the off-diagonal coefficient of the rhs
    // stencil (constant along a curve)
    if (FAM == 1 && b.active && lt == 0 && m > 0) {
        double Mr[3], Sr[3];
        rowcoef(0, Mr, Sr);
        a.kap[b.line] = a.vform ? (Mr[1] - dd * Sr[1]) / (Mr[0] - dd * Sr[0]) : -2.0;
    }
    // fixed part of the upward pass: x_s = rho - kap G_t - nu G_{t-1}
    double kap = has ? -1.0 : 0.0, nu = 0.0;
    for (int j = b.cnt - 2; j >= 0; --j) {
        const size_t sl = b.so + (size_t)j * T + lt;
        double cp = a.fac[sl];
        kap = -cp * kap;
        nu = a.fac[NS + sl] - cp * nu;
    }
    sA[tid] = kap;
    sB[tid] = nu;
    __syncthreads();
    double kapN = lt + 1 < T ? sA[tid + 1] : 0.0;
    double nuN = lt + 1 < T ? sB[tid + 1] : 0.0;
    __syncthreads();
    double A = has ? vpL : 0.0;
    double B = has ? 1.0 - cpL * nuN : 1.0;
    double C = has ? -cpL * kapN : 0.0;
    double* Lc = lanec + (size_t)blockIdx.x * NF * BS;
    Lc[tid] = cpL;
#pragma unroll
    for (int l = 0; l < LMAX; ++l) {
        const int d = 1 << l;
        sA[tid] = A;
        sB[tid] = B;
        sC[tid] = C;
        __syncthreads();
        bool use = l < L;
        bool lo = use && lt >= d, hi = use && lt + d < T;
        double Am = lo ? sA[tid - d] : 0.0, Bm = lo ? sB[tid - d] : 1.0, Cm = lo ? sC[tid - d] : 0.0;
        double Ap = hi ? sA[tid + d] : 0.0, Bp = hi ? sB[tid + d] : 1.0, Cp = hi ? sC[tid + d] : 0.0;
        __syncthreads();
        double k1 = lo ? A / Bm : 0.0, k2 = hi ? C / Bp : 0.0;
        double nA = lo ? -Am * k1 : (use ? 0.0 : A), nC = hi ? -Cp * k2 : (use ? 0.0 : C);
        B = B - (lo ? Cm * k1 : 0.0) - (hi ? Ap * k2 : 0.0);
        A = nA;
        C = nC;
        Lc[(1 + l) * BS + tid] = k1;
        Lc[(1 + LMAX + l) * BS + tid] = k2;
    }
    Lc[(NF - 1) * BS + tid] = 1.0 / B;
    if (lanec32) {
        float* L32 = lanec32 + (size_t)blockIdx.x * NF * BS;
        for (int f = 0; f < NF; ++f) L32[f * BS + tid] = (float)Lc[f * BS + tid];
    }
    if (!a.pivmin) return;  // uniform over the block
    // Thomas pivots of the whole curve (the smallest-pivot diagnostic): the
    // recurrence d_q = B_q - A_q C_{q-1} / d_{q-1} maps (p, r) -> (B_q p -
    // A_q C_{q-1} r, p).  Each thread composes its chunk's maps, a scan over
    // the curve's threads gives every chunk its incoming pivot, and each
    // thread re-runs its rows from it.
    sD[tid] = Clast;
    __syncthreads();
    const double Cin = (lt > 0) ? sD[tid - 1] : 0.0;
    __syncthreads();
    Mob S = has ? mob_mul(P, Mob{B0, -A0 * Cin, 1.0, 0.0}) : Mob{1.0, 0.0, 0.0, 1.0};
    for (int l = 0; l < L; ++l) {  // L is uniform over the block
        const int d = 1 << l;
        sA[tid] = S.a;
        sB[tid] = S.b;
        sC[tid] = S.c;
        sD[tid] = S.d;
        __syncthreads();
        if (lt >= d) S = mob_mul(S, Mob{sA[tid - d], sB[tid - d], sC[tid - d], sD[tid - d]});
        __syncthreads();
    }
    sA[tid] = S.a + S.b;  // state after the thread's rows, from (1, 1)
    sB[tid] = S.c + S.d;
    __syncthreads();
    double dprev = (lt > 0) ? sA[tid - 1] / sB[tid - 1] : 1.0;
    double dmin = INFINITY, Cprev = Cin;
    for (int j = 0; j < b.cnt; ++j) {
        const int q = b.s + j;
        double Mr[3], Sr[3], Aq, Bq, Cq;
        rowcoef(q, Mr, Sr);
        sysrow(q, Mr, Sr, Aq, Bq, Cq);
        const double dq = (q == 0) ? Bq : Bq - Aq * Cprev / dprev;
        dmin = fmin(dmin, fabs(dq));
        dprev = dq;
        Cprev = Cq;
    }
    for (int o = 16; o > 0; o >>= 1) dmin = fmin(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
    if ((tid & 31) == 0 && dmin < INFINITY)
        atomicMin(reinterpret_cast<unsigned long long*>(a.pivmin),
                  (unsigned long long)__double_as_longlong(dmin));
}

// FP64 <-> FP32 conversions on the integer pipe.  On this GPU the FP64 unit
// issues 2 lanes per SM per clock and also executes F2F conversions, so the
// reduced-precision solve converts with bit operations on the IEEE-754 fields.
// toward zero; |x| < 2^-126 gives a signed zero, |x| >= 2^128 an infinity
__device__ __forceinline__ float f64_to_f32(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sgn = hi & 0x80000000u, ah = hi & 0x7fffffffu;
    unsigned f = __funnelshift_r(lo, hi, 29) - (384u << 23);  // exponent bias 1023 -> 127 (mod 2^9)
    if (ah < (897u << 20)) f = 0u;
    else if (ah >= (1151u << 20))
        f = (ah > 0x7ff00000u || (ah == 0x7ff00000u && lo)) ? 0x7fc00000u : 0x7f800000u;
    return __uint_as_float(f | sgn);
}

// exact for normal values; subnormals give a signed zero
__device__ __forceinline__ double f32_to_f64(float x)
{
    const unsigned b = __float_as_uint(x), sgn = b & 0x80000000u, a = b & 0x7fffffffu;
    unsigned hi = sgn | ((a >> 3) + (896u << 20)), lo = b << 29;
    if (a < 0x00800000u) {
        hi = sgn;
        lo = 0u;
    } else if (a >= 0x7f800000u) {
        hi = sgn | 0x7ff00000u | ((a >> 3) & 0x000fffffu);
    }
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float mad(float x, float y, float z) { return __fmaf_rn(x, y, z); }
__device__ __forceinline__ double mad(double x, double y, double z) { return __fma_rn(x, y, z); }

// shared memory of a curve-solve block of BS threads whose longest chunk has
// R rows: the reduction's exchange buffers [2][BS] and the rows' rp values
// [R][BS] (8-byte slots, also in the FP32 elimination)
template <int BS>
__host__ __device__ constexpr size_t solve_smem(int R)
{
    return (size_t)(2 + R) * BS * sizeof(double);
}

template <typename E>
__device__ __forceinline__ float as_f32(E x)
{
    if constexpr (sizeof(E) == 4) return x;
    else return f64_to_f32(x);
}

// Curve solve of one work item (block size T, curves[0 .. BS/T-1], reduced-
// system constants Lc, elimination factors fac in precision E); the whole
// block calls it.  RES = 0: FP64 new-value form, v = x.  RES = 1: residual
// form, the correction x in precision E and v = u + dt x accumulated in FP64
// (u is parked in v between the passes).  The rows' rp values live in
// shared memory [R][BS] between the passes.
template <int BS, int FAM, bool RES, typename E, bool DIR = false>
__device__ __forceinline__ void curve_solve_body(const CurveArgs& a, int Titem, const int* curves,
                                                 const E* __restrict__ Lc, const E* __restrict__ fac,
                                                 unsigned char* smem)
{
    constexpr int LMAX = Items<BS>::LMAX, NF = Items<BS>::NF;
    E (*sR)[BS] = reinterpret_cast<E (*)[BS]>(smem);
    double* __restrict__ buf = reinterpret_cast<double*>(smem + 2 * BS * sizeof(double));
    const int tid = threadIdx.x;
    // row j's 8-byte slot of rp (E)
    auto rp = [&](int j) -> E& { return *reinterpret_cast<E*>(buf + j * BS + tid); };
    const double* __restrict__ u = (a.state && (a.state->iter & 1)) ? a.u_odd : a.u_even;
    double* __restrict__ v = a.v;
    BlockChunk b;
    item_chunk_of(a, Titem, curves, b);
    const int lt = b.lt, T = b.T, L = __ffs(T) - 1;
    if (b.active && b.n < 2 && lt <= b.n) v[b.base + lt] = 0.0;
    const int base = b.base, s = b.s, cnt = b.cnt;
    const size_t NS = a.n_slots;
    const int so = (int)b.so;
    const bool paper = a.paper != 0;
    E rpp = E(0);
    // right-hand side (FP64) of row j from u at its node and the two
    // neighbours, and the row's downward elimination step
    auto row = [&](int j, int sl, double kap, double u0, double u1, double u2) {
        double r;
        if (FAM == 0) {
            r = __ldg(a.Fl + sl);
            if (!paper) {
                r = fma(__ldg(a.srow + sl), u0, r);
                r = fma(__ldg(a.srow + NS + sl), u1, r);
                r = fma(__ldg(a.srow + 2 * NS + sl), u2, r);
            }
        } else {
            r = __ldg(a.srow + sl) * fma(kap, u1, u0 + u2);
        }
        E re;
        if constexpr (sizeof(E) == 4) re = f64_to_f32(r);
        else re = r;
        rpp = mad(-__ldg(fac + 3 * NS + sl), rpp, re);
        rp(j) = rpp;
    };
    if constexpr (DIR) {
        // the state given at the curve's nodes (the direct transfer; 0 at both ends)
        if (cnt > 0) {
            const double kap = (FAM == 1) ? __ldg(a.kap + b.line) : 0.0;
            const double* __restrict__ un = u + base + s;
            double u0 = paper ? 0.0 : __ldg(un), u1 = paper ? 0.0 : __ldg(un + 1);
            for (int j = 0; j < cnt; ++j) {
                const double u2 = paper ? 0.0 : __ldg(un + j + 2);
                row(j, so + j * T + lt, kap, u0, u1, u2);
                u0 = u1;
                u1 = u2;
            }
        }
    } else if (cnt > 0) {
        const double kap = (FAM == 1) ? __ldg(a.kap + b.line) : 0.0;
        auto uslot = [&](int sl) -> double { return gather_w(u, a.nx, __ldg(a.gcell + sl), a.gw, NS, sl); };
        double u0 = 0.0, u1 = 0.0;
        if (!paper) {
            u0 = (s == 0) ? 0.0 : uslot(so + (b.c - 1) * T + (lt - 1));
            u1 = uslot(so + lt);
        }
        // the gather descriptors (cell, corner weights) of the row gathered at
        // iteration j (u at node s+j+2; slot -1: the curve's end, u = 0) are
        // loaded one iteration ahead, so that only the corner loads wait
        auto next_slot = [&](int j) -> int {
            return paper ? -1
                         : (j + 1 < cnt ? so + (j + 1) * T + lt
                                        : (j + 1 == cnt && s + cnt < b.m ? so + lt + 1 : -1));
        };
        int nsl = next_slot(0), ncell = 0;
        double nw0 = 0.0, nw1 = 0.0, nw2 = 0.0, nw3 = 0.0;
        auto load_desc = [&]() {
            ncell = __ldg(a.gcell + nsl);
            nw0 = __ldg(a.gw + nsl);
            nw1 = __ldg(a.gw + NS + nsl);
            nw2 = __ldg(a.gw + 2 * NS + nsl);
            nw3 = __ldg(a.gw + 3 * NS + nsl);
        };
        if (nsl >= 0) load_desc();
        for (int j = 0; j < cnt; ++j) {
            const int sl = so + j * T + lt;
            double u2 = 0.0;
            if (nsl >= 0) {
                const double* r0 = u + ncell;
                u2 = nw0 * __ldg(r0);
                u2 = fma(nw1, __ldg(r0 + 1), u2);
                u2 = fma(nw2, __ldg(r0 + a.nx), u2);
                u2 = fma(nw3, __ldg(r0 + a.nx + 1), u2);
            }
            nsl = next_slot(j + 1);
            if (nsl >= 0) load_desc();
            if constexpr (RES) {
                if (!paper) v[base + s + j + 1] = u1;
            }
            row(j, sl, kap, u0, u1, u2);
            u0 = u1;
            u1 = u2;
        }
    }
    // 3. upward pass over the chunk: rho for its first row
    E rho = E(0);
    for (int j = cnt - 2; j >= 0; --j) rho = mad(-__ldg(fac + so + j * T + lt), rho, rp(j));
    // 4. reduced system of the chunk ends; its factors are loaded a level
    //    ahead, so that each load is in flight while the block waits
    const E lc0 = Lc[tid];
    E k1n = E(0), k2n = E(0), ib = E(0);
    if (L > 0) {
        k1n = Lc[BS + tid];
        k2n = Lc[(1 + LMAX) * BS + tid];
    } else {
        ib = Lc[(NF - 1) * BS + tid];
    }
    sR[0][tid] = rho;
    __syncthreads();
    const E rhoN = lt + 1 < T ? sR[0][tid + 1] : E(0);
    E R = cnt > 0 ? mad(-lc0, rhoN, rpp) : E(0);
    int bsel = 1;
#pragma unroll
    for (int l = 0; l < LMAX; ++l) {
        if (l >= L) break;  // L (levels of this item's curves) is the same for the whole block
        const int d = 1 << l;
        const E k1 = k1n, k2 = k2n;
        if (l + 1 < L) {
            k1n = Lc[(2 + l) * BS + tid];
            k2n = Lc[(2 + LMAX + l) * BS + tid];
        } else {
            ib = Lc[(NF - 1) * BS + tid];
        }
        sR[bsel][tid] = R;
        __syncthreads();
        const E Rm = lt >= d ? sR[bsel][tid - d] : E(0);
        const E Rp = lt + d < T ? sR[bsel][tid + d] : E(0);
        R = mad(-k2, Rp, mad(-k1, Rm, R));
        bsel ^= 1;
    }
    const E G = R * ib;
    sR[bsel][tid] = G;
    __syncthreads();
    const E Gm = lt > 0 ? sR[bsel][tid - 1] : E(0);
    // 5. back substitution; values out
    E x = G;
    float xmax = 0.f;  // residual form: the largest |correction| / dt of the thread's rows
    for (int j = cnt - 1; j >= 0; --j) {
        const int sl = so + j * T + lt;
        if (j < cnt - 1) x = mad(-__ldg(fac + NS + sl), Gm, mad(-__ldg(fac + sl), x, rp(j)));
        const int node = base + s + j + 1;
        if constexpr (RES) {
            double x64;
            if constexpr (sizeof(E) == 4) x64 = f32_to_f64(x);
            else x64 = x;
            // v = u + dt d in FP64 (u parked in v, or the node values themselves)
            const double ub = DIR ? __ldg(u + node) : v[node];
            v[node] = paper ? x64 : fma(a.dt, x64, ub);
            xmax = fmaxf(xmax, fabsf(as_f32(x)));
        } else {
            v[node] = x;
        }
    }
    if (b.active && b.n >= 2 && lt == 0) {
        v[base] = 0.0;
        v[base + b.n] = 0.0;
    }
    if constexpr (RES) {
        // largest correction of the launch (for the solve's statistics)
        if (a.state && !paper) {
            for (int o = 16; o > 0; o >>= 1) xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
            if ((tid & 31) == 0 && xmax > 0.f) {
                const double cmax = a.dt * f32_to_f64(xmax);
                atomicMax(const_cast<unsigned long long*>(&a.state->corr_bits),
                          (unsigned long long)__double_as_longlong(cmax));
            }
        }
    }
}

// one work item of the reduced-precision mode: FP32 corrections until the
// iteration switches to FP64 ones (IterState::hp; a split step outside the
// iteration always solves in FP32)
template <int BS, int FAM>
__device__ __forceinline__ void curve_solve_ref(const CurveArgs& a, int Titem, const int* curves,
                                                const double* lanec, const float* lanec32,
                                                unsigned char* smem)
{
    if (a.state && a.state->hp) curve_solve_body<BS, FAM, true, double>(a, Titem, curves, lanec, a.fac, smem);
    else curve_solve_body<BS, FAM, true, float>(a, Titem, curves, lanec32, a.fac32, smem);
}

// the same from the state at the curve's nodes (the gather pass before it)
template <int BS, int FAM>
__device__ __forceinline__ void curve_solve_ref_dir(const CurveArgs& a, int Titem, const int* curves,
                                                    const double* lanec, const float* lanec32,
                                                    unsigned char* smem)
{
    if (a.state && a.state->hp)
        curve_solve_body<BS, FAM, true, double, true>(a, Titem, curves, lanec, a.fac, smem);
    else curve_solve_body<BS, FAM, true, float, true>(a, Titem, curves, lanec32, a.fac32, smem);
}

// 256-thread blocks are held to 64 registers (4 blocks per SM with their
// shared memory): measured faster than 3 blocks at 74 registers
template <int BS, int FAM, bool REF>
__global__ void __launch_bounds__(BS, BS == 256 ? 4 : (BS == 512 ? 2 : 1)) k_curve_solve(CurveArgs a, const int* item_T,
                                                    const int* item_curve, const double* lanec,
                                                    const float* lanec32)
{
    if (a.state && a.state->done) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = item_T[blockIdx.x];
    const int* cv = item_curve + blockIdx.x * Items<BS>::MAXC;
    const size_t lo = (size_t)blockIdx.x * Items<BS>::NF * BS;
    if constexpr (REF) curve_solve_ref<BS, FAM>(a, T, cv, lanec + lo, lanec32 + lo, smem);
    else curve_solve_body<BS, FAM, false, double>(a, T, cv, lanec + lo, a.fac, smem);
}

// ------------------------------------------------------------ batched problems
// A batch keeps one CurveArgs per (problem, family) in a device table and one
// list of work items over all problems, longest curves first.  The persistent
// kernels below loop over that list with a grid of a few blocks per SM; an
// item whose problem has converged is skipped.
struct BatchItem {
    int prob;     // problem index
    int T;        // block size of the item's curves
    int local;    // item index inside its problem's item set (reduced-system constants)
    int curves[8];
};

// Active work lists of a batch: double-buffered index lists (buffer *sel is
// current) rebuilt by k_batch_compact when a problem converges.
struct ActiveLists {
    int* items[2][2][3];  // [buffer][family][set] indices into the item arrays
    int* blocks[2];       // [buffer] indices into the map block table
    int* count;           // [buffer][2 fam * 3 sets + 1]
    const int* const* blocks_dev;  // device copy of blocks[2] (for the map kernel)
    int* sel;             // current buffer
    int* changed;         // a problem finished in this step
};
constexpr int kCountPerBuf = 7;

// curve solve from the state at the curve's nodes (the direct transfer, or
// after the gather pass): FP64 new values, or (REF) the reduced-precision
// mode's correction added in FP64
template <int BS, int FAM, bool REF = false>
__global__ void __launch_bounds__(BS, BS == 256 ? 4 : (BS == 512 ? 2 : 1)) k_curve_solve_dir(CurveArgs a, const int* item_T,
                                                    const int* item_curve, const double* lanec,
                                                    const float* lanec32)
{
    if (a.state && a.state->done) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t lo = (size_t)blockIdx.x * Items<BS>::NF * BS;
    const int* cv = item_curve + blockIdx.x * Items<BS>::MAXC;
    if constexpr (REF) curve_solve_ref_dir<BS, FAM>(a, item_T[blockIdx.x], cv, lanec + lo, lanec32 + lo, smem);
    else curve_solve_body<BS, FAM, false, double, true>(a, item_T[blockIdx.x], cv, lanec + lo, a.fac, smem);
}

// DIR: the table's u pointers are the families' node values (the batched
// gather pass before the solve fills them)
template <int BS, int FAM, bool REF, bool DIR = false>
__global__ void __launch_bounds__(BS) k_curve_solve_batch(const CurveArgs* __restrict__ table,
                                                          const BatchItem* __restrict__ items,
                                                          ActiveLists act, int set)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int cur = *act.sel;
    const int* list = act.items[cur][FAM][set];
    const int n_act = act.count[cur * kCountPerBuf + FAM * 3 + set];
    for (int ii = blockIdx.x; ii < n_act; ii += gridDim.x) {
        const BatchItem& I = items[list[ii]];
        const CurveArgs& a = table[2 * I.prob + FAM];
        if (a.state->done) continue;  // uniform: one problem per item
        const size_t lo = (size_t)I.local * Items<BS>::NF * BS;
        if constexpr (REF && DIR)
            curve_solve_ref_dir<BS, FAM>(a, I.T, I.curves, a.lanecs[set] + lo, a.lanec32s[set] + lo, smem);
        else if constexpr (REF)
            curve_solve_ref<BS, FAM>(a, I.T, I.curves, a.lanecs[set] + lo, a.lanec32s[set] + lo, smem);
        else
            curve_solve_body<BS, FAM, false, double, DIR>(a, I.T, I.curves, a.lanecs[set] + lo, a.fac, smem);
        __syncthreads();  // shared memory is reused by the next item
    }
}

struct GridArgs {
    int nx, ny;
    const uint8_t* ntype;
    const int* mg;     // [4 N] first node of each crossed segment (boundary: 0 with zero weights)
    const double* mc;  // [8 N] weights of v[g], v[g+1] for the 4 crossings
    const double* v;
    double* out_even;  // written buffer by parity of the step counter (or fixed)
    double* out_odd;
    const double* prev_even;  // previous state for the norms (nullable)
    const double* prev_odd;
    const IterState* state;
    int parity_shift;  // output buffer = parity(iter + shift)
    double* partial;   // [2 * gridDim.x] sums of (u - u_prev)^2 and u^2
};

// block sum of (dd, uu) into dst[0..1]
__device__ __forceinline__ void block_sum2(double dd, double uu, double* dst)
{
    __shared__ double sd[kGridThreads / 32], su[kGridThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        dd += __shfl_down_sync(0xffffffffu, dd, o);
        uu += __shfl_down_sync(0xffffffffu, uu, o);
    }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sd[w] = dd;
        su[w] = uu;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double td = 0, tu = 0;
        for (int q = 0; q < kGridThreads / 32; ++q) {
            td += sd[q];
            tu += su[q];
        }
        dst[0] = td;
        dst[1] = tu;
    }
}

// ---------------------------------------------- direct transfer (per step)
// values at the nodes of the target family from the source family's curve
// values through the crossing tables: value = c0 v[g0] + c1 v[g0 + 1] +
// c2 v[g1] + c3 v[g1 + 1] (end nodes have zero coefficients); with NORMS the
// partial sums of |u - u_prev|^2 and |u|^2 for the convergence test
struct XferArgs {
    long long n;              // target nodes
    const int* xg;            // [2 n]
    const double* xc;         // [4 n]
    const double* v;          // source curve values
    double* out_even;         // output by parity of (iter + parity_shift)
    double* out_odd;
    const double* prev_even;  // previous state by parity of iter (NORMS)
    const double* prev_odd;
    const IterState* state;
    int parity_shift;
    double* partial;
};

template <bool NORMS>
__global__ void __launch_bounds__(kGridThreads) k_curve_xfer(XferArgs a)
{
    if (a.state && a.state->done) return;
    const int it = a.state ? a.state->iter : 0;
    double* __restrict__ out = ((it + a.parity_shift) & 1) ? a.out_odd : a.out_even;
    const double* __restrict__ prev = (it & 1) ? a.prev_odd : a.prev_even;
    const double* __restrict__ v = a.v;
    double dd = 0.0, uu = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < a.n;
         k += (long long)gridDim.x * blockDim.x) {
        const int2 g = *reinterpret_cast<const int2*>(a.xg + 2 * k);
        const double2 c0 = *reinterpret_cast<const double2*>(a.xc + 4 * k);
        const double2 c1 = *reinterpret_cast<const double2*>(a.xc + 4 * k + 2);
        double val = c0.x * __ldg(v + g.x);
        val = fma(c0.y, __ldg(v + g.x + 1), val);
        val = fma(c1.x, __ldg(v + g.y), val);
        val = fma(c1.y, __ldg(v + g.y + 1), val);
        out[k] = val;
        if (NORMS) {
            const double dl = val - prev[k];
            dd = fma(dl, dl, dd);
            uu = fma(val, val, uu);
        }
    }
    if (NORMS) block_sum2(dd, uu, a.partial + 2 * blockIdx.x);
}

// the grid state at every node of a family (bilinear, §6.1), 0 at both ends
// of every curve: one warp per curve
__global__ void k_gather_nodes(int nx, int ny, int n_lines, const int* off, const double* xi,
                               const double* eta, const double* u, double* out)
{
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (l >= n_lines) return;
    const int a0 = off[l], a1 = off[l + 1] - 1;
    for (int k = a0 + lane; k <= a1; k += 32) {
        if (k == a0 || k == a1) {
            out[k] = 0.0;
            continue;
        }
        const double x = xi[k], y = eta[k];
        int i = (int)floor(x), r = (int)floor(y);
        i = i > nx - 2 ? nx - 2 : (i < 0 ? 0 : i);
        r = r > ny - 2 ? ny - 2 : (r < 0 ? 0 : r);
        out[k] = gather_at(u, nx, r * nx + i, x - i, y - r);
    }
}

// midpoint (u_j + u_{j+1/2}) / 2 at the B nodes, u_j the state the last step
// started from (by its parity)
__global__ void k_node_midpoint(const IterState* st, const double* u_even, const double* u_odd,
                                const double* vb, double* out, long long n)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int it = st ? st->iter : 1;
    const double* uj = ((it - 1) & 1) ? u_odd : u_even;
    out[k] = 0.5 * (uj[k] + vb[k]);
}

// combined weights of the curve -> grid map (setup): the row value
// (1-w) vL + w vR and the column value, each crossing v = (1-t) v[g] + t v[g+1],
// averaged, written as 8 products with the curve values
// (weights mode 1: the row value weighted by the column gap and the column
// value by the row gap instead of 1/2 each)
__global__ void k_map_coef(long long N, const uint8_t* ntype, const int* cg, const double* ct,
                           const double* cw, const double* cpos, int weights, int* mg, double* mc)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= N) return;
    double ar = 0.5, ac = 0.5;
    if (weights) {
        double gr = cpos[4 * k + 1] - cpos[4 * k], gc = cpos[4 * k + 3] - cpos[4 * k + 2];
        if (gr + gc > 0.0) {
            ar = gc / (gr + gc);
            ac = gr / (gr + gc);
        }
    }
    for (int q = 0; q < 4; ++q) {
        int g = cg[4 * k + q];
        double t = ct[4 * k + q];
        double w = cw[2 * k + (q >> 1)];
        double side = ((q & 1) ? w : 1.0 - w) * (q < 2 ? ar : ac);
        bool ok = ntype[k] == kInterior && g >= 0;
        mg[4 * k + q] = ok ? g : 0;
        mc[8 * k + 2 * q] = ok ? side * (1.0 - t) : 0.0;
        mc[8 * k + 2 * q + 1] = ok ? side * t : 0.0;
    }
}

// curve -> grid map over nodes first, first + stride, ... of one problem;
// returns the partial sums of the norms of the calling thread
template <bool NORMS>
__device__ __forceinline__ void grid_map_body(const GridArgs& a, long long first, long long stride,
                                              double& dd, double& uu)
{
    int it = a.state ? a.state->iter : 0;
    double* __restrict__ out = ((it + a.parity_shift) & 1) ? a.out_odd : a.out_even;
    const double* __restrict__ prev = (it & 1) ? a.prev_odd : a.prev_even;
    const double* __restrict__ v = a.v;
    const long long N = (long long)a.nx * a.ny;
    for (long long k = first; k < N; k += stride) {
        double val = 0.0;
        if (a.ntype[k] == kInterior) {
            int4 g = *reinterpret_cast<const int4*>(a.mg + 4 * k);
            const double2* c = reinterpret_cast<const double2*>(a.mc + 8 * k);
            double2 c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
            val = c0.x * __ldg(v + g.x);
            val = fma(c0.y, __ldg(v + g.x + 1), val);
            val = fma(c1.x, __ldg(v + g.y), val);
            val = fma(c1.y, __ldg(v + g.y + 1), val);
            val = fma(c2.x, __ldg(v + g.z), val);
            val = fma(c2.y, __ldg(v + g.z + 1), val);
            val = fma(c3.x, __ldg(v + g.w), val);
            val = fma(c3.y, __ldg(v + g.w + 1), val);
            if (NORMS) {
                double dlt = val - prev[k];
                dd = fma(dlt, dlt, dd);
                uu = fma(val, val, uu);
            }
        }
        out[k] = val;
    }
}

template <bool NORMS>
__global__ void __launch_bounds__(kGridThreads) k_grid_map(GridArgs a)
{
    if (a.state && a.state->done) return;
    double dd = 0.0, uu = 0.0;
    grid_map_body<NORMS>(a, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                         (long long)gridDim.x * blockDim.x, dd, uu);
    if (NORMS) block_sum2(dd, uu, a.partial + 2 * blockIdx.x);
}

// batched map: block b works for problem blk_prob[b] as its local block
// blk_local[b] of nblk[p] (table entries 2p + fam); partial sums per local block
template <bool NORMS>
__global__ void __launch_bounds__(kGridThreads) k_grid_map_batch(const GridArgs* __restrict__ table,
                                                                int fam, const int* blk_prob,
                                                                const int* blk_local, const int* nblk,
                                                                const int* const* act_blocks,
                                                                const int* act_count, const int* sel)
{
    const int cur = *sel;
    const int* list = act_blocks[cur];
    const int n_act = act_count[cur * 7 + 6];
    for (int ii = blockIdx.x; ii < n_act; ii += gridDim.x) {
        int bk = list[ii];
        int p = blk_prob[bk], lb = blk_local[bk];
        const GridArgs& a = table[2 * p + fam];
        if (a.state->done) continue;  // uniform per block
        double dd = 0.0, uu = 0.0;
        grid_map_body<NORMS>(a, (long long)lb * blockDim.x + threadIdx.x,
                             (long long)nblk[p] * blockDim.x, dd, uu);
        if (NORMS) block_sum2(dd, uu, a.partial + 2 * lb);
        __syncthreads();  // block_sum2's shared arrays are reused
    }
}

// batched gather pass: the grid state at the nodes of one family of every
// active problem, over the batch's map blocks (problem, local block)
struct GatherArgs {
    long long n;         // curve nodes of the family
    const int* ncell;
    const double* nw;
    int nx;
    const double* u_even;
    const double* u_odd;
    const IterState* state;
    double* out;
};

__global__ void __launch_bounds__(256) k_gather_batch(const GatherArgs* __restrict__ table, int fam,
                                                      const int* blk_prob, const int* blk_local,
                                                      const int* nblk, const int* const* act_blocks,
                                                      const int* act_count, const int* sel)
{
    const int cur = *sel;
    const int* list = act_blocks[cur];
    const int n_act = act_count[cur * 7 + 6];
    for (int ii = blockIdx.x; ii < n_act; ii += gridDim.x) {
        const int bk = list[ii], pr = blk_prob[bk], lb = blk_local[bk];
        const GatherArgs& g = table[2 * pr + fam];
        if (g.state->done) continue;
        const double* __restrict__ u = (g.state->iter & 1) ? g.u_odd : g.u_even;
        const long long stride = (long long)nblk[pr] * blockDim.x;
        for (long long k = (long long)lb * blockDim.x + threadIdx.x; k < g.n; k += stride) {
            const int c = __ldg(g.ncell + k);
            double v = 0.0;
            if (c >= 0) {
                const double2 wa = *reinterpret_cast<const double2*>(g.nw + 4 * k);
                const double2 wb = *reinterpret_cast<const double2*>(g.nw + 4 * k + 2);
                const double* r0 = u + c;
                const double p11 = __ldg(r0), p12 = __ldg(r0 + 1), p21 = __ldg(r0 + g.nx),
                             p22 = __ldg(r0 + g.nx + 1);
                v = wa.x * p11;
                v = fma(wa.y, p12, v);
                v = fma(wb.x, p21, v);
                v = fma(wb.y, p22, v);
            }
            g.out[k] = v;
        }
    }
}

// rebuild the active lists into the other buffer when a problem finished
__global__ void k_batch_compact(ActiveLists act, const BatchItem* const* items, const int* n_items,
                                const int* blk_prob, int n_blk, IterState* const* states)
{
    if (!*act.changed) return;
    const int cur = *act.sel, nxt = cur ^ 1;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (int fam = 0; fam < 2; ++fam)
        for (int k = 0; k < 3; ++k) {
            const int* list = act.items[cur][fam][k];
            int n = act.count[cur * kCountPerBuf + fam * 3 + k];
            for (long long i = t; i < n; i += stride) {
                int idx = list[i];
                if (!states[items[fam * 3 + k][idx].prob]->done) {
                    int pos = atomicAdd(&act.count[nxt * kCountPerBuf + fam * 3 + k], 1);
                    act.items[nxt][fam][k][pos] = idx;
                }
            }
        }
    const int* bl = act.blocks[cur];
    int nb = act.count[cur * kCountPerBuf + 6];
    for (long long i = t; i < nb; i += stride) {
        int bk = bl[i];
        if (!states[blk_prob[bk]]->done) {
            int pos = atomicAdd(&act.count[nxt * kCountPerBuf + 6], 1);
            act.blocks[nxt][pos] = bk;
        }
    }
}

// make the rebuilt lists current and clear the other buffer's counters
__global__ void k_batch_flip(ActiveLists act)
{
    if (!*act.changed) return;
    int nxt = *act.sel ^ 1;
    for (int q = 0; q < kCountPerBuf; ++q) act.count[(nxt ^ 1) * kCountPerBuf + q] = 0;
    *act.sel = nxt;
    *act.changed = 0;
}

// all problems active: identity lists in buffer 0
__global__ void k_batch_reset(ActiveLists act, const int* n_items, int n_blk)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (int fam = 0; fam < 2; ++fam)
        for (int k = 0; k < 3; ++k)
            for (long long i = t; i < n_items[fam * 3 + k]; i += stride) act.items[0][fam][k][i] = (int)i;
    for (long long i = t; i < n_blk; i += stride) act.blocks[0][i] = (int)i;
    if (t == 0) {
        for (int fam = 0; fam < 2; ++fam)
            for (int k = 0; k < 3; ++k) {
                act.count[fam * 3 + k] = n_items[fam * 3 + k];
                act.count[kCountPerBuf + fam * 3 + k] = 0;
            }
        act.count[6] = n_blk;
        act.count[kCountPerBuf + 6] = 0;
        *act.sel = 0;
        *act.changed = 0;
    }
}

// batched convergence test: block p reduces problem p's partial sums; the last
// block to finish clears the graph condition when every problem is done
__global__ void k_check_batch(IterState* const* states, const double* const* partials,
                              const int* nblk, int n_prob, const double* tols, const int* max_iters,
                              unsigned int* ticket, cudaGraphConditionalHandle handle, int* changed)
{
    int p = blockIdx.x;
    IterState* st = states[p];
    const double tol = tols[p];
    const int max_iter = max_iters[p];
    __shared__ double sd[256], su[256];
    __shared__ bool last;
    if (!st->done) {
        const double* part = partials[p];
        double d = 0, u = 0;
        for (int q = threadIdx.x; q < nblk[p]; q += blockDim.x) {
            d += part[2 * q];
            u += part[2 * q + 1];
        }
        sd[threadIdx.x] = d;
        su[threadIdx.x] = u;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) {
                sd[threadIdx.x] += sd[threadIdx.x + w];
                su[threadIdx.x] += su[threadIdx.x + w];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double num = sd[0], den = su[0];
            double rel = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
            if (!isfinite(num) || !isfinite(den)) rel = INFINITY;  // diverged
            int iter = st->iter + 1;
            int conv = tol > 0.0 && rel <= tol;
            st->iter = iter;
            st->rel = rel;
            st->converged = conv;
            st->done = (conv || iter >= max_iter || !isfinite(rel)) ? 1 : 0;
            st->corr = __longlong_as_double((long long)st->corr_bits);
            st->corr_bits = 0ull;
            if (!st->hp) {
                st->fp32_steps += 1;
                if (tol > 0.0 && rel <= kHpSwitch * tol) st->hp = 1;
            }
            if (st->done) *changed = 1;
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        last = t == (unsigned int)(n_prob - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        int active = 0;
        for (int q = 0; q < n_prob; ++q) active |= !((volatile IterState*)states[q])->done;
        *ticket = 0u;
        cudaGraphSetConditional(handle, active ? 1 : 0);
    }
}

__global__ void k_check(IterState* st, const double* partial, int nblocks, double tol,
                        int max_iter, cudaGraphConditionalHandle handle, int use_cond)
{
    if (st->done) {
        if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(handle, 0);
        return;
    }
    __shared__ double sd[256], su[256];
    double d = 0, u = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        d += partial[2 * b];
        u += partial[2 * b + 1];
    }
    sd[threadIdx.x] = d;
    su[threadIdx.x] = u;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sd[threadIdx.x] += sd[threadIdx.x + s];
            su[threadIdx.x] += su[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double num = sd[0], den = su[0];
        double rel = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
        if (!isfinite(num) || !isfinite(den)) rel = INFINITY;  // diverged
        int iter = st->iter + 1;
        int conv = tol > 0.0 && rel <= tol;
        st->iter = iter;
        st->rel = rel;
        st->converged = conv;
        st->done = (conv || iter >= max_iter || !isfinite(rel)) ? 1 : 0;
        st->corr = __longlong_as_double((long long)st->corr_bits);  // this step's largest correction
        st->corr_bits = 0ull;
        if (!st->hp) {
            st->fp32_steps += 1;
            if (tol > 0.0 && rel <= kHpSwitch * tol) st->hp = 1;
        }
        if (use_cond) cudaGraphSetConditional(handle, st->done ? 0 : 1);
    }
}

// out = wa*a + wb*b on every node, where a = u_j and b = u_{j+1/2} of the last
// step (selected by the step counter); used for the Crank-Nicolson midpoint
__global__ void k_finish(const IterState* st, const double* u_even, const double* u_odd,
                         const double* u_half, double* out, double* iter_out, long long N,
                         int midpoint)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= N) return;
    int it = st->iter;
    const double* uj = ((it - 1) & 1) ? u_odd : u_even;   // u_j of the last step
    const double* un = (it & 1) ? u_odd : u_even;         // u_{j+1}
    if (it == 0) {
        out[k] = u_even[k];
        if (iter_out) iter_out[k] = u_even[k];
        return;
    }
    out[k] = midpoint ? 0.5 * (uj[k] + u_half[k]) : un[k];
    if (iter_out) iter_out[k] = un[k];
}

__global__ void k_mask_copy(const uint8_t* ntype, const double* in, double* out, long long N)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= N) return;
    out[k] = (in && ntype[k] == kInterior) ? in[k] : 0.0;
}

__global__ void k_reset(IterState* st)
{
    st->iter = 0;
    st->done = 0;
    st->converged = 0;
    st->rel = INFINITY;
    st->corr_bits = 0ull;
    st->corr = 0.0;
    st->hp = 0;
    st->fp32_steps = 0;
}

__global__ void k_set_bits(double* p, unsigned long long bits)
{
    *reinterpret_cast<unsigned long long*>(p) = bits;
}

}  // namespace

static CurveArgs curve_args(Problem* p, int fam)
{
    Family& F = p->fam[fam];
    CurveArgs a{};
    a.nx = p->grid.nx;
    a.ny = p->grid.ny;
    a.off = F.off;
    a.soff = F.soff;
    a.h = F.h;
    a.gcell = F.gcell;
    a.gw = F.gw;
    a.ncell = F.ncell;
    a.nw = F.nw;
    a.bnorm = F.bnorm;
    a.fval = F.fval;
    a.xi = F.xi;
    a.eta = F.eta;
    a.Fl = F.Fl;
    a.srow = F.srow;
    a.kap = F.kap;
    a.fac = F.fac;
    a.fac32 = F.fac32;
    a.v = F.v;
    a.n_slots = F.n_slots;
    a.R = F.cmax;
    a.mu = p->mu;
    a.supg = p->opts.stabilize;
    // the factorisation the family holds (prepare_family)
    a.td = F.prep_td;
    a.dt = F.prep_dt;
    a.sig = F.prep_sig;
    a.paper = F.prep_paper;
    a.vform = F.prep_vform;
    a.fscale = F.prep_vform ? F.prep_dt : 1.0;
    return a;
}

// split the curves of a family into work items, assign slots and build the
// gather descriptors (host orchestration, at setup).  A curve of m unknowns
// gets the smallest block size T >= 32 (power of two) with T * R >= m, R the
// preferred rows per thread, at most 1024 (the longest curves then take up to
// kCmax rows per thread); items of BS = 256 threads hold 256/T curves of one
// T, curves with T = 512 or 1024 get items of that size.  Items are ordered
// longest curves first.
adr_status setup_groups(Problem* p, int fam, const std::vector<int>& off)
{
    Family& F = p->fam[fam];
    std::vector<int> order(F.n_lines), Tof(F.n_lines);
    ADR_CUDA_TRY(cudaMemcpyAsync(order.data(), F.order, sizeof(int) * F.n_lines, cudaMemcpyDeviceToHost,
                                 p->stream));
    ADR_CUDA_TRY(cudaStreamSynchronize(p->stream));
    std::vector<int> byT[11];  // index log2(T)
    for (int l : order) {
        int m = off[l + 1] - off[l] - 2;
        int T = 32, lg = 5;
        const int R = (p->rows_per_thread >= 1 && p->rows_per_thread <= kCmax) ? p->rows_per_thread : kCmax;
        while (T < 1024 && (long long)T * R < m) {
            T *= 2;
            lg++;
        }
        if ((long long)T * kCmax < m) {
            set_error("a curve has more than 16384 unknowns");
            return ADR_EINVAL;
        }
        byT[lg].push_back(l);
        Tof[l] = T;
    }
    std::vector<int> soff(F.n_lines + 1, 0);
    long long tot = 0;
    F.cmax = 1;
    for (int l = 0; l < F.n_lines; ++l) {
        soff[l] = (int)tot;
        int m = off[l + 1] - off[l] - 2;
        if (m > 0) tot += (long long)Tof[l] * ((m + Tof[l] - 1) / Tof[l]);
        if (m > 0) F.cmax = std::max(F.cmax, (m + Tof[l] - 1) / Tof[l]);
        if (tot > 0x7fffffffLL) {
            set_error("too many curve rows");
            return ADR_EINVAL;
        }
    }
    soff[F.n_lines] = (int)tot;
    F.n_slots = (int)tot + 1;
    size_t NS = F.n_slots;
    TRY_S(dev_alloc(p, &F.soff, F.n_lines + 1));
    // buffers from the stream-ordered pool are written in the stream's order
    ADR_CUDA_TRY(cudaMemcpyAsync(F.soff, soff.data(), sizeof(int) * soff.size(), cudaMemcpyHostToDevice,
                                 p->stream));
    TRY_S(dev_alloc(p, &F.gcell, NS));
    TRY_S(dev_alloc(p, &F.gw, 4 * NS));
    if (!p->opts.transfer) {
        // node-order gather descriptors and node values of the separate gather pass
        const size_t nn = (size_t)F.n_nodes + 1;
        TRY_S(dev_alloc(p, &F.ncell, nn));
        TRY_S(dev_alloc(p, &F.nw, 4 * nn));
        TRY_S(dev_alloc(p, &F.ug, nn));
        ADR_CUDA_TRY(cudaMemsetAsync(F.ncell, 0xff, sizeof(int) * nn, p->stream));  // -1: curve ends
    }
    TRY_S(dev_alloc(p, &F.fac, 4 * NS));
    if (p->opts.prec == ADR_FP32_REFINE) TRY_S(dev_alloc(p, &F.fac32, 4 * NS));
    if (fam == 0) {
        TRY_S(dev_alloc(p, &F.Fl, NS));
        TRY_S(dev_alloc(p, &F.srow, 3 * NS));
    } else {
        TRY_S(dev_alloc(p, &F.srow, NS));
        TRY_S(dev_alloc(p, &F.kap, (size_t)F.n_lines + 1));
    }
    F.prep_valid = false;
    F.load_plain = false;
    CurveArgs a = curve_args(p, fam);
    cudaStream_t st = p->stream;
    for (int k = 0; k < kItemSets; ++k) {
        const int BS = 256 << k, maxc = BS / 32, nf = 2 * (8 + k) + 2;
        std::vector<int> iT, icv;
        for (int lg = 8 + k; lg >= (k == 0 ? 5 : 8 + k); --lg) {
            const std::vector<int>& L = byT[lg];
            int T = 1 << lg, per = BS / T;
            for (size_t q = 0; q < L.size(); q += per) {
                iT.push_back(T);
                for (int r = 0; r < maxc; ++r)
                    icv.push_back((r < per && q + r < L.size()) ? L[q + r] : -1);
            }
        }
        ItemSet& I = F.iset[k];
        I.BS = BS;
        I.count = (int)iT.size();
        if (I.count == 0) continue;
        TRY_S(dev_alloc(p, &I.T, I.count));
        TRY_S(dev_alloc(p, &I.curve, (size_t)I.count * maxc));
        TRY_S(dev_alloc(p, &I.lanec, (size_t)I.count * nf * BS));
        if (p->opts.prec == ADR_FP32_REFINE) TRY_S(dev_alloc(p, &I.lanec32, (size_t)I.count * nf * BS));
        ADR_CUDA_TRY(cudaMemcpyAsync(I.T, iT.data(), sizeof(int) * iT.size(), cudaMemcpyHostToDevice,
                                     p->stream));
        ADR_CUDA_TRY(cudaMemcpyAsync(I.curve, icv.data(), sizeof(int) * icv.size(), cudaMemcpyHostToDevice,
                                     p->stream));
        if (BS == 256) k_curve_gdesc<256><<<I.count, 256, 0, st>>>(a, I.T, I.curve);
        else if (BS == 512) k_curve_gdesc<512><<<I.count, 512, 0, st>>>(a, I.T, I.curve);
        else k_curve_gdesc<1024><<<I.count, 1024, 0, st>>>(a, I.T, I.curve);
    }
    ADR_CUDA_TRY(cudaGetLastError());
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    return ADR_OK;
}

static void free_alt(Problem* p, Family& F);

void release_groups(Problem* p, int fam)
{
    Family& F = p->fam[fam];
    if (F.alt.allocated) free_alt(p, F);
    void* bufs[] = {F.soff, F.gcell, F.gw, F.fac, F.fac32, F.Fl, F.srow, F.kap, F.ncell, F.nw, F.ug};
    for (void* q : bufs) dev_free(p, q);
    F.ncell = nullptr;
    F.nw = nullptr;
    F.ug = nullptr;
    F.kap = nullptr;
    F.soff = nullptr;
    F.gcell = nullptr;
    F.gw = nullptr;
    F.fac = nullptr;
    F.fac32 = nullptr;
    F.Fl = nullptr;
    F.srow = nullptr;
    for (int k = 0; k < kItemSets; ++k) {
        ItemSet& I = F.iset[k];
        dev_free(p, I.T);
        dev_free(p, I.curve);
        dev_free(p, I.lanec);
        dev_free(p, I.lanec32);
        I = ItemSet();
    }
    F.prep_valid = false;
    F.load_plain = false;
}

// exchange family 0's active factorisation with the one it keeps aside
static void swap_fac(Family& F)
{
    FacState& A = F.alt;
    std::swap(F.fac, A.fac);
    std::swap(F.fac32, A.fac32);
    std::swap(F.srow, A.srow);
    std::swap(F.Fl, A.Fl);
    for (int k = 0; k < kItemSets; ++k) {
        std::swap(F.iset[k].lanec, A.lanec[k]);
        std::swap(F.iset[k].lanec32, A.lanec32[k]);
    }
    std::swap(F.prep_valid, A.valid);
    std::swap(F.prep_td, A.td);
    std::swap(F.prep_dt, A.dt);
    std::swap(F.prep_sig, A.sig);
    std::swap(F.prep_paper, A.paper);
    std::swap(F.prep_vform, A.vform);
    std::swap(F.load_plain, A.load_plain);
}

// buffers for family 0's second factorisation (kind = paper), sized as the first
static adr_status alloc_alt(Problem* p, int paper)
{
    Family& F = p->fam[0];
    FacState& A = F.alt;
    const size_t NS = F.n_slots;
    const bool ref = p->opts.prec == ADR_FP32_REFINE;
    TRY_S(dev_alloc(p, &A.fac, 4 * NS));
    if (ref) TRY_S(dev_alloc(p, &A.fac32, 4 * NS));
    TRY_S(dev_alloc(p, &A.srow, 3 * NS));
    TRY_S(dev_alloc(p, &A.Fl, NS));
    for (int k = 0; k < kItemSets; ++k) {
        const ItemSet& I = F.iset[k];
        if (!I.count) continue;
        const size_t nf = 2 * (8 + k) + 2;
        TRY_S(dev_alloc(p, &A.lanec[k], (size_t)I.count * nf * I.BS));
        if (ref) TRY_S(dev_alloc(p, &A.lanec32[k], (size_t)I.count * nf * I.BS));
    }
    A.allocated = true;
    A.valid = false;
    A.paper = paper;
    A.load_plain = false;
    return ADR_OK;
}

static void free_alt(Problem* p, Family& F)
{
    FacState& A = F.alt;
    void* bufs[] = {A.fac, A.fac32, A.srow, A.Fl};
    for (void* q : bufs) dev_free(p, q);
    for (int k = 0; k < kItemSets; ++k) {
        dev_free(p, A.lanec[k]);
        dev_free(p, A.lanec32[k]);
    }
    A = FacState();
}

adr_status ensure_iteration_active(Problem* p)
{
    Family& F = p->fam[0];
    if (!F.prep_paper) return ADR_OK;
    if (!F.alt.allocated) TRY_S(alloc_alt(p, 0));
    swap_fac(F);
    return ADR_OK;
}

// Factor the family's curve systems for (theta dt, dt, sigma) or the steady
// start (paper), and record the smallest Thomas pivot of the family.  Family
// 0 keeps both kinds once both were asked for (see FacState).
adr_status prepare_family(Problem* p, int fam, double td, double dt, double sig, int paper)
{
    Family& F = p->fam[fam];
    if (fam == 0 && F.prep_paper != paper) {
        if (!F.alt.allocated) TRY_S(alloc_alt(p, paper));
        swap_fac(F);  // the kept factorisation is the kind asked for
    }
    const int vform = (p->opts.prec == ADR_FP64 && !paper) ? 1 : 0;
    if (F.prep_valid && F.prep_td == td && F.prep_dt == dt && F.prep_sig == sig &&
        F.prep_paper == paper)
        return ADR_OK;
    F.prep_td = td;
    F.prep_dt = dt;
    F.prep_sig = sig;
    F.prep_paper = paper;
    F.prep_vform = vform;
    CurveArgs a = curve_args(p, fam);
    cudaStream_t st = p->stream;
    if (!paper) {
        // the smallest pivot is the iteration's systems' (the steady start's is not scanned)
        a.pivmin = p->pivmin + fam;
        k_set_bits<<<1, 1, 0, st>>>(a.pivmin, 0x7ff0000000000000ull);  // +inf: no pivot yet
    }
#define ADR_PREP(BS_, I_)                                                                          \
    if (I_.count) {                                                                                \
        if (fam == 0)                                                                              \
            k_curve_prep<BS_, 0><<<I_.count, BS_, 0, st>>>(a, I_.T, I_.curve, I_.lanec, I_.lanec32); \
        else                                                                                       \
            k_curve_prep<BS_, 1><<<I_.count, BS_, 0, st>>>(a, I_.T, I_.curve, I_.lanec, I_.lanec32); \
    }
    ADR_PREP(256, F.iset[0])
    ADR_PREP(512, F.iset[1])
    ADR_PREP(1024, F.iset[2])
#undef ADR_PREP
    ADR_CUDA_TRY(cudaGetLastError());
    F.prep_valid = true;
    if (fam == 0) F.load_plain = false;  // the load carries the row factors
    return ADR_OK;
}

adr_status load_family(Problem* p, const double* fextra, double fx_scale)
{
    Family& F = p->fam[0];
    if (!fextra && F.load_plain) return ADR_OK;
    CurveArgs a = curve_args(p, 0);
    a.fextra = fextra;
    a.fx_scale = fx_scale;
    cudaStream_t st = p->stream;
    const ItemSet &I0 = F.iset[0], &I1 = F.iset[1], &I2 = F.iset[2];
    if (I0.count) k_curve_load<256><<<I0.count, 256, 0, st>>>(a, I0.T, I0.curve);
    if (I1.count) k_curve_load<512><<<I1.count, 512, 0, st>>>(a, I1.T, I1.curve);
    if (I2.count) k_curve_load<1024><<<I2.count, 1024, 0, st>>>(a, I2.T, I2.curve);
    ADR_CUDA_TRY(cudaGetLastError());
    F.load_plain = fextra == nullptr;
    return ADR_OK;
}

// the curve-solve kernels may use more than 48 KB of dynamic shared memory
template <int BS, int FAM, bool REF>
static cudaError_t solve_attr()
{
    const int bytes = (int)solve_smem<BS>(kCmax);
    cudaError_t e = cudaFuncSetAttribute(k_curve_solve<BS, FAM, REF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_curve_solve_batch<BS, FAM, REF>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_curve_solve_batch<BS, FAM, REF, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_curve_solve_dir<BS, FAM, REF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    return e;
}

static adr_status ensure_solve_attrs()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    ADR_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return ADR_OK;
    cudaError_t e = cudaSuccess;
    cudaError_t r[] = {solve_attr<256, 0, false>(), solve_attr<256, 1, false>(), solve_attr<512, 0, false>(),
                       solve_attr<512, 1, false>(), solve_attr<1024, 0, false>(), solve_attr<1024, 1, false>(),
                       solve_attr<256, 0, true>(),  solve_attr<256, 1, true>(),  solve_attr<512, 0, true>(),
                       solve_attr<512, 1, true>(),  solve_attr<1024, 0, true>(), solve_attr<1024, 1, true>()};
    for (cudaError_t q : r)
        if (q != cudaSuccess) e = q;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute (curve solve shared memory)");
    if (dev >= 0 && dev < 64) done[dev] = true;
    return ADR_OK;
}

adr_status launch_line_solve(Problem* p, int fam, double dt, const double* u_even,
                             const double* u_odd, bool use_state, int paper)
{
    Family& F = p->fam[fam];
    if (!F.prep_valid || F.prep_paper != paper || (!paper && F.prep_dt != dt)) {
        set_error("internal: curve systems not factored for this step");
        return ADR_EINVAL;
    }
    TRY_S(ensure_solve_attrs());
    CurveArgs a = curve_args(p, fam);
    a.u_even = u_even;
    a.u_odd = u_odd;
    a.state = use_state ? p->state : nullptr;
    const bool ref = p->opts.prec == ADR_FP32_REFINE;
    const int R = F.cmax;  // rows of the family's longest chunk
    cudaStream_t st = p->stream;
#define ADR_SOLVE(BS_, I_)                                                                         \
    if (I_.count) {                                                                                \
        const size_t sm = solve_smem<BS_>(R);                                                      \
        if (ref) {                                                                                 \
            if (fam == 0) k_curve_solve<BS_, 0, true><<<I_.count, BS_, sm, st>>>(a, I_.T, I_.curve, I_.lanec, I_.lanec32); \
            else k_curve_solve<BS_, 1, true><<<I_.count, BS_, sm, st>>>(a, I_.T, I_.curve, I_.lanec, I_.lanec32);         \
        } else {                                                                                   \
            if (fam == 0) k_curve_solve<BS_, 0, false><<<I_.count, BS_, sm, st>>>(a, I_.T, I_.curve, I_.lanec, I_.lanec32); \
            else k_curve_solve<BS_, 1, false><<<I_.count, BS_, sm, st>>>(a, I_.T, I_.curve, I_.lanec, I_.lanec32);         \
        }                                                                                          \
    }
    ADR_SOLVE(1024, F.iset[2])
    ADR_SOLVE(512, F.iset[1])
    ADR_SOLVE(256, F.iset[0])
#undef ADR_SOLVE
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

// the curve solve of the direct transfer: u_even / u_odd are node arrays of
// the family (selected by the step's parity when use_state)
adr_status launch_line_solve_dir(Problem* p, int fam, double dt, const double* u_even,
                                 const double* u_odd, bool use_state)
{
    Family& F = p->fam[fam];
    if (!F.prep_valid || F.prep_paper || F.prep_dt != dt) {
        set_error("internal: curve systems not factored for this step");
        return ADR_EINVAL;
    }
    const bool ref = p->opts.prec == ADR_FP32_REFINE;
    TRY_S(ensure_solve_attrs());
    CurveArgs a = curve_args(p, fam);
    a.u_even = u_even;
    a.u_odd = u_odd;
    a.state = use_state ? p->state : nullptr;
    const int R = F.cmax;
    cudaStream_t st = p->stream;
#define ADR_SOLVE_DIR(BS_, I_)                                                                     \
    if (I_.count) {                                                                                \
        const size_t sm = solve_smem<BS_>(R);                                                      \
        if (ref) {                                                                                 \
            if (fam == 0) k_curve_solve_dir<BS_, 0, true><<<I_.count, BS_, sm, st>>>(a, I_.T, I_.curve, I_.lanec, I_.lanec32); \
            else k_curve_solve_dir<BS_, 1, true><<<I_.count, BS_, sm, st>>>(a, I_.T, I_.curve, I_.lanec, I_.lanec32);         \
        } else {                                                                                   \
            if (fam == 0) k_curve_solve_dir<BS_, 0><<<I_.count, BS_, sm, st>>>(a, I_.T, I_.curve, I_.lanec, I_.lanec32); \
            else k_curve_solve_dir<BS_, 1><<<I_.count, BS_, sm, st>>>(a, I_.T, I_.curve, I_.lanec, I_.lanec32);         \
        }                                                                                          \
    }
    ADR_SOLVE_DIR(1024, F.iset[2])
    ADR_SOLVE_DIR(512, F.iset[1])
    ADR_SOLVE_DIR(256, F.iset[0])
#undef ADR_SOLVE_DIR
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

// the gather pass runs one node per thread: every node's loads are in flight
// at once instead of behind a grid-stride loop
static int gather_blocks(const Family& F)
{
    const long long b = ((long long)F.n_nodes + 255) / 256;
    return (int)(b > 0 ? (b < 0x7fffffffLL ? b : 0x7fffffff) : 1);
}

// one curve solve through the grid in FP64: the gather pass into the
// family's node values, then the curve solve from them (the same arithmetic
// as the solve's own gather, split so that the gathers' latency does not
// hold up the elimination chain); other modes keep the gather in the solve
adr_status launch_substep_solve(Problem* p, int fam, double dt, const double* u_even, const double* u_odd,
                                bool use_state)
{
    Family& F = p->fam[fam];
    if (!F.ug) return launch_line_solve(p, fam, dt, u_even, u_odd, use_state, 0);
    const long long n = F.n_nodes;
    const int blocks = gather_blocks(F);
    k_gather_grid<<<blocks, 256, 0, p->stream>>>(n, F.ncell, F.nw, p->grid.nx, u_even, u_odd,
                                                 use_state ? p->state : nullptr, F.ug);
    ADR_CUDA_TRY(cudaGetLastError());
    return launch_line_solve_dir(p, fam, dt, F.ug, F.ug, use_state);
}

// the two passes apart (kernel timing): the gather alone, the solve alone
adr_status launch_gather_pass(Problem* p, int fam, const double* u)
{
    Family& F = p->fam[fam];
    if (!F.ug) return ADR_OK;
    k_gather_grid<<<gather_blocks(F), 256, 0, p->stream>>>(F.n_nodes, F.ncell, F.nw, p->grid.nx, u, u,
                                                             nullptr, F.ug);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

adr_status launch_solve_pass(Problem* p, int fam, double dt, const double* u)
{
    Family& F = p->fam[fam];
    if (!F.ug) return launch_line_solve(p, fam, dt, u, u, false, 0);
    return launch_line_solve_dir(p, fam, dt, F.ug, F.ug, false);
}

// direct transfer into the nodes of family to_fam from values v of the other
// family; out by the parity of (iter + shift) when use_state; with norms,
// against prev (by parity) into the problem's partial sums
adr_status launch_xfer(Problem* p, int to_fam, const double* v, double* out_even, double* out_odd,
                       int shift, const double* prev_even, const double* prev_odd, bool use_state,
                       bool norms)
{
    const Family& T = p->fam[to_fam];
    XferArgs a;
    a.n = T.n_nodes;
    a.xg = T.xg;
    a.xc = T.xc;
    a.v = v;
    a.out_even = out_even;
    a.out_odd = out_odd;
    a.prev_even = prev_even;
    a.prev_odd = prev_odd;
    a.state = use_state ? p->state : nullptr;
    a.parity_shift = shift;
    a.partial = p->partial;
    const int blocks = grid_map_blocks(p);  // the check kernel reads this many partial sums
    if (norms) k_curve_xfer<true><<<blocks, kGridThreads, 0, p->stream>>>(a);
    else k_curve_xfer<false><<<blocks, kGridThreads, 0, p->stream>>>(a);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

adr_status launch_gather_nodes(Problem* p, int fam, const double* u, double* out)
{
    const Family& F = p->fam[fam];
    const int blocks = (int)(((long long)F.n_lines * 32 + 255) / 256);
    k_gather_nodes<<<blocks > 0 ? blocks : 1, 256, 0, p->stream>>>(p->grid.nx, p->grid.ny, F.n_lines, F.off,
                                                                  F.xi, F.eta, u, out);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

adr_status launch_node_midpoint(Problem* p, const double* u_even, const double* u_odd, const double* vb,
                                double* out, bool use_state)
{
    const long long n = p->fam[0].n_nodes;
    k_node_midpoint<<<(int)((n + 255) / 256), 256, 0, p->stream>>>(use_state ? p->state : nullptr, u_even,
                                                                   u_odd, vb, out, n);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

adr_status launch_map_coef(Problem* p, int fam)
{
    Family& F = p->fam[fam];
    long long N = p->N;
    k_map_coef<<<(int)((N + 255) / 256), 256, 0, p->stream>>>(N, p->ntype, F.cg, F.ct, F.cw, F.cpos,
                                                            p->opts.interp_weights, F.mg, F.mc);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

adr_status launch_grid_map_ex(Problem* p, int fam, double* out_even, double* out_odd,
                              int parity_shift, const double* prev_even, const double* prev_odd,
                              bool use_state, bool norms, const double* vin)
{
    Family& F = p->fam[fam];
    GridArgs a;
    a.nx = p->grid.nx;
    a.ny = p->grid.ny;
    a.ntype = p->ntype;
    a.mg = F.mg;
    a.mc = F.mc;
    a.v = vin ? vin : F.v;
    a.out_even = out_even;
    a.out_odd = out_odd;
    a.prev_even = prev_even;
    a.prev_odd = prev_odd;
    a.state = use_state ? p->state : nullptr;
    a.parity_shift = parity_shift;
    a.partial = p->partial;
    int blocks = grid_map_blocks(p);
    if (norms) k_grid_map<true><<<blocks, kGridThreads, 0, p->stream>>>(a);
    else k_grid_map<false><<<blocks, kGridThreads, 0, p->stream>>>(a);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

// grid-stride map: at most 8 blocks of 256 threads per SM
int grid_map_blocks(const Problem* p)
{
    long long need = (p->N + kGridThreads - 1) / kGridThreads;
    int per_sm = (p->map_blocks_per_sm >= 1 && p->map_blocks_per_sm <= 8) ? p->map_blocks_per_sm : 4;
    long long cap = (long long)per_sm * (p->n_sm > 0 ? p->n_sm : 152);
    return (int)(need < cap ? need : cap);
}

adr_status launch_check_ex(Problem* p, double tol, int max_iter,
                           cudaGraphConditionalHandle handle, bool use_cond)
{
    k_check<<<1, 256, 0, p->stream>>>(p->state, p->partial, grid_map_blocks(p), tol, max_iter,
                                      handle, use_cond ? 1 : 0);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

adr_status launch_finish(Problem* p, double* out, double* iter_out, bool midpoint)
{
    long long N = p->N;
    k_finish<<<(int)((N + 255) / 256), 256, 0, p->stream>>>(p->state, p->ubuf[0], p->ubuf[1],
                                                            p->ubuf[2], out, iter_out, N,
                                                            midpoint ? 1 : 0);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

adr_status launch_mask_copy(Problem* p, const double* in, double* out)
{
    long long N = p->N;
    k_mask_copy<<<(int)((N + 255) / 256), 256, 0, p->stream>>>(p->ntype, in, out, N);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

adr_status launch_state_reset(Problem* p)
{
    k_reset<<<1, 1, 0, p->stream>>>(p->state);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}


// ------------------------------------------------------------ batch tables

struct BatchDev {
    int n = 0;
    CurveArgs* ctab = nullptr;   // [2n]
    GridArgs* gtab = nullptr;    // [2n]
    BatchItem* items[kItemSets] = {nullptr, nullptr, nullptr};
    int n_items[kItemSets] = {0, 0, 0};
    int grid_items[kItemSets] = {0, 0, 0};  // persistent grid size per set
    int* blk_prob = nullptr;
    int* blk_local = nullptr;
    int* nblk = nullptr;
    int n_blk = 0;
    IterState** states = nullptr;
    double** partials = nullptr;
    double* tol = nullptr;
    int* max_iter = nullptr;
    unsigned int* ticket = nullptr;
    bool ref = false;
    int R = 1;  // rows of the longest chunk of the batch's problems (shared-memory size)
    // active lists (see ActiveLists)
    ActiveLists act{};
    const BatchItem** d_items = nullptr;  // [6] item arrays per family and set
    int* d_n_items = nullptr;             // [6]
    int map_grid = 0;
    // work items per family and set, with their persistent grid sizes
    BatchItem* it[2][kItemSets] = {};
    int nit[2][kItemSets] = {};
    int git[2][kItemSets] = {};
    GatherArgs* gath = nullptr;  // [2n] gather passes (null: the solves gather themselves)
    void* aa_table = nullptr;  // per-problem Anderson arguments (null: no problem extrapolates)
    int aa_mmax = 0;
    std::vector<void*> owned;
};

template <typename T>
static adr_status bdev_alloc(BatchDev* b, T** ptr, size_t count)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
        return ADR_ENOMEM;
    }
    b->owned.push_back(q);
    *ptr = static_cast<T*>(q);
    return ADR_OK;
}

void batch_dev_destroy(BatchDev* b)
{
    if (!b) return;
    for (void* q : b->owned) cudaFree(q);
    delete b;
}

static adr_status batch_dev_items(BatchDev* b, Problem* const* ps, int fam, BatchItem** items_out,
                                  int* counts, int* grids);

// Build the device tables of a batch.  dts[i]: pseudo step of problem i.
adr_status batch_dev_create(Problem* const* ps, int n, const double* dts, const double* tols,
                            const int* max_iters, BatchDev** out)
{
    BatchDev* b = new BatchDev;
    b->n = n;
    b->ref = ps[0]->opts.prec == ADR_FP32_REFINE;
    for (int i = 0; i < n; ++i) b->R = std::max({b->R, ps[i]->fam[0].cmax, ps[i]->fam[1].cmax});
    {
        adr_status sa = ensure_solve_attrs();
        if (sa != ADR_OK) {
            delete b;
            return sa;
        }
    }
    auto fail = [&](adr_status s) {
        batch_dev_destroy(b);
        return s;
    };
    std::vector<CurveArgs> ct(2 * n);
    std::vector<GridArgs> gt(2 * n);
    std::vector<GatherArgs> ga(2 * n);
    bool split = true;  // every problem has its gather pass
    for (int i = 0; i < n; ++i) split = split && ps[i]->fam[0].ug && ps[i]->fam[1].ug;
    std::vector<int> bp, bl, nb(n);
    std::vector<IterState*> sts(n);
    std::vector<double*> parts(n);
    for (int i = 0; i < n; ++i) {
        Problem* p = ps[i];
        {
            adr_status se = ensure_iteration_active(p);  // the tables hold its buffers
            if (se != ADR_OK) return fail(se);
        }
        for (int fam = 0; fam < 2; ++fam) {
            CurveArgs a = curve_args(p, fam);
            a.u_even = fam == 0 ? p->ubuf[0] : p->ubuf[2];
            a.u_odd = fam == 0 ? p->ubuf[1] : p->ubuf[2];
            a.state = p->state;
            if (split) {
                const Family& F = p->fam[fam];
                GatherArgs g{F.n_nodes, F.ncell, F.nw, p->grid.nx, a.u_even, a.u_odd, p->state, F.ug};
                ga[2 * i + fam] = g;
                a.u_even = a.u_odd = F.ug;  // the solve reads the node values
            }
            a.dt = dts[i];
            a.td = p->opts.theta * dts[i];
            a.paper = 0;
            a.vform = p->opts.prec == ADR_FP64;
            for (int k = 0; k < kItemSets; ++k) {
                a.lanecs[k] = p->fam[fam].iset[k].lanec;
                a.lanec32s[k] = p->fam[fam].iset[k].lanec32;
            }
            ct[2 * i + fam] = a;
            GridArgs g{};
            g.nx = p->grid.nx;
            g.ny = p->grid.ny;
            g.ntype = p->ntype;
            g.mg = p->fam[fam].mg;
            g.mc = p->fam[fam].mc;
            g.v = p->fam[fam].v;
            g.state = p->state;
            g.partial = p->partial;
            if (fam == 0) {
                g.out_even = g.out_odd = p->ubuf[2];
                g.parity_shift = 0;
            } else {
                g.out_even = p->ubuf[0];
                g.out_odd = p->ubuf[1];
                g.prev_even = p->ubuf[0];
                g.prev_odd = p->ubuf[1];
                g.parity_shift = 1;
            }
            gt[2 * i + fam] = g;
        }
        // work items of both families share the item lists (the B and G
        // curves of a problem differ, so items are per family): the batch
        // keeps one list per family and set
        nb[i] = grid_map_blocks(p);
        for (int q = 0; q < nb[i]; ++q) {
            bp.push_back(i);
            bl.push_back(q);
        }
        sts[i] = p->state;
        parts[i] = p->partial;
    }
    b->n_blk = (int)bp.size();
    adr_status s;
    if (split) {
        if ((s = bdev_alloc(b, &b->gath, 2 * n))) return fail(s);
        cudaError_t eg = cudaMemcpy(b->gath, ga.data(), sizeof(GatherArgs) * ga.size(), cudaMemcpyHostToDevice);
        if (eg != cudaSuccess) return fail(cuda_fail(eg, "batch tables"));
    }
    if ((s = bdev_alloc(b, &b->ctab, 2 * n)) || (s = bdev_alloc(b, &b->gtab, 2 * n)) ||
        (s = bdev_alloc(b, &b->blk_prob, b->n_blk)) || (s = bdev_alloc(b, &b->blk_local, b->n_blk)) ||
        (s = bdev_alloc(b, &b->nblk, n)) || (s = bdev_alloc(b, &b->states, n)) ||
        (s = bdev_alloc(b, &b->partials, n)) || (s = bdev_alloc(b, &b->tol, n)) ||
        (s = bdev_alloc(b, &b->max_iter, n)) || (s = bdev_alloc(b, &b->ticket, 1)))
        return fail(s);
    cudaError_t e;
    if ((e = cudaMemcpy(b->ctab, ct.data(), sizeof(CurveArgs) * ct.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->gtab, gt.data(), sizeof(GridArgs) * gt.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->blk_prob, bp.data(), sizeof(int) * bp.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->blk_local, bl.data(), sizeof(int) * bl.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->nblk, nb.data(), sizeof(int) * n, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->states, sts.data(), sizeof(IterState*) * n, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->partials, parts.data(), sizeof(double*) * n, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->tol, tols, sizeof(double) * n, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->max_iter, max_iters, sizeof(int) * n, cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(b->ticket, 0, sizeof(unsigned int))))
        return fail(cuda_fail(e, "batch tables"));
    for (int fam = 0; fam < 2; ++fam)
        if ((s = batch_dev_items(b, ps, fam, b->it[fam], b->nit[fam], b->git[fam]))) return fail(s);
    // active lists
    std::vector<const BatchItem*> ip(6);
    std::vector<int> ni(6);
    for (int fam = 0; fam < 2; ++fam)
        for (int k = 0; k < 3; ++k) {
            ip[fam * 3 + k] = b->it[fam][k];
            ni[fam * 3 + k] = b->nit[fam][k];
            for (int buf = 0; buf < 2; ++buf)
                if ((s = bdev_alloc(b, &b->act.items[buf][fam][k], ni[fam * 3 + k] + 1))) return fail(s);
        }
    for (int buf = 0; buf < 2; ++buf)
        if ((s = bdev_alloc(b, &b->act.blocks[buf], b->n_blk + 1))) return fail(s);
    {
        int** bd = nullptr;
        if ((s = bdev_alloc(b, &bd, 2))) return fail(s);
        if ((e = cudaMemcpy(bd, b->act.blocks, sizeof(int*) * 2, cudaMemcpyHostToDevice)))
            return fail(cuda_fail(e, "batch lists"));
        b->act.blocks_dev = bd;
    }
    if ((s = bdev_alloc(b, &b->act.count, 2 * kCountPerBuf)) || (s = bdev_alloc(b, &b->act.sel, 1)) ||
        (s = bdev_alloc(b, &b->act.changed, 1)) || (s = bdev_alloc(b, &b->d_items, 6)) ||
        (s = bdev_alloc(b, &b->d_n_items, 6)))
        return fail(s);
    if ((e = cudaMemcpy(b->d_items, ip.data(), sizeof(BatchItem*) * 6, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->d_n_items, ni.data(), sizeof(int) * 6, cudaMemcpyHostToDevice)))
        return fail(cuda_fail(e, "batch lists"));
    {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        b->map_grid = std::min(b->n_blk, 8 * nsm);
    }
    if ((s = anderson_batch_table(ps, n, &b->aa_table, &b->aa_mmax))) return fail(s);
    if (b->aa_table) b->owned.push_back(b->aa_table);
    *out = b;
    return ADR_OK;
}

adr_status batch_dev_reset(BatchDev* b, cudaStream_t st)
{
    k_batch_reset<<<256, 256, 0, st>>>(b->act, b->d_n_items, b->n_blk);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

// Items of one family over all problems (one list per set), longest first.
static adr_status batch_dev_items(BatchDev* b, Problem* const* ps, int fam, BatchItem** items_out,
                           int* counts, int* grids)
{
    std::vector<BatchItem> its[kItemSets];
    for (int i = 0; i < b->n; ++i) {
        Family& F = ps[i]->fam[fam];
        for (int k = 0; k < kItemSets; ++k) {
            const ItemSet& I = F.iset[k];
            if (!I.count) continue;
            int maxc = I.BS / 32;
            std::vector<int> T(I.count), cv((size_t)I.count * maxc);
            cudaError_t e;
            if ((e = cudaMemcpy(T.data(), I.T, sizeof(int) * I.count, cudaMemcpyDeviceToHost)) ||
                (e = cudaMemcpy(cv.data(), I.curve, sizeof(int) * cv.size(), cudaMemcpyDeviceToHost)))
                return cuda_fail(e, "batch items");
            for (int q = 0; q < I.count; ++q) {
                BatchItem bi;
                bi.prob = i;
                bi.T = T[q];
                bi.local = q;
                for (int r = 0; r < 8; ++r) bi.curves[r] = r < maxc ? cv[(size_t)q * maxc + r] : -1;
                its[k].push_back(bi);
            }
        }
    }
    for (int k = 0; k < kItemSets; ++k) {
        std::stable_sort(its[k].begin(), its[k].end(),
                         [](const BatchItem& x, const BatchItem& y) { return x.T > y.T; });
        counts[k] = (int)its[k].size();
        items_out[k] = nullptr;
        grids[k] = 0;
        if (!counts[k]) continue;
        TRY_S(bdev_alloc(b, &items_out[k], its[k].size()));
        ADR_CUDA_TRY(cudaMemcpy(items_out[k], its[k].data(), sizeof(BatchItem) * its[k].size(),
                                cudaMemcpyHostToDevice));
        int BS = 256 << k, per_sm = 0, dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e;
        const int R = b->R;
        if (BS == 256)
            e = b->ref ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_curve_solve_batch<256, 0, true>, 256, solve_smem<256>(R))
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_curve_solve_batch<256, 0, false>, 256, solve_smem<256>(R));
        else if (BS == 512)
            e = b->ref ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_curve_solve_batch<512, 0, true>, 512, solve_smem<512>(R))
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_curve_solve_batch<512, 0, false>, 512, solve_smem<512>(R));
        else
            e = b->ref ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_curve_solve_batch<1024, 0, true>, 1024, solve_smem<1024>(R))
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_curve_solve_batch<1024, 0, false>, 1024, solve_smem<1024>(R));
        if (e != cudaSuccess) return cuda_fail(e, "occupancy");
        int g = (per_sm > 0 ? per_sm : 1) * nsm;
        grids[k] = counts[k] < g ? counts[k] : g;
    }
    return ADR_OK;
}

// one split step of every active problem (captured in the batch graph)
adr_status batch_dev_step(BatchDev* b, cudaStream_t st, cudaGraphConditionalHandle cond)
{
    BatchItem* const* itB = b->it[0];
    BatchItem* const* itG = b->it[1];
    const int *nB = b->nit[0], *gB = b->git[0], *nG = b->nit[1], *gG = b->git[1];
    const int R = b->R;
    const bool dir = b->gath != nullptr;  // gather passes, then solves from the node values
#define ADR_BATCH_SOLVE_BS(BS_, FAM_, IT, G)                                                        \
    if (b->ref) {                                                                                  \
        if (dir) k_curve_solve_batch<BS_, FAM_, true, true><<<G[k], BS_, solve_smem<BS_>(R), st>>>(b->ctab, IT[k], b->act, k); \
        else k_curve_solve_batch<BS_, FAM_, true><<<G[k], BS_, solve_smem<BS_>(R), st>>>(b->ctab, IT[k], b->act, k);          \
    } else {                                                                                       \
        if (dir) k_curve_solve_batch<BS_, FAM_, false, true><<<G[k], BS_, solve_smem<BS_>(R), st>>>(b->ctab, IT[k], b->act, k); \
        else k_curve_solve_batch<BS_, FAM_, false><<<G[k], BS_, solve_smem<BS_>(R), st>>>(b->ctab, IT[k], b->act, k);          \
    }
#define ADR_BATCH_SOLVE(FAM_, IT, N, G)                                                            \
    if (dir)                                                                                       \
        k_gather_batch<<<b->map_grid, 256, 0, st>>>(b->gath, FAM_, b->blk_prob, b->blk_local, b->nblk, \
                                                    b->act.blocks_dev, b->act.count, b->act.sel);    \
    for (int k = kItemSets - 1; k >= 0; --k) {                                                     \
        if (!N[k]) continue;                                                                       \
        int BS = 256 << k;                                                                         \
        if (BS == 256) {                                                                           \
            ADR_BATCH_SOLVE_BS(256, FAM_, IT, G)                                                   \
        } else if (BS == 512) {                                                                    \
            ADR_BATCH_SOLVE_BS(512, FAM_, IT, G)                                                   \
        } else {                                                                                   \
            ADR_BATCH_SOLVE_BS(1024, FAM_, IT, G)                                                  \
        }                                                                                          \
    }
    ADR_BATCH_SOLVE(0, itB, nB, gB)
    k_grid_map_batch<false><<<b->map_grid, kGridThreads, 0, st>>>(b->gtab, 0, b->blk_prob, b->blk_local,
                                                                 b->nblk, b->act.blocks_dev, b->act.count,
                                                                 b->act.sel);
    ADR_BATCH_SOLVE(1, itG, nG, gG)
    k_grid_map_batch<true><<<b->map_grid, kGridThreads, 0, st>>>(b->gtab, 1, b->blk_prob, b->blk_local,
                                                                b->nblk, b->act.blocks_dev, b->act.count,
                                                                b->act.sel);
#undef ADR_BATCH_SOLVE
#undef ADR_BATCH_SOLVE_BS
    k_check_batch<<<b->n, 256, 0, st>>>(b->states, (const double* const*)b->partials, b->nblk, b->n,
                                        b->tol, b->max_iter, b->ticket, cond, b->act.changed);
    if (b->aa_table) {
        // the extrapolated next states of the problems that go on
        AaBatchView v{b->aa_table, b->n, b->aa_mmax, b->map_grid, b->blk_prob, b->blk_local, b->nblk,
                      b->act.blocks_dev, b->act.count, b->act.sel};
        TRY_S(launch_anderson_batch(v, st));
    }
    k_batch_compact<<<b->map_grid, 256, 0, st>>>(b->act, b->d_items, b->d_n_items, b->blk_prob,
                                                 b->n_blk, b->states);
    k_batch_flip<<<1, 1, 0, st>>>(b->act);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

}  // namespace adr
