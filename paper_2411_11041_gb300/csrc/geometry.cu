// Setup kernels: domain, curve families B and G, and the curve -> grid
// crossing structure (§6).  Run once per problem.  This file is compiled with
// -fmad=false so that every coordinate follows plain IEEE operations in the
// written order; the integer decisions that depend on them (node counts,
// snapped grid coordinates, chosen crossings) are then reproducible.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kThreads = 256;

inline int blocks_for(long long n, int t = kThreads)
{
    long long b = (n + t - 1) / t;
    return (int)(b < 1 ? 1 : b);
}

// status bits raised by setup kernels
enum : int { kErrInvalid = 1, kErrGeom = 2, kErrCapacity = 4, kErrUncovered = 8 };

__device__ __forceinline__ double snap(double v)
{
    double r = rint(v);
    return fabs(v - r) <= kSnapTol ? r : v;
}

__device__ __forceinline__ int cell_on(const GridView& g, int i, int r)
{
    if (i < 0 || r < 0 || i >= g.nx - 1 || r >= g.ny - 1) return 0;
    return g.cell[(size_t)r * (g.nx - 1) + i];
}

// interior of Omega_h: every cell whose closure holds the point is active
__device__ int interior_point(const GridView& g, double xi, double eta)
{
    if (!isfinite(xi) || !isfinite(eta)) return 0;
    if (xi < -1.0 || eta < -1.0 || xi > g.nx || eta > g.ny) return 0;
    double fx = floor(xi), fy = floor(eta);
    int i0 = (int)fx, i1 = (int)fx, r0 = (int)fy, r1 = (int)fy;
    if (xi == fx) i0 = (int)fx - 1;
    if (eta == fy) r0 = (int)fy - 1;
    for (int r = r0; r <= r1; ++r)
        for (int i = i0; i <= i1; ++i)
            if (!cell_on(g, i, r)) return 0;
    return 1;
}

// bilinear interpolation (§6.1), cell i = min(floor(xi), nx-2), clamped at 0
__device__ double bilin(const GridView& g, const double* a, double xi, double eta)
{
    int i = (int)floor(xi), r = (int)floor(eta);
    if (i > g.nx - 2) i = g.nx - 2;
    if (i < 0) i = 0;
    if (r > g.ny - 2) r = g.ny - 2;
    if (r < 0) r = 0;
    double lx = xi - i, ly = eta - r;
    const double* r0 = a + (size_t)r * g.nx;
    const double* r1 = r0 + g.nx;
    double p11 = r0[i], p12 = r0[i + 1], p21 = r1[i], p22 = r1[i + 1];
    return (1.0 - ly) * (1.0 - lx) * p11 + (1.0 - ly) * lx * p12 + ly * (1.0 - lx) * p21 +
           ly * lx * p22;
}

// beta1 and beta2 bilinear at one point: bilin's cell, local coordinates,
// weights and sums, with the cell and the four weights computed once for the
// two fields (the same values, bit for bit, as two calls of bilin).  The
// traces are chains of dependent FP64 operations, each of which costs tens of
// cycles, so every operation taken off a stage shortens them.
__device__ __forceinline__ void bilin_beta(const GridView& g, double xi, double eta, double* b1,
                                           double* b2)
{
    int i = __double2int_rd(xi), r = __double2int_rd(eta);  // (int)floor, one conversion
    if (i > g.nx - 2) i = g.nx - 2;
    if (i < 0) i = 0;
    if (r > g.ny - 2) r = g.ny - 2;
    if (r < 0) r = 0;
    const double lx = xi - i, ly = eta - r;
    const double ax = 1.0 - lx, ay = 1.0 - ly;
    const double w11 = ay * ax, w12 = ay * lx, w21 = ly * ax, w22 = ly * lx;
    const size_t o = (size_t)r * g.nx + i;
    const double* p = g.beta1 + o;
    const double* q = g.beta2 + o;
    const double p11 = p[0], p12 = p[1], p21 = p[g.nx], p22 = p[g.nx + 1];
    const double q11 = q[0], q12 = q[1], q21 = q[g.nx], q22 = q[g.nx + 1];
    *b1 = w11 * p11 + w12 * p12 + w21 * p21 + w22 * p22;
    *b2 = w11 * q11 + w12 * q12 + w21 * q21 + w22 * q22;
}

// physical unit direction of family fam at the index coordinates (xi, eta):
// b (B) or p (G), §3
__device__ __forceinline__ int direction(const GridView& g, int fam, double xi, double eta,
                                         double* dx, double* dy)
{
    double b1, b2;
    bilin_beta(g, xi, eta, &b1, &b2);
    double nb = sqrt(b1 * b1 + b2 * b2);
    if (!(nb > 0.0)) return -1;
    if (fam == 0) {
        *dx = b1 / nb;
        *dy = b2 / nb;
    } else {
        *dx = b2 / nb;
        *dy = -b1 / nb;
    }
    return 0;
}

// classical RK4 step of x' = dir(x) over an arc length ds (eqs.
// CauchyBeta/CauchyGamma), in index coordinates: the step is (sx, sy) =
// (ds / hx, ds / hy) along the two axes
__device__ int rk4(const GridView& g, int fam, double X, double Y, double sx, double sy,
                   double* Xo, double* Yo)
{
    double k1x, k1y, k2x, k2y, k3x, k3y, k4x, k4y;
    if (direction(g, fam, X, Y, &k1x, &k1y)) return -1;
    if (direction(g, fam, X + 0.5 * sx * k1x, Y + 0.5 * sy * k1y, &k2x, &k2y)) return -1;
    if (direction(g, fam, X + 0.5 * sx * k2x, Y + 0.5 * sy * k2y, &k3x, &k3y)) return -1;
    if (direction(g, fam, X + sx * k3x, Y + sy * k3y, &k4x, &k4y)) return -1;
    *Xo = X + sx / 6.0 * (k1x + 2.0 * k2x + 2.0 * k3x + k4x);
    *Yo = Y + sy / 6.0 * (k1y + 2.0 * k2y + 2.0 * k3y + k4y);
    return 0;
}

__device__ __forceinline__ int elements_for(const GridView& g, double L)
{
    int n = (int)ceil(L / g.hs - kNodeTol);
    return n < 1 ? 1 : n;
}

// ------------------------------------------------------------- domain

__global__ void k_cells(const uint8_t* mask, int nx, int ny, uint8_t* cell)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long nc = (long long)(nx - 1) * (ny - 1);
    if (k >= nc) return;
    int r = (int)(k / (nx - 1)), i = (int)(k % (nx - 1));
    size_t a = (size_t)r * nx + i;
    cell[k] = (mask[a] && mask[a + 1] && mask[a + nx] && mask[a + nx + 1]) ? 1 : 0;
}

__global__ void k_ntype(GridView g, uint8_t* ntype, int* counts /* [0] interior, [1] in */)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= (long long)g.nx * g.ny) return;
    int r = (int)(k / g.nx), i = (int)(k % g.nx);
    int c00 = cell_on(g, i - 1, r - 1), c10 = cell_on(g, i, r - 1);
    int c01 = cell_on(g, i - 1, r), c11 = cell_on(g, i, r);
    uint8_t t = kOutside;
    if (c00 || c10 || c01 || c11) t = (c00 && c10 && c01 && c11) ? kInterior : kDirichlet;
    ntype[k] = t;
    if (t == kInterior) atomicAdd(&counts[0], 1);
    if (t != kOutside) atomicMin(&counts[2], (int)k);  // first node of Omega_h
}

// field checks over Omega_h: finite data, |beta| > 0, constant field, max |beta|;
// each block reduces its nodes first and issues one atomic per result
__global__ void k_fields(GridView g, int first, int* status, int* nonconst,
                         unsigned long long* bmax_bits)
{
    __shared__ unsigned long long smax[kThreads / 32];
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int bad = 0, nc = 0;
    unsigned long long bm = 0;  // bits of |beta| >= 0 order like the values
    if (k < (long long)g.nx * g.ny && g.ntype[k] != kOutside) {
        double b1 = g.beta1[k], b2 = g.beta2[k];
        double nb = sqrt(b1 * b1 + b2 * b2);
        bad = !(nb > 0.0) || !isfinite(nb) || !isfinite(g.f[k]);
        nc = b1 != g.beta1[first] || b2 != g.beta2[first];
        if (isfinite(nb)) bm = (unsigned long long)__double_as_longlong(nb);
    }
    bad = __syncthreads_or(bad);
    nc = __syncthreads_or(nc);
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, bm, o);
        bm = v > bm ? v : bm;
    }
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = bm;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) bm = smax[w] > bm ? smax[w] : bm;
        if (bad) atomicOr(status, kErrInvalid);
        if (nc) atomicOr(nonconst, 1);
        if (bm) atomicMax(bmax_bits, bm);
    }
}

// -------------------------------------------------- straight curve families
// For a constant field the curves are the lines p.(x - x_ref) = k h_s (B) and
// b.(x - x_ref) = k h_s (G), x_ref = (x0, y0), cut into the maximal pieces
// inside Omega_h; s is arc length along the line direction.

struct LineParams {
    double dx, dy, nxv, nyv;
    long long kmin, kmax;
};

__global__ void k_line_params(GridView g, int fam, int first, LineParams* out)
{
    double b1 = g.beta1[first], b2 = g.beta2[first];
    double nb = sqrt(b1 * b1 + b2 * b2);
    double bx = b1 / nb, by = b2 / nb, px = by, py = -bx;
    LineParams P;
    P.dx = fam == 0 ? bx : px;
    P.dy = fam == 0 ? by : py;
    P.nxv = fam == 0 ? px : bx;
    P.nyv = fam == 0 ? py : by;
    double qc[4] = {0.0, P.nxv * g.W, P.nyv * g.H, P.nxv * g.W + P.nyv * g.H};
    double qmin = qc[0], qmax = qc[0];
    for (int c = 1; c < 4; ++c) {
        if (qc[c] < qmin) qmin = qc[c];
        if (qc[c] > qmax) qmax = qc[c];
    }
    P.kmin = (long long)ceil(qmin / g.hs - 1e-9);
    P.kmax = (long long)floor(qmax / g.hs + 1e-9);
    *out = P;
}

// Walks the pieces of line k between consecutive grid-line crossings and
// emits the maximal runs of interior pieces.  FILL = false counts, true writes.
template <bool FILL>
__device__ void straight_line(const GridView& g, const LineParams& P, long long k, int* n_lines,
                              int* n_nodes, int line0, int node0, int* off, double* h,
                              double* xs, double* es)
{
    double dx = P.dx, dy = P.dy;
    double ox = k * g.hs * P.nxv, oy = k * g.hs * P.nyv;
    double slo = -INFINITY, shi = INFINITY;
    double lim[2] = {g.W, g.H}, o[2] = {ox, oy}, d[2] = {dx, dy}, hh[2] = {g.hx, g.hy};
    double top[2] = {(double)(g.nx - 1), (double)(g.ny - 1)};
    for (int a = 0; a < 2; ++a) {
        if (d[a] == 0.0) {
            double c = snap(o[a] / hh[a]);
            if (c < 0.0 || c > top[a]) return;
        } else {
            double s0 = (0.0 - o[a]) / d[a], s1 = (lim[a] - o[a]) / d[a];
            if (s0 > s1) {
                double t = s0;
                s0 = s1;
                s1 = t;
            }
            if (s0 > slo) slo = s0;
            if (s1 < shi) shi = s1;
        }
    }
    if (!(shi > slo)) return;
    // breakpoint generators: grid lines g*hh crossed inside (slo, shi), in s order
    long long gcur[2], gend[2];
    int gstep[2];
    for (int a = 0; a < 2; ++a) {
        gstep[a] = 0;
        if (d[a] == 0.0) continue;
        double c0 = (o[a] + slo * d[a]) / hh[a], c1 = (o[a] + shi * d[a]) / hh[a];
        double lo = c0 < c1 ? c0 : c1, hi = c0 < c1 ? c1 : c0;
        long long ga = (long long)ceil(lo - 1e-9), gb = (long long)floor(hi + 1e-9);
        if (ga > gb) continue;
        if (d[a] > 0) {
            gcur[a] = ga;
            gend[a] = gb;
            gstep[a] = 1;
        } else {
            gcur[a] = gb;
            gend[a] = ga;
            gstep[a] = -1;
        }
    }
    auto next_of = [&](int a) -> double {
        while (gstep[a] != 0) {
            double s = (gcur[a] * hh[a] - o[a]) / d[a];
            if (s > slo && s < shi) return s;
            if (gcur[a] == gend[a]) {
                gstep[a] = 0;
                break;
            }
            gcur[a] += gstep[a];
        }
        return INFINITY;
    };
    auto advance = [&](int a) {
        if (gcur[a] == gend[a]) gstep[a] = 0;
        else gcur[a] += gstep[a];
    };
    int lines = 0, nodes = 0;
    auto emit = [&](double sa, double sb) {
        double L = sb - sa;
        int n = elements_for(g, L);
        if (FILL) {
            int base = node0 + nodes;
            for (int j = 0; j <= n; ++j) {
                double s = (j == n) ? sb : sa + j * (L / n);
                xs[base + j] = snap((ox + s * dx) / g.hx);
                es[base + j] = snap((oy + s * dy) / g.hy);
            }
            off[line0 + lines] = base;
            h[line0 + lines] = L / n;
        }
        lines += 1;
        nodes += n + 1;
    };
    double prev = slo, run_a = 0.0, run_b = 0.0;
    int open = 0;
    for (;;) {
        double sa = next_of(0), sb = next_of(1);
        double nxt;
        int which;
        if (sa <= sb && sa < shi) {
            nxt = sa;
            which = 0;
        } else if (sb < shi) {
            nxt = sb;
            which = 1;
        } else {
            nxt = shi;
            which = 2;
        }
        double s0 = prev, s1 = nxt;
        if (s1 - s0 > 1e-9 * g.hs) {
            double sm = 0.5 * (s0 + s1);
            double xi = snap((ox + sm * dx) / g.hx), eta = snap((oy + sm * dy) / g.hy);
            if (interior_point(g, xi, eta)) {
                if (!open) {
                    run_a = s0;
                    open = 1;
                }
                run_b = s1;
            } else if (open) {
                emit(run_a, run_b);
                open = 0;
            }
        }
        if (which == 2) break;
        advance(which);
        prev = nxt;
    }
    if (open) emit(run_a, run_b);
    *n_lines = lines;
    *n_nodes = nodes;
}

__global__ void k_straight_count(GridView g, const LineParams* P, long long* cl, long long* cn)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long nk = P->kmax - P->kmin + 1;
    if (t >= nk) return;
    int nl = 0, nn = 0;
    straight_line<false>(g, *P, P->kmin + t, &nl, &nn, 0, 0, nullptr, nullptr, nullptr,
                         nullptr);
    cl[t] = nl;
    cn[t] = nn;
}

__global__ void k_straight_fill(GridView g, const LineParams* P, const long long* cl,
                                const long long* cn, int* off, double* h, double* xs, double* es)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long nk = P->kmax - P->kmin + 1;
    if (t >= nk) return;
    int nl = 0, nn = 0;
    straight_line<true>(g, *P, P->kmin + t, &nl, &nn, (int)cl[t], (int)cn[t], off, h, xs, es);
}

// exclusive scan of a small int64 array by one block; out[n] = total
__global__ void k_scan(const long long* in, long long* out, long long n)
{
    __shared__ long long buf[1024];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long base = 0; base < n; base += 1024) {
        long long i = base + threadIdx.x;
        long long v = i < n ? in[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int s = 1; s < 1024; s <<= 1) {
            long long add = threadIdx.x >= s ? buf[threadIdx.x - s] : 0;
            __syncthreads();
            buf[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < n) out[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

// exclusive scan of many counts: every block scans 1024 of them and records
// its total, one block scans the totals (k_scan), and the block offsets are
// added back
__global__ void k_scan_blocks(const long long* in, long long* out, long long n, long long* bsum)
{
    __shared__ long long buf[1024];
    const long long i = blockIdx.x * 1024LL + threadIdx.x;
    const long long v = i < n ? in[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int s = 1; s < 1024; s <<= 1) {
        long long add = threadIdx.x >= s ? buf[threadIdx.x - s] : 0;
        __syncthreads();
        buf[threadIdx.x] += add;
        __syncthreads();
    }
    if (i < n) out[i] = buf[threadIdx.x] - v;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = buf[1023];
}

__global__ void k_scan_add(long long* out, long long n, const long long* boff)
{
    const long long i = blockIdx.x * 1024LL + threadIdx.x;
    if (i < n) out[i] += boff[blockIdx.x];
}

// ---------------------------------------------------- traced curve families
// Seeds on the inflow part of the boundary (eq. cauchyStartSets): the staircase
// boundary is walked loop by loop counter-clockwise (domain on the left), each
// loop from its lowest-leftmost bottom edge; edge e carries the transverse
// measure max(0, -n_e . dir) |e| with dir from the nodal mean of beta on e;
// seeds sit where the running measure reaches (k + 1/2) h_s.

__device__ int hedge_dir(const GridView& g, int i, int r)
{
    int up = cell_on(g, i, r), dn = cell_on(g, i, r - 1);
    return up && !dn ? 1 : (dn && !up ? -1 : 0);
}
__device__ int vedge_dir(const GridView& g, int i, int r)
{
    int lf = cell_on(g, i - 1, r), rt = cell_on(g, i, r);
    return lf && !rt ? 1 : (rt && !lf ? -1 : 0);
}
__device__ int out_edge(const GridView& g, int i, int r, int d)
{
    switch (d) {
    case 0: return i <= g.nx - 2 && hedge_dir(g, i, r) == 1;
    case 1: return r <= g.ny - 2 && vedge_dir(g, i, r) == 1;
    case 2: return i >= 1 && hedge_dir(g, i - 1, r) == -1;
    default: return r >= 1 && vedge_dir(g, i, r - 1) == -1;
    }
}
__device__ const int kDXI[4] = {1, 0, -1, 0};
__device__ const int kDETA[4] = {0, 1, 0, -1};

__global__ void k_count_bedges(GridView g, int* count)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= (long long)g.nx * g.ny) return;
    int r = (int)(k / g.nx), i = (int)(k % g.nx);
    int c = 0;
    if (i < g.nx - 1 && hedge_dir(g, i, r)) c++;
    if (r < g.ny - 1 && vedge_dir(g, i, r)) c++;
    if (c) atomicAdd(count, c);
}

// loop starts: the +x boundary edges of every row, in (row, column) order;
// one thread per row counts, then writes its row's edges at its offset
__global__ void k_row_cand_count(GridView g, long long* cnt)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.ny) return;
    long long c = 0;
    for (int i = 0; i < g.nx - 1; ++i) c += hedge_dir(g, i, r) == 1;
    cnt[r] = c;
}
__global__ void k_row_cand_fill(GridView g, const long long* start, int* cand)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.ny) return;
    long long pos = start[r];
    for (int i = 0; i < g.nx - 1; ++i)
        if (hedge_dir(g, i, r) == 1) cand[pos++] = r * (g.nx - 1) + i;
}

// one thread per family (block f): walk the loops from the candidate starts
// and place the seeds (X0, Y0 physical offsets) at sx/sy + f*cap
// Seeds on the inflow boundary (eq. cauchyStartSets).  The boundary of the
// staircase domain is walked loop by loop, counter-clockwise, each loop from
// its first +x edge in (row, column) order; an edge's weight is its inflow
// measure max(0, -n . dir(mid)) |e|, and a seed goes where the running measure
// reaches (k + 1/2) h_s.  The walk is split so that only the running sum is
// serial: every boundary edge's successor is found in parallel (the walk's
// turn rule is local), the boundary edges get compact ids, one thread follows
// the successors in shared memory, the weights are computed in parallel, one
// warp per family accumulates them in walk order (the same sums, so the seeds
// are bit-identical), every edge's first seed index follows from the sums in
// parallel, and the seeds are written in parallel.
//
// Boundary edges carry undirected ids: the horizontal edge (i, r)-(i+1, r) is
// r (nx-1) + i, the vertical edge (i, r)-(i, r+1) is nh + r nx + i.

__device__ __forceinline__ int edge_id(const GridView& g, int i, int r, int d)
{
    const int nh = g.ny * (g.nx - 1);
    switch (d) {
    case 0: return r * (g.nx - 1) + i;
    case 2: return r * (g.nx - 1) + i - 1;
    case 1: return nh + r * g.nx + i;
    default: return nh + (r - 1) * g.nx + i;
    }
}

// per undirected edge: its walk start vertex and direction (packed
// (r nx + i) * 4 + d, -1 when it is not a boundary edge) and its successor
__global__ void k_bnd_succ(GridView g, int* info, int* succ)
{
    const long long nh = (long long)g.ny * (g.nx - 1), nv = (long long)g.nx * (g.ny - 1);
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= nh + nv) return;
    int i, r, d;
    if (e < nh) {
        r = (int)(e / (g.nx - 1));
        i = (int)(e % (g.nx - 1));
        const int s = hedge_dir(g, i, r);
        if (s == 0) {
            info[e] = -1;
            succ[e] = -1;
            return;
        }
        d = s > 0 ? 0 : 2;
        if (s < 0) i += 1;
    } else {
        const long long q = e - nh;
        r = (int)(q / g.nx);
        i = (int)(q % g.nx);
        const int s = vedge_dir(g, i, r);
        if (s == 0) {
            info[e] = -1;
            succ[e] = -1;
            return;
        }
        d = s > 0 ? 1 : 3;
        if (s < 0) r += 1;
    }
    info[e] = (r * g.nx + i) * 4 + d;
    const int ib = i + kDXI[d], rb = r + kDETA[d];
    const int pref[3] = {(d + 1) & 3, d, (d + 3) & 3};
    int nxt = -1;
    for (int q = 0; q < 3; ++q)
        if (out_edge(g, ib, rb, pref[q])) {
            nxt = edge_id(g, ib, rb, pref[q]);
            break;
        }
    succ[e] = nxt;
}

// compact ids of the boundary edges (in any order: only the walk and the
// kernels after it use them, through cinfo); one atomic per warp
__global__ void k_bnd_compact(long long ne, const int* info, int* cid, int* cinfo, int* cedge,
                              int* nb, int cap)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int in = e < ne ? info[e] : -1;
    const unsigned m = __ballot_sync(0xffffffffu, in >= 0);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(nb, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (in >= 0) {
        const int id = base + __popc(m & ((1u << lane) - 1u));
        if (id < cap) {
            cid[e] = id;
            cinfo[id] = in;
            cedge[id] = (int)e;
        }
    }
}

// the successor of every boundary edge as a compact id (-1: none)
__global__ void k_bnd_csucc(const int* nbp, const int* cedge, const int* succ, const int* cid,
                            int* csucc, int cap)
{
    const int nb = *nbp;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb || t >= cap) return;
    const int s = succ[cedge[t]];
    const int c = s >= 0 ? cid[s] : -1;
    csucc[t] = c >= 0 && c < nb && c < cap ? c : -1;
}

// The walk, over compact ids: loop after loop, each from the first unvisited
// candidate in candidate order, following the successors until an edge comes
// round again.  The successors and the visited flags sit in shared memory when
// they fit (use_smem), else in global memory.  Warp 0 runs it: the lanes test
// 32 candidates at a time, lane 0 follows the successors.
__global__ void k_bnd_walk(const int* cand, long long ncand, const int* cid, const int* nbp,
                           const int* csucc, uint8_t* cvis, int use_smem, int smem_cap,
                           long long total, int* order, int* norder)
{
    extern __shared__ int walk_sm[];
    const int nb = *nbp;
    const int* S = csucc;
    uint8_t* V = cvis;
    if (use_smem && nb <= smem_cap) {
        int* sS = walk_sm;
        uint8_t* sV = reinterpret_cast<uint8_t*>(walk_sm + smem_cap);
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            sS[t] = csucc[t];
            sV[t] = 0;
        }
        __syncthreads();
        S = sS;
        V = sV;
    }
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    int pos = 0;
    for (long long c0 = 0; c0 < ncand; c0 += 32) {
        const long long c = c0 + lane;
        int e = c < ncand ? cid[cand[c]] : -1;
        if (e >= nb) e = -1;
        unsigned m = __ballot_sync(0xffffffffu, e >= 0 && !V[e]);
        while (m) {
            const int j = __ffs(m) - 1;
            const int start = __shfl_sync(0xffffffffu, e, j);
            if (lane == 0) {
                int x = start;
                long long steps = 0;
                int sx = S[x], vx = V[x];  // the successor and the flag of x, fetched together
                for (;;) {
                    if (vx) break;
                    V[x] = 1;
                    if (pos < total) order[pos] = x;
                    pos++;
                    if (sx < 0 || ++steps > total + 4) break;
                    x = sx;
                    sx = S[x];
                    vx = V[x];
                }
            }
            pos = __shfl_sync(0xffffffffu, pos, 0);
            __syncwarp();
            m = __ballot_sync(0xffffffffu, lane > j && e >= 0 && !V[e]);
        }
    }
    if (lane == 0) *norder = pos < total ? pos : (int)total;
}

// inflow weight of every walked edge, for both families ([fam][pos])
__global__ void k_bnd_weight(GridView g, const int* order, const int* norder, const int* info,
                             double* w, int cap_order, int* status)
{
    const int n = *norder;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n <= 0 || t >= 2LL * n) return;
    const int fam = (int)(t / n), pos = (int)(t % n);
    const int in = info[order[pos]];
    const int d = in & 3, v = in >> 2, r = v / g.nx, i = v % g.nx;
    const int ib = i + kDXI[d], rb = r + kDETA[d];
    const size_t A = (size_t)r * g.nx + i, B = (size_t)rb * g.nx + ib;
    const double m1 = 0.5 * (g.beta1[A] + g.beta1[B]), m2 = 0.5 * (g.beta2[A] + g.beta2[B]);
    const double nm = sqrt(m1 * m1 + m2 * m2);
    if (!(nm > 0.0)) {
        atomicOr(status, kErrGeom);
        w[(size_t)fam * cap_order + pos] = 0.0;
        return;
    }
    const double vx = fam == 0 ? m1 / nm : m2 / nm, vy = fam == 0 ? m2 / nm : -m1 / nm;
    const double nxo = (double)kDETA[d], nyo = (double)(-kDXI[d]);
    const double len = (d & 1) ? g.hy : g.hx;
    w[(size_t)fam * cap_order + pos] = -(nxo * vx + nyo * vy) * len;
}

// the running inflow measure in walk order, one warp per family: cb[pos] is
// the measure before edge pos and cb[n] the total, the sum taken edge by edge
// in walk order.  The lanes fetch the next 32 weights while every lane runs
// the same serial sum over the current 32; lane t keeps the value before
// edge base + t for a coalesced store.
__global__ void k_bnd_scan(const int* norder, const double* w, int cap_order, double* cb)
{
    const int fam = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (fam > 1) return;
    const int n = *norder;
    const double* wf = w + (size_t)fam * cap_order;
    double* cbf = cb + (size_t)fam * (cap_order + 1);
    double cum = 0.0;
    double wn = lane < n ? wf[lane] : 0.0;
    for (int base = 0; base < n; base += 32) {
        const double wl = wn;
        wn = base + 32 + lane < n ? wf[base + 32 + lane] : 0.0;
        double mine = 0.0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const double wv = __shfl_sync(0xffffffffu, wl, j);
            if (lane == j) mine = cum;
            if (wv > 0.0) cum += wv;  // past n the weights are 0
        }
        if (base + lane < n) cbf[base + lane] = mine;
    }
    if (lane == 0) cbf[n] = cum;
}

// seed level of index k, (k + 1/2) h_s
__device__ __forceinline__ double seed_level(const GridView& g, long long k)
{
    return (k + 0.5) * g.hs;
}

// The first seed index of every edge, kf[pos] (kf[n] = seeds in all): the
// smallest k >= 0 whose level is not below cb[pos].  Raising k edge by edge
// while the level is below cum + w gives the same k: the measure never
// decreases and the level rises with k, so each edge's k is the smallest one
// for the measure after it.
__global__ void k_bnd_kidx(GridView g, const int* norder, const double* cb, int cap_order,
                           long long* kf, int* status)
{
    const int n = *norder;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n < 0 || t >= 2LL * (n + 1)) return;
    const int fam = (int)(t / (n + 1)), pos = (int)(t % (n + 1));
    const double X = cb[(size_t)fam * (cap_order + 1) + pos];
    long long k = 0;
    if (!isfinite(X)) {
        atomicOr(status, kErrGeom);
    } else if (seed_level(g, 0) < X) {
        const double e = ceil(X / g.hs - 0.5);
        k = e > 0.0 ? (long long)e : 0;
        for (int it = 0; it < 8 && k > 0 && seed_level(g, k - 1) >= X; ++it) k--;
        for (int it = 0; it < 8 && seed_level(g, k) < X; ++it) k++;
        if ((k > 0 && seed_level(g, k - 1) >= X) || seed_level(g, k) < X) atomicOr(status, kErrGeom);
    }
    kf[(size_t)fam * (cap_order + 1) + pos] = k;
}

// the seeds (index coordinates) of every edge, in parallel ([fam][pos])
__global__ void k_bnd_emit(GridView g, const int* order, const int* norder, const int* info,
                           const double* w, const long long* kf, const double* cb, int cap_order,
                           double* sx_all, double* sy_all, int cap, int* nseeds, int* status)
{
    const int n = *norder;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n <= 0 || t >= 2LL * n) return;
    const int fam = (int)(t / n), pos = (int)(t % n);
    const long long* kff = kf + (size_t)fam * (cap_order + 1);
    const double wv = w[(size_t)fam * cap_order + pos];
    const double cum = cb[(size_t)fam * (cap_order + 1) + pos];
    const int in = info[order[pos]];
    const int d = in & 3, v = in >> 2, r = v / g.nx, i = v % g.nx;
    for (long long k = kff[pos]; k < kff[pos + 1]; ++k) {
        if (k >= cap) break;
        const double phi = ((k + 0.5) * g.hs - cum) / wv;
        sx_all[(size_t)fam * cap + k] = i + phi * kDXI[d];
        sy_all[(size_t)fam * cap + k] = r + phi * kDETA[d];
    }
    if (pos == 0) {
        const long long ns = kff[n];
        if (ns > cap) atomicOr(status, kErrCapacity);
        nseeds[fam] = (int)(ns > cap ? cap : ns);
    }
}

// Accepted RK4 points of the traced curves, kept so that the node placement
// reads them instead of integrating again.  Points of one curve sit in chunks
// of kPoolChunk taken from a shared pool; a curve whose points do not fit
// (pool exhausted, more than kPoolMaxChunks chunks) is re-traced instead,
// which gives the same points.
constexpr int kPoolChunk = 512;
constexpr int kPoolMaxChunks = 512;
struct PointPool {
    double2* pts;        // [n_chunks * kPoolChunk]
    int* tab;            // [seed slot * kPoolMaxChunks + c]: pool chunk of the curve's chunk c
    int* stored;         // [seed slot]: 1 when every accepted point of the curve is in the pool
    unsigned int* next;  // chunks handed out
    unsigned int n_chunks;
};

// seed t of the combined launch: family 0 takes t < nseeds[0], family 1 the
// rest; per-seed arrays of family f live at offset f*cap
__device__ __forceinline__ bool seed_of(const int* nseeds, int cap, int t, int* fam, int* s)
{
    if (t < nseeds[0]) {
        *fam = 0;
        *s = t;
        return true;
    }
    if (t < nseeds[0] + nseeds[1]) {
        *fam = 1;
        *s = cap + (t - nseeds[0]);
        return true;
    }
    return false;
}

// Two warps trace each 32 curves: lane l of warp 0 and lane l of warp 1 work
// on the same curve.  Warp 0 computes the x halves of every RK4 stage (beta1
// at the stage point, the x component of the direction, the x coordinate),
// warp 1 the y halves, and the two trade what the other half needs through
// shared memory: the cell index and local coordinate, then the field value,
// at every stage, and the new point with its interior-test halves at every
// step.  An FP64 warp instruction holds its sub-partition's FP64 unit for
// about 64 cycles, and the two warps run on different sub-partitions, so a
// stage's chain is about a third shorter.  Every value comes from the same
// operations as in rk4, direction and interior_point, so the points are the
// same.  All lanes of both warps reach every barrier: a lane whose curve is
// done computes on its last point and drops the result.
struct Trade {
    double a, b;
    int i, j, k;
};

// publish this warp's values for the lane, read the other warp's; the buffer
// alternates, so that one barrier per trade suffices
__device__ __forceinline__ Trade trade(Trade (*buf)[2][32], int& nb, int w, int lane, Trade mine)
{
    buf[nb][w][lane] = mine;
    __syncthreads();
    Trade o = buf[nb][w ^ 1][lane];
    nb ^= 1;
    return o;
}

// this warp's direction component at the stage point whose own coordinate is
// c (the other warp holds the other coordinate); bad is raised where |beta|
// is not positive (direction's failure)
__device__ __forceinline__ double half_direction(const GridView& g, int w, int fam, double c,
                                                 Trade (*buf)[2][32], int& nb, int lane, bool& bad)
{
    const int lim = w == 0 ? g.nx - 2 : g.ny - 2;
    int q = __double2int_rd(c);
    if (q > lim) q = lim;
    if (q < 0) q = 0;
    const double l = c - q, a = 1.0 - l;
    const Trade t = trade(buf, nb, w, lane, Trade{l, a, q, 0, 0});
    const int i = w == 0 ? q : t.i, r = w == 0 ? t.i : q;
    const double lx = w == 0 ? l : t.a, ax = w == 0 ? a : t.b;
    const double ly = w == 0 ? t.a : l, ay = w == 0 ? t.b : a;
    const double w11 = ay * ax, w12 = ay * lx, w21 = ly * ax, w22 = ly * lx;
    const double* p = (w == 0 ? g.beta1 : g.beta2) + ((size_t)r * g.nx + i);
    const double v = w11 * p[0] + w12 * p[1] + w21 * p[g.nx] + w22 * p[g.nx + 1];
    const Trade u = trade(buf, nb, w, lane, Trade{v, 0.0, 0, 0, 0});
    const double b1 = w == 0 ? v : u.a, b2 = w == 0 ? u.a : v;
    const double nrm = sqrt(b1 * b1 + b2 * b2);
    if (!(nrm > 0.0)) bad = true;
    const double num = w == 0 ? (fam == 0 ? b1 : b2) : (fam == 0 ? b2 : -b1);
    return num / nrm;
}

// this warp's coordinate after one classical RK4 step of step component st
__device__ __forceinline__ double half_rk4(const GridView& g, int w, int fam, double c, double st,
                                           Trade (*buf)[2][32], int& nb, int lane, bool& bad)
{
    const double k1 = half_direction(g, w, fam, c, buf, nb, lane, bad);
    const double k2 = half_direction(g, w, fam, c + 0.5 * st * k1, buf, nb, lane, bad);
    const double k3 = half_direction(g, w, fam, c + 0.5 * st * k2, buf, nb, lane, bad);
    const double k4 = half_direction(g, w, fam, c + st * k3, buf, nb, lane, bad);
    return c + st / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
}

// Trace every curve: number of full RK4 steps M, length L and exit point; the
// accepted points P_1 .. P_M go to the pool when it has room.  A curve takes
// full RK4 steps while their end points lie inside Omega_h, then locates its
// exit within the first step that leaves by kBisectIters bisections of that
// step, then takes the partial step found.  Each lane runs this as a state
// machine, and every pass of the loop makes one RK4 step per lane (a full
// step, a bisection trial or the final partial step): the same steps with the
// same arguments as tracing each curve alone.  A lane that bisected on a
// branch of its own would add its 61 steps to the warp's time, once for every
// curve of the warp.
__global__ void __launch_bounds__(64) k_trace_count(GridView g, int cap, const double* sx0,
                                                    const double* sy0, const int* nseeds, int* M,
                                                    double* L, double* XE, double* YE,
                                                    long long* cn, int* status, PointPool pool)
{
    __shared__ Trade buf[2][2][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int fam = 0, s = 0;
    const bool have = seed_of(nseeds, cap, blockIdx.x * 32 + lane, &fam, &s);
    const double ds = g.hs / kTraceStepsPerH;
    const double sx = ds / g.hx, sy = ds / g.hy;  // the step in index units
    const double stp = w == 0 ? sx : sy;          // this warp's component
    const double lim = w == 0 ? (double)g.nx : (double)g.ny;
    const double cap_len = 10.0 * 2.0 * (g.W + g.H);
    double X = have ? sx0[s] : 0.0, Y = have ? sy0[s] : 0.0;
    double lo = 0.0, hi = 1.0, xe = 0.0, ye = 0.0;
    long long npts = 0;
    enum { kStep, kBisect, kFinal, kDone, kFailed };
    int phase = have ? kStep : kDone, it = 0, nb = 0;
    bool keep = w == 0 && have && pool.n_chunks > 0;  // warp 0 writes the pool
    int* tab = pool.tab + (size_t)s * kPoolMaxChunks;
    int chunk = -1;
    if (keep) pool.stored[s] = 0;
    while (__any_sync(0xffffffffu, phase < kDone)) {
        const bool act = phase < kDone;
        const double mid = 0.5 * (lo + hi);
        double st = stp;
        if (phase == kBisect) st = mid * stp;
        else if (phase == kFinal) st = lo * stp;
        if (act && phase == kStep) npts++;
        bool bad = false;
        const double c = half_rk4(g, w, fam, w == 0 ? X : Y, st, buf, nb, lane, bad);
        // this half of interior_point(snap(Xn), snap(Yn)), then the other's
        const double cs = snap(c);
        const bool ok = isfinite(cs) && !(cs < -1.0) && !(cs > lim);
        const double fc = floor(cs);
        const int q1 = ok ? (int)fc : 0, q0 = ok && cs == fc ? q1 - 1 : q1;
        const Trade t = trade(buf, nb, w, lane, Trade{c, 0.0, q0, q1, ok ? 1 : 0});
        if (!act) continue;
        const double Xn = w == 0 ? c : t.a, Yn = w == 0 ? t.a : c;
        if (bad) {
            phase = kFailed;
            continue;
        }
        if (phase == kFinal) {
            xe = Xn;
            ye = Yn;
            phase = kDone;
            continue;
        }
        bool inside = ok && t.k;
        if (inside) {
            const int i0 = w == 0 ? q0 : t.i, i1 = w == 0 ? q1 : t.j;
            const int r0 = w == 0 ? t.i : q0, r1 = w == 0 ? t.j : q1;
            for (int r = r0; r <= r1 && inside; ++r)
                for (int i = i0; i <= i1; ++i)
                    if (!cell_on(g, i, r)) {
                        inside = false;
                        break;
                    }
        }
        if (phase == kStep) {
            if (inside) {
                X = Xn;
                Y = Yn;
                if (keep) {  // P_q, q = npts, at pool index q - 1 of the curve
                    long long i = npts - 1;
                    int c2 = (int)(i / kPoolChunk), o = (int)(i % kPoolChunk);
                    if (o == 0) {
                        unsigned int got = c2 < kPoolMaxChunks ? atomicAdd(pool.next, 1u) : pool.n_chunks;
                        if (got >= pool.n_chunks) keep = false;
                        else {
                            chunk = (int)got;
                            tab[c2] = chunk;
                        }
                    }
                    if (keep) pool.pts[(size_t)chunk * kPoolChunk + o] = make_double2(X, Y);
                }
                if (npts * ds > cap_len) phase = kFailed;
            } else {
                phase = kBisect;
                lo = 0.0;
                hi = 1.0;
                it = 0;
            }
        } else {  // kBisect
            if (inside) lo = mid;
            else hi = mid;
            if (++it == kBisectIters) {
                if (lo > 0.0) {
                    phase = kFinal;
                } else {
                    xe = X;
                    ye = Y;
                    phase = kDone;
                }
            }
        }
    }
    if (!have || w != 0) return;
    int m = 0;
    double len = 0.0;
    if (phase == kDone) {
        m = (int)(npts - 1);
        len = (npts - 1) * ds + lo * ds;
        if (keep) pool.stored[s] = 1;
    } else {
        atomicOr(status, kErrGeom);
        xe = sx0[s];
        ye = sy0[s];
    }
    M[s] = m;
    L[s] = len;
    XE[s] = xe;
    YE[s] = ye;
    cn[s] = elements_for(g, len) + 1;
}

// re-trace the M RK4 steps and place n+1 nodes uniformly in arc length
struct FillOut {
    int* off;
    double* h;
    double* xs;
    double* es;
};

// place n+1 nodes uniformly in arc length on the polyline P_0 .. P_M, exit
// point: node j at s_j = j L / n lies on the RK4 step q = floor(s_j / ds)
// (linear between its end points).  One warp per curve; a curve whose points
// are not in the pool is re-traced by lane 0.
__global__ void k_trace_fill(GridView g, int cap, const double* sx, const double* sy,
                             const int* nseeds, const int* M, const double* L, const double* XE,
                             const double* YE, const long long* noff, FillOut o0, FillOut o1,
                             PointPool pool)
{
    int fam, s;
    const int lane = threadIdx.x & 31;
    if (!seed_of(nseeds, cap, (blockIdx.x * blockDim.x + threadIdx.x) >> 5, &fam, &s)) return;
    const FillOut& o = fam == 0 ? o0 : o1;
    int* off = o.off;
    double* h = o.h;
    double* xs = o.xs;
    double* es = o.es;
    int li = fam == 0 ? s : s - cap;  // curve index inside its family
    double ds = g.hs / kTraceStepsPerH;
    double len = L[s];
    int m = M[s];
    int n = elements_for(g, len);
    int base = (int)noff[s];
    const double xe = XE[s], ye = YE[s];
    if (lane == 0) {
        off[li] = base;
        h[li] = len / n;
    }
    if (pool.n_chunks > 0 && pool.stored[s]) {
        const int* tab = pool.tab + (size_t)s * kPoolMaxChunks;
        for (int j = lane; j <= n; j += 32) {
            double X, Y;
            if (j == n) {
                X = xe;
                Y = ye;
            } else {
                double sj = j * (len / n);
                int q = (int)floor(sj / ds);
                if (q > m) q = m;
                double Xa, Ya, Xb, Yb;
                if (q == 0) {
                    Xa = sx[s];
                    Ya = sy[s];
                } else {
                    double2 a = pool.pts[(size_t)tab[(q - 1) / kPoolChunk] * kPoolChunk + (q - 1) % kPoolChunk];
                    Xa = a.x;
                    Ya = a.y;
                }
                if (q < m) {
                    double2 b = pool.pts[(size_t)tab[q / kPoolChunk] * kPoolChunk + q % kPoolChunk];
                    Xb = b.x;
                    Yb = b.y;
                } else {
                    Xb = xe;
                    Yb = ye;
                }
                double s0 = q * ds, s1 = (q < m) ? (q + 1) * ds : len;
                double fr = (s1 > s0) ? (sj - s0) / (s1 - s0) : 0.0;
                X = Xa + fr * (Xb - Xa);
                Y = Ya + fr * (Yb - Ya);
            }
            xs[base + j] = snap(X);
            es[base + j] = snap(Y);
        }
        return;
    }
    if (lane != 0) return;
    // (Xa, Ya) = P_q, (Xb, Yb) = P_{q+1}; P_0 is the seed, P_{m+1} the exit point
    int q = 0;
    double Xa = sx[s], Ya = sy[s], Xb, Yb;
    const double stx = ds / g.hx, sty = ds / g.hy;  // the step in index units
    if (m > 0) rk4(g, fam, Xa, Ya, stx, sty, &Xb, &Yb);
    else {
        Xb = xe;
        Yb = ye;
    }
    for (int j = 0; j <= n; ++j) {
        double X, Y;
        if (j == n) {
            X = xe;
            Y = ye;
        } else {
            double sj = j * (len / n);
            int qj = (int)floor(sj / ds);
            if (qj > m) qj = m;
            while (q < qj) {
                q++;
                Xa = Xb;
                Ya = Yb;
                if (q < m) rk4(g, fam, Xa, Ya, stx, sty, &Xb, &Yb);
                else {
                    Xb = xe;
                    Yb = ye;
                }
            }
            double s0 = q * ds, s1 = (q < m) ? (q + 1) * ds : len;
            double fr = (s1 > s0) ? (sj - s0) / (s1 - s0) : 0.0;
            X = Xa + fr * (Xb - Xa);
            Y = Ya + fr * (Yb - Ya);
        }
        xs[base + j] = snap(X);
        es[base + j] = snap(Y);
    }
}

// --------------------------------------------------------- node data

__global__ void k_node_data(GridView g, int n_nodes, const double* xs, const double* es,
                            double* bnorm, double* fval)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_nodes) return;
    double b1 = bilin(g, g.beta1, xs[k], es[k]);
    double b2 = bilin(g, g.beta2, xs[k], es[k]);
    bnorm[k] = sqrt(b1 * b1 + b2 * b2);
    fval[k] = bilin(g, g.f, xs[k], es[k]);
}

__global__ void k_line_of_node(int n_lines, const int* off, int* lon, int* maxlen)
{
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_lines) return;
    int a = off[l], b = off[l + 1];
    for (int k = a; k < b; ++k) lon[k] = l;
    atomicMax(maxlen, b - a);
}

// ------------------------------------------------- curve -> grid crossings
// §6: every grid line is cut into segments by the grid nodes; each segment
// keeps its crossing with the smallest and with the largest coordinate (ties:
// smaller curve-segment index, then smaller t).  Built with atomics in three
// rounds (position, segment index, t); the result does not depend on order.

struct Slots {
    unsigned long long* minpos;  // bits of a non-negative double
    unsigned long long* maxpos;
    int* ming;
    int* maxg;
    unsigned long long* mint;
    unsigned long long* maxt;
};

__device__ __forceinline__ unsigned long long dbits(double v)
{
    return (unsigned long long)__double_as_longlong(v + 0.0);
}

template <int ROUND>
__device__ void record(const Slots& S, size_t base, int nseg, double pos, int g, double t)
{
    double fp = floor(pos);
    int e0 = (int)fp, e1 = (int)fp;
    if (pos == fp) e0 = (int)fp - 1;
    unsigned long long pb = dbits(pos), tb = dbits(t);
    for (int e = e0; e <= e1; ++e) {
        if (e < 0 || e >= nseg) continue;
        size_t s = base + e;
        if (ROUND == 0) {
            atomicMin(&S.minpos[s], pb);
            atomicMax(&S.maxpos[s], pb);
        } else if (ROUND == 1) {
            if (S.minpos[s] == pb) atomicMin(&S.ming[s], g);
            if (S.maxpos[s] == pb) atomicMin(&S.maxg[s], g);
        } else {
            if (S.minpos[s] == pb && S.ming[s] == g) atomicMin(&S.mint[s], tb);
            if (S.maxpos[s] == pb && S.maxg[s] == g) atomicMin(&S.maxt[s], tb);
        }
    }
}

template <int ROUND>
__global__ void k_cross(GridView g, int n_nodes, const int* lon, const double* xs,
                        const double* es, Slots rows, Slots cols)
{
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi + 1 >= n_nodes || lon[gi] != lon[gi + 1]) return;
    int nx = g.nx, ny = g.ny;
    double xa = xs[gi], xb = xs[gi + 1], ea = es[gi], eb = es[gi + 1];
    if (ea == eb) {
        if (ea == floor(ea) && ea >= 0 && ea <= ny - 1) {
            size_t base = (size_t)ea * (nx - 1);
            record<ROUND>(rows, base, nx - 1, xa, gi, 0.0);
            record<ROUND>(rows, base, nx - 1, xb, gi, 1.0);
        }
    } else {
        double lo = ea < eb ? ea : eb, hi = ea < eb ? eb : ea;
        for (long long r = (long long)ceil(lo); r <= (long long)floor(hi); ++r) {
            if (r < 0 || r > ny - 1) continue;
            double t, pos;
            if (r == ea) {
                t = 0.0;
                pos = xa;
            } else if (r == eb) {
                t = 1.0;
                pos = xb;
            } else {
                t = (r - ea) / (eb - ea);
                pos = snap(xa + t * (xb - xa));
            }
            record<ROUND>(rows, (size_t)r * (nx - 1), nx - 1, pos, gi, t);
        }
    }
    if (xa == xb) {
        if (xa == floor(xa) && xa >= 0 && xa <= nx - 1) {
            size_t base = (size_t)xa * (ny - 1);
            record<ROUND>(cols, base, ny - 1, ea, gi, 0.0);
            record<ROUND>(cols, base, ny - 1, eb, gi, 1.0);
        }
    } else {
        double lo = xa < xb ? xa : xb, hi = xa < xb ? xb : xa;
        for (long long i = (long long)ceil(lo); i <= (long long)floor(hi); ++i) {
            if (i < 0 || i > nx - 1) continue;
            double t, pos;
            if (i == xa) {
                t = 0.0;
                pos = ea;
            } else if (i == xb) {
                t = 1.0;
                pos = eb;
            } else {
                t = (i - xa) / (xb - xa);
                pos = snap(ea + t * (eb - ea));
            }
            record<ROUND>(cols, (size_t)i * (ny - 1), ny - 1, pos, gi, t);
        }
    }
}

__global__ void k_slots_init(Slots s, size_t n)
{
    size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    s.minpos[k] = ~0ull;
    s.maxpos[k] = 0ull;
    s.ming[k] = 0x7fffffff;
    s.maxg[k] = 0x7fffffff;
    s.mint[k] = ~0ull;
    s.maxt[k] = ~0ull;
}

// nearest crossing on each side of every interior node (a non-interior grid
// node met first stands for the boundary, value 0)
__global__ void k_node_desc(GridView g, Slots rows, Slots cols, int* cg, double* ct,
                            double* cw, double* cpos, int* status)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int nx = g.nx, ny = g.ny;
    if (k >= (long long)nx * ny) return;
    int r = (int)(k / nx), i = (int)(k % nx);
    if (g.ntype[k] != kInterior) {
        for (int q = 0; q < 4; ++q) {
            cg[4 * k + q] = -2;
            ct[4 * k + q] = 0.0;
            cpos[4 * k + q] = 0.0;
        }
        cw[2 * k] = cw[2 * k + 1] = 0.0;
        return;
    }
    int G[4];
    double T[4], Pp[4];
    size_t rb = (size_t)r * (nx - 1), cb = (size_t)i * (ny - 1);
    for (int e = i - 1;; --e) {
        if (rows.minpos[rb + e] != ~0ull) {
            G[0] = rows.maxg[rb + e];
            T[0] = __longlong_as_double((long long)rows.maxt[rb + e]);
            Pp[0] = __longlong_as_double((long long)rows.maxpos[rb + e]);
            break;
        }
        if (g.ntype[(size_t)r * nx + e] != kInterior) {
            G[0] = -1;
            T[0] = 0.0;
            Pp[0] = e;
            break;
        }
    }
    for (int e = i;; ++e) {
        if (rows.minpos[rb + e] != ~0ull) {
            G[1] = rows.ming[rb + e];
            T[1] = __longlong_as_double((long long)rows.mint[rb + e]);
            Pp[1] = __longlong_as_double((long long)rows.minpos[rb + e]);
            break;
        }
        if (g.ntype[(size_t)r * nx + e + 1] != kInterior) {
            G[1] = -1;
            T[1] = 0.0;
            Pp[1] = e + 1;
            break;
        }
    }
    for (int e = r - 1;; --e) {
        if (cols.minpos[cb + e] != ~0ull) {
            G[2] = cols.maxg[cb + e];
            T[2] = __longlong_as_double((long long)cols.maxt[cb + e]);
            Pp[2] = __longlong_as_double((long long)cols.maxpos[cb + e]);
            break;
        }
        if (g.ntype[(size_t)e * nx + i] != kInterior) {
            G[2] = -1;
            T[2] = 0.0;
            Pp[2] = e;
            break;
        }
    }
    for (int e = r;; ++e) {
        if (cols.minpos[cb + e] != ~0ull) {
            G[3] = cols.ming[cb + e];
            T[3] = __longlong_as_double((long long)cols.mint[cb + e]);
            Pp[3] = __longlong_as_double((long long)cols.minpos[cb + e]);
            break;
        }
        if (g.ntype[(size_t)(e + 1) * nx + i] != kInterior) {
            G[3] = -1;
            T[3] = 0.0;
            Pp[3] = e + 1;
            break;
        }
    }
    for (int q = 0; q < 4; ++q) {
        cg[4 * k + q] = G[q];
        ct[4 * k + q] = T[q];
        cpos[4 * k + q] = Pp[q];
    }
    // no curve of the family on either grid line through the node before the
    // boundary: the family does not cover the node (§3, §6)
    if (G[0] == -1 && G[1] == -1 && G[2] == -1 && G[3] == -1) atomicOr(status, kErrUncovered);
    cw[2 * k] = (Pp[1] == Pp[0]) ? 0.0 : (i - Pp[0]) / (Pp[1] - Pp[0]);
    cw[2 * k + 1] = (Pp[3] == Pp[2]) ? 0.0 : (r - Pp[2]) / (Pp[3] - Pp[2]);
}

// longest-first order of the curves (work balance of the sweep kernels):
// counting sort by length, ties by curve index
__global__ void k_len_hist(int n_lines, const int* off, int* hist)
{
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_lines) return;
    atomicAdd(&hist[off[l + 1] - off[l]], 1);
}
__global__ void k_len_order(int n_lines, const int* off, const long long* start, int maxlen,
                            int* order)
{
    // one thread per length bucket keeps index order inside the bucket
    int len = blockIdx.x * blockDim.x + threadIdx.x;
    if (len > maxlen) return;
    long long pos = start[maxlen - len];
    for (int l = 0; l < n_lines; ++l)
        if (off[l + 1] - off[l] == len) order[pos++] = l;
}

__global__ void k_reverse_hist(const int* hist, long long* rev, int maxlen)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > maxlen) return;
    rev[k] = hist[maxlen - k];
}

// setup temporaries: stream-ordered from the library's pool, freed in stream
// order when the guard goes out of scope
// ------------------------------------ direct transfer between the families
// The crossings of every target curve (family tf) with the polylines of the
// source family (1 - tf), for carrying values between the families without
// the grid (the improvement the paper's conclusions propose).  Source segments
// are listed per grid cell (every cell their bounding box covers).  One thread
// per target element tests every segment listed in the cells its bounding box
// covers and takes a crossing in the cell that holds it, so that each counts
// once.  Each element keeps its crossings of smallest and largest position
// along the curve and the smallest ones on its two end nodes; every target
// node then takes its nearest crossing on each side, as a search over all
// crossings of its curve would.

__device__ __forceinline__ int cell_clamp(double v, int n)
{
    int c = (int)floor(v);
    return c < 0 ? 0 : (c > n - 1 ? n - 1 : c);
}

// source segments per grid cell: counts
__global__ void k_xseg_count(int n_nodes, const int* lon, const double* xs, const double* es, int ncx,
                             int ncy, long long* cnt)
{
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi + 1 >= n_nodes || lon[gi] != lon[gi + 1]) return;
    const int i0 = cell_clamp(fmin(xs[gi], xs[gi + 1]), ncx), i1 = cell_clamp(fmax(xs[gi], xs[gi + 1]), ncx);
    const int r0 = cell_clamp(fmin(es[gi], es[gi + 1]), ncy), r1 = cell_clamp(fmax(es[gi], es[gi + 1]), ncy);
    for (int r = r0; r <= r1; ++r)
        for (int i = i0; i <= i1; ++i)
            atomicAdd(reinterpret_cast<unsigned long long*>(&cnt[(size_t)r * ncx + i]), 1ull);
}

// source segments per grid cell: the lists (order within a cell does not
// matter: the choices below are keyed)
__global__ void k_xseg_fill(int n_nodes, const int* lon, const double* xs, const double* es, int ncx,
                            int ncy, long long* cursor, int* list)
{
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi + 1 >= n_nodes || lon[gi] != lon[gi + 1]) return;
    const int i0 = cell_clamp(fmin(xs[gi], xs[gi + 1]), ncx), i1 = cell_clamp(fmax(xs[gi], xs[gi + 1]), ncx);
    const int r0 = cell_clamp(fmin(es[gi], es[gi + 1]), ncy), r1 = cell_clamp(fmax(es[gi], es[gi + 1]), ncy);
    for (int r = r0; r <= r1; ++r)
        for (int i = i0; i <= i1; ++i) {
            long long q = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&cursor[(size_t)r * ncx + i]), 1ull);
            list[q] = gi;
        }
}

// per target element: crossings of smallest / largest position (ties: smaller
// source segment, then smaller t), and the smallest ones exactly on its first
// and last node
struct XSlots {
    double* mnpos;
    int* mng;
    double* mnt;
    double* mxpos;
    int* mxg;
    double* mxt;
    int* stg;  // on the element's first node (-1: none)
    double* stt;
    int* eng;  // on its last node
    double* ent;
};

__device__ __forceinline__ bool key_lt(double pa, int ga, double ta, double pb, int gb, double tb, bool max)
{
    if (pa != pb) return max ? pa > pb : pa < pb;
    if (ga != gb) return ga < gb;
    return ta < tb;
}

// crossing of A-B and C-D (index coordinates): A + a (B - A) = C + b (D - C)
// with 0 <= a, b <= 1 (parallel segments give none)
__device__ __forceinline__ bool seg_cross(double ax, double ay, double bx, double by, double cx, double cy,
                                          double dx, double dy, double* a, double* b)
{
    const double ex = bx - ax, ey = by - ay, fx = dx - cx, fy = dy - cy;
    const double det = ex * fy - ey * fx;
    if (det == 0.0) return false;
    const double gx = cx - ax, gy = cy - ay;
    const double aa = (gx * fy - gy * fx) / det;
    const double bb = (gx * ey - gy * ex) / det;
    if (!(aa >= 0.0 && aa <= 1.0 && bb >= 0.0 && bb <= 1.0)) return false;
    *a = aa;
    *b = bb;
    return true;
}

__global__ void k_xquery(int nt, const int* lont, const int* offt, const double* xt, const double* et,
                         const double* xs, const double* es, int ncx, int ncy, const long long* start,
                         const int* list, XSlots S)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e + 1 >= nt || lont[e] != lont[e + 1]) return;
    const int el = e - offt[lont[e]];  // element index along its curve
    const double ax = xt[e], ay = et[e], bx = xt[e + 1], by = et[e + 1];
    double mnp = 0, mnt_ = 0, mxp = 0, mxt_ = 0, stt_ = 0, ent_ = 0;
    int mng_ = -1, mxg_ = -1, stg_ = -1, eng_ = -1;
    const int i0 = cell_clamp(fmin(ax, bx), ncx), i1 = cell_clamp(fmax(ax, bx), ncx);
    const int r0 = cell_clamp(fmin(ay, by), ncy), r1 = cell_clamp(fmax(ay, by), ncy);
    for (int r = r0; r <= r1; ++r)
        for (int i = i0; i <= i1; ++i) {
            const size_t c = (size_t)r * ncx + i;
            for (long long q = start[c]; q < start[c + 1]; ++q) {
                const int sg = list[q];
                double a, b;
                if (!seg_cross(ax, ay, bx, by, xs[sg], es[sg], xs[sg + 1], es[sg + 1], &a, &b)) continue;
                const double px = ax + a * (bx - ax), py = ay + a * (by - ay);
                if (cell_clamp(px, ncx) != i || cell_clamp(py, ncy) != r) continue;  // counted in its own cell
                const double pos = el + a;
                if (mng_ < 0 || key_lt(pos, sg, b, mnp, mng_, mnt_, false)) {
                    mnp = pos;
                    mng_ = sg;
                    mnt_ = b;
                }
                if (mxg_ < 0 || key_lt(pos, sg, b, mxp, mxg_, mxt_, true)) {
                    mxp = pos;
                    mxg_ = sg;
                    mxt_ = b;
                }
                if (pos == (double)el && (stg_ < 0 || sg < stg_ || (sg == stg_ && b < stt_))) {
                    stg_ = sg;
                    stt_ = b;
                }
                if (pos == (double)(el + 1) && (eng_ < 0 || sg < eng_ || (sg == eng_ && b < ent_))) {
                    eng_ = sg;
                    ent_ = b;
                }
            }
        }
    S.mnpos[e] = mnp;
    S.mng[e] = mng_;
    S.mnt[e] = mnt_;
    S.mxpos[e] = mxp;
    S.mxg[e] = mxg_;
    S.mxt[e] = mxt_;
    S.stg[e] = stg_;
    S.stt[e] = stt_;
    S.eng[e] = eng_;
    S.ent[e] = ent_;
}

// the crossings held by element e of a curve whose first node is base and
// which has n elements, as the oracle's per-element record: its own, the
// crossing on node e found by element e - 1, the one on node e + 1 found by
// element e + 1; the one of smallest (max = false) or largest key
__device__ __forceinline__ bool xslot_pick(const XSlots& S, int base, int n, int e, bool max, double* pos,
                                           int* sg, double* t)
{
    bool ok = false;
    const int ge = base + e;
    if (S.mng[ge] >= 0) {
        ok = true;
        *pos = max ? S.mxpos[ge] : S.mnpos[ge];
        *sg = max ? S.mxg[ge] : S.mng[ge];
        *t = max ? S.mxt[ge] : S.mnt[ge];
    }
    if (e >= 1 && S.eng[ge - 1] >= 0) {  // on node e, from element e - 1
        const double p = (double)e;
        if (!ok || key_lt(p, S.eng[ge - 1], S.ent[ge - 1], *pos, *sg, *t, max)) {
            ok = true;
            *pos = p;
            *sg = S.eng[ge - 1];
            *t = S.ent[ge - 1];
        }
    }
    if (e + 1 < n && S.stg[ge + 1] >= 0) {  // on node e + 1, from element e + 1
        const double p = (double)(e + 1);
        if (!ok || key_lt(p, S.stg[ge + 1], S.stt[ge + 1], *pos, *sg, *t, max)) {
            ok = true;
            *pos = p;
            *sg = S.stg[ge + 1];
            *t = S.stt[ge + 1];
        }
    }
    return ok;
}

// per target node: the nearest crossing on each side along its curve (the
// curve's end, value 0, where a side has none) and the 4 coefficients of the
// transfer: value = c0 v[g0] + c1 v[g0 + 1] + c2 v[g1] + c3 v[g1 + 1]
__global__ void k_xnodes(int nt, const int* lont, const int* offt, XSlots S, int* xseg, double* xtt,
                         double* xpos, int* xg, double* xc)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const int l = lont[k], base = offt[l], n = offt[l + 1] - 1 - base, kk = k - base;
    if (kk == 0 || kk == n || n < 2) {  // end node: u = 0
        for (int q = 0; q < 2; ++q) {
            xseg[2 * k + q] = -2;
            xtt[2 * k + q] = 0.0;
            xpos[2 * k + q] = 0.0;
            xg[2 * k + q] = 0;
        }
        for (int q = 0; q < 4; ++q) xc[4 * k + q] = 0.0;
        return;
    }
    double pl = 0.0, tl = 0.0, pr = (double)n, tr = 0.0;
    int gl = -1, gr = -1;
    for (int e = kk - 1; e >= 0; --e)
        if (xslot_pick(S, base, n, e, true, &pl, &gl, &tl)) break;
    for (int e = kk; e < n; ++e)
        if (xslot_pick(S, base, n, e, false, &pr, &gr, &tr)) break;
    if (gl < 0) {
        pl = 0.0;
        tl = 0.0;
    }
    if (gr < 0) {
        pr = (double)n;
        tr = 0.0;
    }
    xseg[2 * k] = gl;
    xtt[2 * k] = tl;
    xpos[2 * k] = pl;
    xseg[2 * k + 1] = gr;
    xtt[2 * k + 1] = tr;
    xpos[2 * k + 1] = pr;
    const double w = (pr == pl) ? 0.0 : ((double)kk - pl) / (pr - pl);
    xg[2 * k] = gl >= 0 ? gl : 0;
    xg[2 * k + 1] = gr >= 0 ? gr : 0;
    xc[4 * k] = gl >= 0 ? (1.0 - w) * (1.0 - tl) : 0.0;
    xc[4 * k + 1] = gl >= 0 ? (1.0 - w) * tl : 0.0;
    xc[4 * k + 2] = gr >= 0 ? w * (1.0 - tr) : 0.0;
    xc[4 * k + 3] = gr >= 0 ? w * tr : 0.0;
}

struct TmpGuard {
    std::vector<void*> v;
    cudaStream_t st = nullptr;
    ~TmpGuard()
    {
        for (void* q : v) cudaFreeAsync(q, st);
    }
};

template <typename T>
adr_status alloc_tmp(TmpGuard& tg, T** p, size_t n)
{
    void* q = nullptr;
    cudaError_t e = pool_alloc(&q, n * sizeof(T) + 16, tg.st);
    if (e != cudaSuccess) {
        set_error(std::string("device allocation failed: ") + cudaGetErrorString(e));
        return ADR_ENOMEM;
    }
    tg.v.push_back(q);
    *p = static_cast<T*>(q);
    return ADR_OK;
}

#define TRY(x)                         \
    do {                               \
        adr_status _s = (x);           \
        if (_s != ADR_OK) return _s;   \
    } while (0)

adr_status finish_family(Problem* p, int fam, TmpGuard& tg, int* status_d)
{
    Family& F = p->fam[fam];
    cudaStream_t st = p->stream;
    const GridView& g = p->gv;
    int N = p->N;
    TRY(dev_alloc(p, &F.bnorm, F.n_nodes));
    TRY(dev_alloc(p, &F.fval, F.n_nodes));
    TRY(dev_alloc(p, &F.v, F.n_nodes + 1));
    TRY(dev_alloc(p, &F.cg, 4 * (size_t)N));
    TRY(dev_alloc(p, &F.ct, 4 * (size_t)N));
    TRY(dev_alloc(p, &F.cw, 2 * (size_t)N));
    TRY(dev_alloc(p, &F.cpos, 4 * (size_t)N));
    TRY(dev_alloc(p, &F.order, F.n_lines + 1));
    k_node_data<<<blocks_for(F.n_nodes), kThreads, 0, st>>>(g, F.n_nodes, F.xi, F.eta, F.bnorm,
                                                          F.fval);
    int* lon;
    int* maxlen;
    TRY(alloc_tmp(tg, &lon, F.n_nodes + 1));
    TRY(alloc_tmp(tg, &maxlen, 1));
    ADR_CUDA_TRY(cudaMemsetAsync(maxlen, 0, sizeof(int), st));
    k_line_of_node<<<blocks_for(F.n_lines), kThreads, 0, st>>>(F.n_lines, F.off, lon, maxlen);
    ADR_CUDA_TRY(cudaMemcpyAsync(&F.max_nodes, maxlen, sizeof(int), cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    // curves sorted longest first
    int ml = F.max_nodes;
    int* hist;
    long long *rev, *start;
    TRY(alloc_tmp(tg, &hist, ml + 1));
    TRY(alloc_tmp(tg, &rev, ml + 2));
    TRY(alloc_tmp(tg, &start, ml + 2));
    ADR_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int) * (ml + 1), st));
    k_len_hist<<<blocks_for(F.n_lines), kThreads, 0, st>>>(F.n_lines, F.off, hist);
    k_reverse_hist<<<blocks_for(ml + 1), kThreads, 0, st>>>(hist, rev, ml);
    k_scan<<<1, 1024, 0, st>>>(rev, start, ml + 1);
    k_len_order<<<blocks_for(ml + 1, 64), 64, 0, st>>>(F.n_lines, F.off, start, ml, F.order);
    // crossing slots
    size_t nr = (size_t)p->grid.ny * (p->grid.nx - 1), nc = (size_t)p->grid.nx * (p->grid.ny - 1);
    Slots R, C;
    TRY(alloc_tmp(tg, &R.minpos, nr));
    TRY(alloc_tmp(tg, &R.maxpos, nr));
    TRY(alloc_tmp(tg, &R.ming, nr));
    TRY(alloc_tmp(tg, &R.maxg, nr));
    TRY(alloc_tmp(tg, &R.mint, nr));
    TRY(alloc_tmp(tg, &R.maxt, nr));
    TRY(alloc_tmp(tg, &C.minpos, nc));
    TRY(alloc_tmp(tg, &C.maxpos, nc));
    TRY(alloc_tmp(tg, &C.ming, nc));
    TRY(alloc_tmp(tg, &C.maxg, nc));
    TRY(alloc_tmp(tg, &C.mint, nc));
    TRY(alloc_tmp(tg, &C.maxt, nc));
    k_slots_init<<<blocks_for((long long)nr), kThreads, 0, st>>>(R, nr);
    k_slots_init<<<blocks_for((long long)nc), kThreads, 0, st>>>(C, nc);
    int nb = blocks_for(F.n_nodes);
    k_cross<0><<<nb, kThreads, 0, st>>>(g, F.n_nodes, lon, F.xi, F.eta, R, C);
    k_cross<1><<<nb, kThreads, 0, st>>>(g, F.n_nodes, lon, F.xi, F.eta, R, C);
    k_cross<2><<<nb, kThreads, 0, st>>>(g, F.n_nodes, lon, F.xi, F.eta, R, C);
    k_node_desc<<<blocks_for(N), kThreads, 0, st>>>(g, R, C, F.cg, F.ct, F.cw, F.cpos, status_d);
    TRY(dev_alloc(p, &F.mg, 4 * (size_t)N));
    TRY(dev_alloc(p, &F.mc, 8 * (size_t)N));
    TRY(launch_map_coef(p, fam));
    ADR_CUDA_TRY(cudaGetLastError());
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    return ADR_OK;
}

adr_status build_straight(Problem* p, int fam, int first, TmpGuard& tg)
{
    Family& F = p->fam[fam];
    cudaStream_t st = p->stream;
    LineParams* P;
    TRY(alloc_tmp(tg, &P, 1));
    k_line_params<<<1, 1, 0, st>>>(p->gv, fam, first, P);
    LineParams hp;
    ADR_CUDA_TRY(cudaMemcpyAsync(&hp, P, sizeof hp, cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    long long nk = hp.kmax - hp.kmin + 1;
    if (nk < 1) {
        set_error("no curve crosses the domain");
        return ADR_EGEOM;
    }
    long long *cl, *cn, *ol, *on;
    TRY(alloc_tmp(tg, &cl, nk));
    TRY(alloc_tmp(tg, &cn, nk));
    TRY(alloc_tmp(tg, &ol, nk + 1));
    TRY(alloc_tmp(tg, &on, nk + 1));
    k_straight_count<<<blocks_for(nk, 64), 64, 0, st>>>(p->gv, P, cl, cn);
    k_scan<<<1, 1024, 0, st>>>(cl, ol, nk);
    k_scan<<<1, 1024, 0, st>>>(cn, on, nk);
    long long tl = 0, tn = 0;
    ADR_CUDA_TRY(cudaMemcpyAsync(&tl, ol + nk, sizeof tl, cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaMemcpyAsync(&tn, on + nk, sizeof tn, cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    if (tl < 1 || tn > 0x7fffffffLL) {
        set_error(tl < 1 ? "no curve inside the domain" : "too many curve nodes");
        return tl < 1 ? ADR_EGEOM : ADR_EINVAL;
    }
    F.n_lines = (int)tl;
    F.n_nodes = (int)tn;
    TRY(dev_alloc(p, &F.off, F.n_lines + 1));
    TRY(dev_alloc(p, &F.h, F.n_lines));
    TRY(dev_alloc(p, &F.xi, F.n_nodes));
    TRY(dev_alloc(p, &F.eta, F.n_nodes));
    k_straight_fill<<<blocks_for(nk, 64), 64, 0, st>>>(p->gv, P, ol, on, F.off, F.h, F.xi, F.eta);
    int nn = F.n_nodes;
    ADR_CUDA_TRY(cudaMemcpyAsync(F.off + F.n_lines, &nn, sizeof(int), cudaMemcpyHostToDevice, st));
    ADR_CUDA_TRY(cudaGetLastError());
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    return ADR_OK;
}

adr_status build_curved_both(Problem* p, int* status_d, TmpGuard& tg)
{
    cudaStream_t st = p->stream;
    const GridView& g = p->gv;
    int nx = p->grid.nx, ny = p->grid.ny;
    int* cnt;  // [0] boundary edges, [1..2] seeds per family
    TRY(alloc_tmp(tg, &cnt, 3));
    ADR_CUDA_TRY(cudaMemsetAsync(cnt, 0, 3 * sizeof(int), st));
    k_count_bedges<<<blocks_for((long long)nx * ny), kThreads, 0, st>>>(g, cnt);
    // loop-start candidates in (row, column) order
    long long *rc, *rs;
    TRY(alloc_tmp(tg, &rc, ny));
    TRY(alloc_tmp(tg, &rs, ny + 1));
    k_row_cand_count<<<blocks_for(ny, 64), 64, 0, st>>>(g, rc);
    k_scan<<<1, 1024, 0, st>>>(rc, rs, ny);
    int nbe = 0;
    long long ncand = 0;
    ADR_CUDA_TRY(cudaMemcpyAsync(&nbe, cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaMemcpyAsync(&ncand, rs + ny, sizeof ncand, cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    int* cand;
    TRY(alloc_tmp(tg, &cand, ncand + 1));
    k_row_cand_fill<<<blocks_for(ny, 64), 64, 0, st>>>(g, rs, cand);
    double hmax = p->gv.hx > p->gv.hy ? p->gv.hx : p->gv.hy;
    int cap = (int)(nbe * ceil(hmax / p->gv.hs)) + 4;
    const long long ne = (long long)ny * (nx - 1) + (long long)nx * (ny - 1);
    int *info, *succ, *cid, *order, *norder;
    TRY(alloc_tmp(tg, &info, ne));
    TRY(alloc_tmp(tg, &succ, ne));
    TRY(alloc_tmp(tg, &cid, ne));
    TRY(alloc_tmp(tg, &order, (size_t)nbe + 1));
    TRY(alloc_tmp(tg, &norder, 1));
    ADR_CUDA_TRY(cudaMemsetAsync(cid, 0xff, ne * sizeof(int), st));
    // compact boundary edges: info, global id, successor, visited flag
    int *cinfo, *cedge, *csucc, *nbc;
    uint8_t* cvis;
    TRY(alloc_tmp(tg, &cinfo, (size_t)nbe + 1));
    TRY(alloc_tmp(tg, &cedge, (size_t)nbe + 1));
    TRY(alloc_tmp(tg, &csucc, (size_t)nbe + 1));
    TRY(alloc_tmp(tg, &cvis, (size_t)nbe + 1));
    TRY(alloc_tmp(tg, &nbc, 1));
    ADR_CUDA_TRY(cudaMemsetAsync(cvis, 0, (size_t)nbe + 1, st));
    ADR_CUDA_TRY(cudaMemsetAsync(nbc, 0, sizeof(int), st));
    const int cap_order = nbe + 1;
    double *w, *cb;
    long long* kf;
    TRY(alloc_tmp(tg, &w, 2 * (size_t)cap_order));
    TRY(alloc_tmp(tg, &cb, 2 * ((size_t)cap_order + 1)));
    TRY(alloc_tmp(tg, &kf, 2 * ((size_t)cap_order + 1)));
    double *sx, *sy;
    TRY(alloc_tmp(tg, &sx, 2 * (size_t)cap));
    TRY(alloc_tmp(tg, &sy, 2 * (size_t)cap));
    // the walk keeps successors and flags (5 bytes an edge) in shared memory
    // when they fit in a block's opt-in limit
    int dev = 0, smem_max = 0;
    ADR_CUDA_TRY(cudaGetDevice(&dev));
    ADR_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t walk_smem = (size_t)nbe * 5 + 16;
    const int use_smem = nbe > 0 && walk_smem <= (size_t)smem_max;
    if (use_smem)
        ADR_CUDA_TRY(cudaFuncSetAttribute(k_bnd_walk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)walk_smem));
    k_bnd_succ<<<blocks_for(ne), kThreads, 0, st>>>(g, info, succ);
    k_bnd_compact<<<blocks_for(ne), kThreads, 0, st>>>(ne, info, cid, cinfo, cedge, nbc,
                                                             nbe + 1);
    k_bnd_csucc<<<blocks_for((long long)nbe + 1), kThreads, 0, st>>>(nbc, cedge, succ, cid, csucc,
                                                                      nbe + 1);
    k_bnd_walk<<<1, 1024, use_smem ? walk_smem : 0, st>>>(cand, ncand, cid, nbc, csucc, cvis,
                                                          use_smem, nbe, nbe, order, norder);
    k_bnd_weight<<<blocks_for(2LL * nbe), kThreads, 0, st>>>(g, order, norder, cinfo, w, cap_order,
                                                           status_d);
    k_bnd_scan<<<1, 64, 0, st>>>(norder, w, cap_order, cb);
    k_bnd_kidx<<<blocks_for(2LL * (nbe + 2)), kThreads, 0, st>>>(g, norder, cb, cap_order, kf,
                                                               status_d);
    k_bnd_emit<<<blocks_for(2LL * nbe), kThreads, 0, st>>>(g, order, norder, cinfo, w, kf, cb,
                                                         cap_order, sx, sy, cap, cnt + 1, status_d);
    int ns[2] = {0, 0};
    ADR_CUDA_TRY(cudaMemcpyAsync(ns, cnt + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    if (ns[0] < 1 || ns[1] < 1) {
        set_error("no inflow boundary for a curve family");
        return ADR_EGEOM;
    }
    int* M;
    double *L, *XE, *YE;
    long long *cn, *on;
    size_t n2 = 2 * (size_t)cap;
    TRY(alloc_tmp(tg, &M, n2));
    TRY(alloc_tmp(tg, &L, n2));
    TRY(alloc_tmp(tg, &XE, n2));
    TRY(alloc_tmp(tg, &YE, n2));
    TRY(alloc_tmp(tg, &cn, n2));
    TRY(alloc_tmp(tg, &on, n2 + 2));
    int tot = ns[0] + ns[1];
    // point pool: about kTraceStepsPerH^2 accepted points per hs^2 of the
    // domain in each family, with room to spare and one partial chunk per
    // curve; without room (or memory) the node placement re-traces
    PointPool pool{};
    {
        double area = (double)(nx - 1) * (ny - 1) * p->gv.hx * p->gv.hy;
        double est = 2.5 * kTraceStepsPerH * area / (p->gv.hs * p->gv.hs) + (double)tot * kPoolChunk;
        double chunks = ceil(est / kPoolChunk);
        const double max_chunks = (double)(3ull << 30) / (sizeof(double2) * kPoolChunk);
        if (chunks > max_chunks) chunks = max_chunks;
        pool.n_chunks = (unsigned int)chunks;
        void* q = nullptr;
        if (cudaMalloc(&q, (size_t)pool.n_chunks * kPoolChunk * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();  // no pool: every curve is re-traced
            pool.n_chunks = 0;
        } else {
            tg.v.push_back(q);
            pool.pts = static_cast<double2*>(q);
            TRY(alloc_tmp(tg, &pool.tab, n2 * kPoolMaxChunks));
            TRY(alloc_tmp(tg, &pool.stored, n2));
            TRY(alloc_tmp(tg, &pool.next, 1));
            ADR_CUDA_TRY(cudaMemsetAsync(pool.next, 0, sizeof(unsigned int), st));
        }
    }
    // 32 curves per block of two warps: the per-curve traces are serial chains
    k_trace_count<<<blocks_for(tot, 32), 64, 0, st>>>(g, cap, sx, sy, cnt + 1, M, L, XE, YE, cn,
                                                      status_d, pool);
    k_scan<<<1, 1024, 0, st>>>(cn, on, ns[0]);
    k_scan<<<1, 1024, 0, st>>>(cn + cap, on + cap, ns[1]);
    long long tn[2] = {0, 0};
    ADR_CUDA_TRY(cudaMemcpyAsync(&tn[0], on + ns[0], sizeof(long long), cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaMemcpyAsync(&tn[1], on + cap + ns[1], sizeof(long long), cudaMemcpyDeviceToHost,
                                 st));
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    FillOut fo[2];
    for (int fam = 0; fam < 2; ++fam) {
        if (tn[fam] > 0x7fffffffLL) {
            set_error("too many curve nodes");
            return ADR_EINVAL;
        }
        Family& F = p->fam[fam];
        F.n_lines = ns[fam];
        F.n_nodes = (int)tn[fam];
        TRY(dev_alloc(p, &F.off, F.n_lines + 1));
        TRY(dev_alloc(p, &F.h, F.n_lines));
        TRY(dev_alloc(p, &F.xi, F.n_nodes));
        TRY(dev_alloc(p, &F.eta, F.n_nodes));
        fo[fam] = {F.off, F.h, F.xi, F.eta};
    }
    k_trace_fill<<<blocks_for(32LL * tot, 128), 128, 0, st>>>(g, cap, sx, sy, cnt + 1, M, L, XE, YE,
                                                               on, fo[0], fo[1], pool);
    for (int fam = 0; fam < 2; ++fam) {
        int nn = p->fam[fam].n_nodes;
        ADR_CUDA_TRY(cudaMemcpyAsync(p->fam[fam].off + p->fam[fam].n_lines, &nn, sizeof(int),
                                     cudaMemcpyHostToDevice, st));
        ADR_CUDA_TRY(cudaStreamSynchronize(st));
    }
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

}  // namespace

// crossing tables of the direct transfer, both directions (opts.transfer = 1)
adr_status build_transfer(Problem* p)
{
    cudaStream_t st = p->stream;
    TmpGuard tg;
    tg.st = st;
    const int ncx = p->grid.nx - 1, ncy = p->grid.ny - 1;
    const size_t ncell = (size_t)ncx * ncy;
    int* lon[2];
    for (int f = 0; f < 2; ++f) {
        Family& F = p->fam[f];
        int* maxlen;
        TRY(alloc_tmp(tg, &lon[f], F.n_nodes + 1));
        TRY(alloc_tmp(tg, &maxlen, 1));
        ADR_CUDA_TRY(cudaMemsetAsync(maxlen, 0, sizeof(int), st));
        k_line_of_node<<<blocks_for(F.n_lines), kThreads, 0, st>>>(F.n_lines, F.off, lon[f], maxlen);
    }
    for (int tf = 0; tf < 2; ++tf) {
        Family& T = p->fam[tf];
        const Family& S = p->fam[1 - tf];
        long long *cnt, *start;
        TRY(alloc_tmp(tg, &cnt, ncell + 1));
        TRY(alloc_tmp(tg, &start, ncell + 1));
        ADR_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(long long) * (ncell + 1), st));
        k_xseg_count<<<blocks_for(S.n_nodes), kThreads, 0, st>>>(S.n_nodes, lon[1 - tf], S.xi, S.eta, ncx,
                                                               ncy, cnt);
        {
            const long long nb = ((long long)ncell + 1023) / 1024;
            long long *bsum, *boff;
            TRY(alloc_tmp(tg, &bsum, (size_t)nb + 1));
            TRY(alloc_tmp(tg, &boff, (size_t)nb + 1));
            k_scan_blocks<<<(unsigned)nb, 1024, 0, st>>>(cnt, start, (long long)ncell, bsum);
            k_scan<<<1, 1024, 0, st>>>(bsum, boff, nb);
            k_scan_add<<<(unsigned)nb, 1024, 0, st>>>(start, (long long)ncell, boff);
            ADR_CUDA_TRY(cudaMemcpyAsync(start + ncell, boff + nb, sizeof(long long), cudaMemcpyDeviceToDevice,
                                         st));
        }
        long long total = 0;
        ADR_CUDA_TRY(cudaMemcpyAsync(&total, start + ncell, sizeof total, cudaMemcpyDeviceToHost, st));
        ADR_CUDA_TRY(cudaStreamSynchronize(st));
        int* list;
        TRY(alloc_tmp(tg, &list, (size_t)total + 1));
        ADR_CUDA_TRY(cudaMemcpyAsync(cnt, start, sizeof(long long) * ncell, cudaMemcpyDeviceToDevice, st));
        k_xseg_fill<<<blocks_for(S.n_nodes), kThreads, 0, st>>>(S.n_nodes, lon[1 - tf], S.xi, S.eta, ncx, ncy,
                                                              cnt, list);
        XSlots X;
        const size_t nt = (size_t)T.n_nodes + 1;
        TRY(alloc_tmp(tg, &X.mnpos, nt));
        TRY(alloc_tmp(tg, &X.mng, nt));
        TRY(alloc_tmp(tg, &X.mnt, nt));
        TRY(alloc_tmp(tg, &X.mxpos, nt));
        TRY(alloc_tmp(tg, &X.mxg, nt));
        TRY(alloc_tmp(tg, &X.mxt, nt));
        TRY(alloc_tmp(tg, &X.stg, nt));
        TRY(alloc_tmp(tg, &X.stt, nt));
        TRY(alloc_tmp(tg, &X.eng, nt));
        TRY(alloc_tmp(tg, &X.ent, nt));
        k_xquery<<<blocks_for(T.n_nodes), kThreads, 0, st>>>(T.n_nodes, lon[tf], T.off, T.xi, T.eta, S.xi,
                                                           S.eta, ncx, ncy, start, list, X);
        TRY(dev_alloc(p, &T.xseg, 2 * nt));
        TRY(dev_alloc(p, &T.xtt, 2 * nt));
        TRY(dev_alloc(p, &T.xpos, 2 * nt));
        TRY(dev_alloc(p, &T.xg, 2 * nt));
        TRY(dev_alloc(p, &T.xc, 4 * nt));
        k_xnodes<<<blocks_for(T.n_nodes), kThreads, 0, st>>>(T.n_nodes, lon[tf], T.off, X, T.xseg, T.xtt,
                                                           T.xpos, T.xg, T.xc);
        ADR_CUDA_TRY(cudaGetLastError());
        ADR_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return ADR_OK;
}

adr_status build_geometry(Problem* p, const uint8_t* mask)
{
    cudaStream_t st = p->stream;
    int nx = p->grid.nx, ny = p->grid.ny;
    size_t N = (size_t)nx * ny, NC = (size_t)(nx - 1) * (ny - 1);
    TmpGuard tg;
    tg.st = st;
    TRY(dev_alloc(p, &p->cell, NC));
    TRY(dev_alloc(p, &p->ntype, N));
    k_cells<<<blocks_for((long long)NC), kThreads, 0, st>>>(mask, nx, ny, p->cell);
    GridView& g = p->gv;
    g.nx = nx;
    g.ny = ny;
    g.W = p->grid.x1 - p->grid.x0;
    g.H = p->grid.y1 - p->grid.y0;
    g.hx = g.W / (nx - 1);
    g.hy = g.H / (ny - 1);
    g.hs = g.hx < g.hy ? g.hx : g.hy;
    g.cell = p->cell;
    g.ntype = p->ntype;
    g.beta1 = p->beta1;
    g.beta2 = p->beta2;
    g.f = p->f;
    int* info;  // [0] interior count, [1] status, [2] first node, [3] nonconst
    unsigned long long* bmax;
    TRY(alloc_tmp(tg, &info, 4));
    TRY(alloc_tmp(tg, &bmax, 1));
    int init[4] = {0, 0, 0x7fffffff, 0};
    ADR_CUDA_TRY(cudaMemcpyAsync(info, init, sizeof init, cudaMemcpyHostToDevice, st));
    ADR_CUDA_TRY(cudaMemsetAsync(bmax, 0, sizeof(unsigned long long), st));
    k_ntype<<<blocks_for((long long)N), kThreads, 0, st>>>(g, p->ntype, info);
    int hinfo[4];
    ADR_CUDA_TRY(cudaMemcpyAsync(hinfo, info, sizeof hinfo, cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    if (hinfo[2] == 0x7fffffff) {
        set_error("empty domain: no grid cell has four corners in the mask");
        return ADR_EINVAL;
    }
    int first = hinfo[2];
    p->n_interior = hinfo[0];
    k_fields<<<blocks_for((long long)N), kThreads, 0, st>>>(g, first, info + 1, info + 3, bmax);
    unsigned long long hb = 0;
    ADR_CUDA_TRY(cudaMemcpyAsync(hinfo, info, sizeof hinfo, cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaMemcpyAsync(&hb, bmax, sizeof hb, cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    if (hinfo[1] & kErrInvalid) {
        set_error("beta is zero or data is not finite at a node of the domain");
        return ADR_EINVAL;
    }
    p->const_beta = hinfo[3] == 0;
    double bm;
    long long bits = (long long)hb;
    memcpy(&bm, &bits, sizeof bm);
    p->bmax = bm;
    adr_status s = ADR_OK;
    if (p->const_beta) {
        for (int fam = 0; fam < 2 && s == ADR_OK; ++fam) s = build_straight(p, fam, first, tg);
    } else {
        s = build_curved_both(p, info + 1, tg);
    }
    if (s != ADR_OK) return s;
    ADR_CUDA_TRY(cudaMemcpyAsync(hinfo, info, sizeof hinfo, cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    if (hinfo[1] & kErrGeom) {
        set_error("curve tracing failed (closed integral curve or |beta| = 0 on a curve)");
        return ADR_EGEOM;
    }
    if (hinfo[1] & kErrCapacity) {
        set_error("internal: seed capacity exceeded");
        return ADR_EGEOM;
    }
    for (int fam = 0; fam < 2; ++fam) {
        s = finish_family(p, fam, tg, info + 1);
        if (s != ADR_OK) return s;
    }
    ADR_CUDA_TRY(cudaMemcpyAsync(hinfo, info, sizeof hinfo, cudaMemcpyDeviceToHost, st));
    ADR_CUDA_TRY(cudaStreamSynchronize(st));
    if (hinfo[1] & kErrUncovered) {
        set_error("a curve family leaves an interior node uncovered (stagnation point or "
                  "closed integral curves of beta or gamma)");
        return ADR_EGEOM;
    }
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

}  // namespace adr
