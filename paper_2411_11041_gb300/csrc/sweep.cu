// Directional sweep kernels (the hot path).
//
//  k_line_sweep  one warp per curve: bilinear gather of the grid state onto
//                the curve nodes (§6.1), linear-FEM assembly of the substep
//                system (§6 eqs. SemiDiscrSplit1Dbeta / SemiDiscrSplit1Dgamma),
//                partitioned tridiagonal solve, curve values u + dt d out.
//  k_grid_map    one thread per grid node: curve -> grid interpolation through
//                the nearest crossings on the node's row and column (§6), with
//                the relative-update norms fused in.
//  k_check       one block: convergence test and the CUDA-graph loop condition.
#include <cuda_runtime.h>

#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kLineWarps = 4;  // warps (curves) per block of the line kernel
constexpr int kGridThreads = 256;

struct LineArgs {
    int nx, ny;
    const double* u_even;  // grid state read by the gather: u_even or u_odd by
    const double* u_odd;   // the parity of the step counter
    const double* fextra;  // nullable: extra nodal load (B family only)
    double fx_scale;
    const IterState* state;
    int n_lines;
    const int* order;
    const int* off;
    const double* h;
    const double* xi;
    const double* eta;
    const double* bnorm;
    const double* fval;
    double* v;
    double* scr;  // 3 planes of n_nodes
    int n_nodes;
    double mu, sig, theta, dt;
    int paper_u0;  // 1: steady solve S u0 = F, values out
};

__device__ __forceinline__ double gather(const double* __restrict__ u, int nx, int ny, double xi,
                                         double eta)
{
    int i = (int)floor(xi), r = (int)floor(eta);
    i = i > nx - 2 ? nx - 2 : (i < 0 ? 0 : i);
    r = r > ny - 2 ? ny - 2 : (r < 0 ? 0 : r);
    double lx = xi - i, ly = eta - r;
    const double* r0 = u + (size_t)r * nx + i;
    double p11 = __ldg(r0), p12 = __ldg(r0 + 1), p21 = __ldg(r0 + nx), p22 = __ldg(r0 + nx + 1);
    double b = p11 + lx * (p12 - p11);
    double t = p21 + lx * (p22 - p21);
    return b + ly * (t - b);
}

template <int FAM>
__device__ __forceinline__ void node_vals(const LineArgs& a, const double* __restrict__ u, int base,
                                          int n, int k, double& uk, double& bk, double& fk)
{
    int g = base + k;
    if (k == 0 || k == n || a.paper_u0) uk = 0.0;
    else uk = gather(u, a.nx, a.ny, __ldg(a.xi + g), __ldg(a.eta + g));
    if (FAM == 0) {
        bk = __ldg(a.bnorm + g);
        fk = __ldg(a.fval + g);
        if (a.fextra) fk += a.fx_scale * gather(a.fextra, a.nx, a.ny, __ldg(a.xi + g), __ldg(a.eta + g));
    } else {
        bk = 0.0;
        fk = 0.0;
    }
}

template <int FAM>
__global__ void __launch_bounds__(32 * kLineWarps) k_line_sweep(LineArgs a)
{
    if (a.state && a.state->done) return;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= a.n_lines) return;
    const double* __restrict__ u = (a.state && (a.state->iter & 1)) ? a.u_odd : a.u_even;
    int line = a.order[warp];
    int base = a.off[line];
    int n = a.off[line + 1] - base - 1;  // elements
    double* __restrict__ v = a.v;
    if (n < 2) {
        if (lane <= n) v[base + lane] = 0.0;
        return;
    }
    const int m = n - 1;  // unknowns = rows 0..m-1  (row q <-> node q+1)
    const int c = (m + 31) >> 5;
    const int s = lane * c;
    const int e = min(m, s + c);
    const bool has = s < m;
    const double h = a.h[line];
    const double Mo = h / 6.0, Md = 2.0 * h / 3.0, Ko = -1.0 / h, Kd = 2.0 / h;
    const double td = a.paper_u0 ? 1.0 : a.theta * a.dt;
    const double mw = a.paper_u0 ? 0.0 : 1.0;  // weight of the mass term in the system matrix
    double* __restrict__ cpS = a.scr;
    double* __restrict__ vpS = a.scr + a.n_nodes;
    double* __restrict__ rpS = a.scr + 2 * (size_t)a.n_nodes;

    double cpL = 0, vpL = 0, rpL = 0;  // last row of this lane's chunk
    if (has) {
        double u0, b0, f0, u1, b1, f1, u2, b2, f2;
        node_vals<FAM>(a, u, base, n, s, u0, b0, f0);
        node_vals<FAM>(a, u, base, n, s + 1, u1, b1, f1);
        double cpp = 0, vpp = 0, rpp = 0;
        for (int q = s; q < e; ++q) {
            node_vals<FAM>(a, u, base, n, q + 2, u2, b2, f2);
            double Ssub, Sdia, Ssup, F;
            if (FAM == 0) {
                double Csub = -(b0 * (1.0 / 6.0) + b1 * (1.0 / 3.0));
                double Cdia = (b0 - b2) * (1.0 / 6.0);
                double Csup = b1 * (1.0 / 3.0) + b2 * (1.0 / 6.0);
                Ssub = a.mu * Ko + Csub + a.sig * Mo;
                Sdia = a.mu * Kd + Cdia + a.sig * Md;
                Ssup = a.mu * Ko + Csup + a.sig * Mo;
                F = Mo * (f0 + 4.0 * f1 + f2);
            } else {
                Ssub = a.mu * Ko;
                Sdia = a.mu * Kd;
                Ssup = Ssub;
                F = 0.0;
            }
            double r = F - (Ssub * u0 + Sdia * u1 + Ssup * u2);
            double A = (q == 0) ? 0.0 : mw * Mo + td * Ssub;
            double B = mw * Md + td * Sdia;
            double C = (q == m - 1) ? 0.0 : mw * Mo + td * Ssup;
            double cp, vp, rp;
            if (q == s) {
                double inv = 1.0 / B;
                cp = C * inv;
                vp = A * inv;
                rp = r * inv;
            } else {
                double inv = 1.0 / (B - A * cpp);
                cp = C * inv;
                vp = -A * vpp * inv;
                rp = (r - A * rpp) * inv;
            }
            int g = base + q;
            cpS[g] = cp;
            vpS[g] = vp;
            rpS[g] = rp;
            v[g + 1] = u1;  // state on the curve; the increment is added below
            cpp = cp;
            vpp = vp;
            rpp = rp;
            u0 = u1;
            b0 = b1;
            f0 = f1;
            u1 = u2;
            b1 = b2;
            f1 = f2;
        }
        cpL = cpp;
        vpL = vpp;
        rpL = rpp;
    }
    // upward sweep: x_s = rho - kap * G_j - nu * G_{j-1}
    double rho = 0.0, kap = -1.0, nu = 0.0;
    if (has) {
        for (int q = e - 2; q >= s; --q) {
            int g = base + q;
            double cp = cpS[g];
            rho = rpS[g] - cp * rho;
            kap = -cp * kap;
            nu = vpS[g] - cp * nu;
        }
    } else {
        kap = 0.0;
    }
    double rhoN = __shfl_down_sync(0xffffffffu, rho, 1);
    double kapN = __shfl_down_sync(0xffffffffu, kap, 1);
    double nuN = __shfl_down_sync(0xffffffffu, nu, 1);
    if (lane == 31) rhoN = kapN = nuN = 0.0;
    // reduced system over the chunk ends G_j (one equation per lane)
    double A = has ? vpL : 0.0;
    double B = has ? 1.0 - cpL * nuN : 1.0;
    double C = has ? -cpL * kapN : 0.0;
    double R = has ? rpL - cpL * rhoN : 0.0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        double Am = __shfl_up_sync(0xffffffffu, A, d), Bm = __shfl_up_sync(0xffffffffu, B, d);
        double Cm = __shfl_up_sync(0xffffffffu, C, d), Rm = __shfl_up_sync(0xffffffffu, R, d);
        double Ap = __shfl_down_sync(0xffffffffu, A, d), Bp = __shfl_down_sync(0xffffffffu, B, d);
        double Cp = __shfl_down_sync(0xffffffffu, C, d), Rp = __shfl_down_sync(0xffffffffu, R, d);
        double k1 = lane >= d ? A / Bm : 0.0;
        double k2 = lane + d < 32 ? C / Bp : 0.0;
        double nA = lane >= d ? -Am * k1 : 0.0;
        double nC = lane + d < 32 ? -Cp * k2 : 0.0;
        B = B - (lane >= d ? Cm * k1 : 0.0) - (lane + d < 32 ? Ap * k2 : 0.0);
        R = R - (lane >= d ? Rm * k1 : 0.0) - (lane + d < 32 ? Rp * k2 : 0.0);
        A = nA;
        C = nC;
    }
    double G = R / B;
    double Gm = __shfl_up_sync(0xffffffffu, G, 1);
    if (lane == 0) Gm = 0.0;
    if (has) {
        const double w = a.paper_u0 ? 1.0 : a.dt;
        double x = G;
        int g = base + e - 1;
        v[g + 1] = (a.paper_u0 ? 0.0 : v[g + 1]) + w * x;
        for (int q = e - 2; q >= s; --q) {
            g = base + q;
            x = rpS[g] - cpS[g] * x - vpS[g] * Gm;
            v[g + 1] = (a.paper_u0 ? 0.0 : v[g + 1]) + w * x;
        }
    }
    if (lane == 0) {
        v[base] = 0.0;
        v[base + n] = 0.0;
    }
}

struct GridArgs {
    int nx, ny;
    const uint8_t* ntype;
    const int* cg;
    const double* ct;
    const double* cw;
    const double* v;
    double* out_even;  // written buffer by parity of the step counter (or fixed)
    double* out_odd;
    const double* prev_even;  // previous state for the norms (nullable)
    const double* prev_odd;
    const IterState* state;
    int parity_shift;  // output buffer = parity(iter + shift)
    double* partial;   // [2 * gridDim.x] sums of (u - u_prev)^2 and u^2
};

__device__ __forceinline__ double cross_val(const double* __restrict__ v, int g, double t)
{
    if (g < 0) return 0.0;
    double a = __ldg(v + g), b = __ldg(v + g + 1);
    return a + t * (b - a);
}

template <bool NORMS>
__global__ void __launch_bounds__(kGridThreads) k_grid_map(GridArgs a)
{
    if (a.state && a.state->done) return;
    int it = a.state ? a.state->iter : 0;
    double* __restrict__ out = ((it + a.parity_shift) & 1) ? a.out_odd : a.out_even;
    const double* __restrict__ prev = (it & 1) ? a.prev_odd : a.prev_even;
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long N = (long long)a.nx * a.ny;
    double dd = 0.0, uu = 0.0;
    if (k < N) {
        double val = 0.0;
        if (a.ntype[k] == kInterior) {
            int4 g = *reinterpret_cast<const int4*>(a.cg + 4 * k);
            double2 t01 = *reinterpret_cast<const double2*>(a.ct + 4 * k);
            double2 t23 = *reinterpret_cast<const double2*>(a.ct + 4 * k + 2);
            double2 w = *reinterpret_cast<const double2*>(a.cw + 2 * k);
            double vL = cross_val(a.v, g.x, t01.x), vR = cross_val(a.v, g.y, t01.y);
            double vD = cross_val(a.v, g.z, t23.x), vU = cross_val(a.v, g.w, t23.y);
            double row = vL + w.x * (vR - vL);
            double col = vD + w.y * (vU - vD);
            val = 0.5 * (row + col);
            if (NORMS) {
                double dlt = val - prev[k];
                dd = dlt * dlt;
                uu = val * val;
            }
        }
        out[k] = val;
    }
    if (NORMS) {
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
            a.partial[2 * blockIdx.x] = td;
            a.partial[2 * blockIdx.x + 1] = tu;
        }
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
        int iter = st->iter + 1;
        int conv = tol > 0.0 && rel <= tol;
        st->iter = iter;
        st->rel = rel;
        st->converged = conv;
        st->done = (conv || iter >= max_iter) ? 1 : 0;
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
}

}  // namespace

adr_status launch_line_sweep_ex(Problem* p, int fam, double theta, double dt, double sig,
                                const double* u_even, const double* u_odd, bool use_state,
                                const double* fextra, double fx_scale, int paper_u0)
{
    Family& F = p->fam[fam];
    LineArgs a;
    a.nx = p->grid.nx;
    a.ny = p->grid.ny;
    a.u_even = u_even;
    a.u_odd = u_odd;
    a.fextra = fam == 0 ? fextra : nullptr;
    a.fx_scale = fx_scale;
    a.state = use_state ? p->state : nullptr;
    a.n_lines = F.n_lines;
    a.order = F.order;
    a.off = F.off;
    a.h = F.h;
    a.xi = F.xi;
    a.eta = F.eta;
    a.bnorm = F.bnorm;
    a.fval = F.fval;
    a.v = F.v;
    a.scr = F.scr;
    a.n_nodes = F.n_nodes;
    a.mu = p->mu;
    a.sig = sig;
    a.theta = theta;
    a.dt = dt;
    a.paper_u0 = paper_u0;
    int threads = 32 * kLineWarps;
    int blocks = (F.n_lines + kLineWarps - 1) / kLineWarps;
    if (fam == 0) k_line_sweep<0><<<blocks, threads, 0, p->stream>>>(a);
    else k_line_sweep<1><<<blocks, threads, 0, p->stream>>>(a);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

adr_status launch_grid_map_ex(Problem* p, int fam, double* out_even, double* out_odd,
                              int parity_shift, const double* prev_even, const double* prev_odd,
                              bool use_state, bool norms)
{
    Family& F = p->fam[fam];
    GridArgs a;
    a.nx = p->grid.nx;
    a.ny = p->grid.ny;
    a.ntype = p->ntype;
    a.cg = F.cg;
    a.ct = F.ct;
    a.cw = F.cw;
    a.v = F.v;
    a.out_even = out_even;
    a.out_odd = out_odd;
    a.prev_even = prev_even;
    a.prev_odd = prev_odd;
    a.state = use_state ? p->state : nullptr;
    a.parity_shift = parity_shift;
    a.partial = p->partial;
    int blocks = (int)((p->N + kGridThreads - 1) / kGridThreads);
    if (norms) k_grid_map<true><<<blocks, kGridThreads, 0, p->stream>>>(a);
    else k_grid_map<false><<<blocks, kGridThreads, 0, p->stream>>>(a);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

int grid_map_blocks(const Problem* p) { return (int)((p->N + kGridThreads - 1) / kGridThreads); }

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

}  // namespace adr
