// Anderson extrapolation of the stationary iteration (opts.anderson = m).
//
// The split step is a fixed-point map u -> g = Φ(u).  With f_k = g_k - u_k,
// the next state is u_{k+1} = g_k - Σ_i γ_i (g_{k-i+1} - g_{k-i}) over the
// last min(m, k) differences, γ minimising |f_k - Σ_i γ_i (f_{k-i+1} - f_{k-i})|.
// Any γ leaves the fixed points of Φ in place, so the converged state is the
// plain iteration's; only the number of steps changes.  γ comes from the
// normal equations, whose entries are formed from the raw products
// <f_a, f_b> of the last m + 1 residuals (one new row per step), factored by
// Cholesky with the newest difference first; a column whose pivot falls to
// 1e-12 of its diagonal entry (or below) ends the factorisation and only the
// columns before it are used.
//
// Per step, after the convergence check (all three return once the
// iteration is done):
//   k_aa_dots    f_k = g_k - u_k and g_k into their history slots, the
//                products <f_k, f_{k-j}>, j = 0..min(m, k), as block partials
//   k_aa_solve   one block: the partials summed, the new row of products, the
//                weights c_j of u_{k+1} = Σ_j c_j g_{k-j}
//   k_aa_update  u_{k+1} into the state buffer the next step reads
// The state vector is the grid (transfer through the grid) or the B-curve
// node values (direct transfer); both are 0 where the iteration holds no
// unknown, so the products run over every entry.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "adr_internal.cuh"

namespace adr {

namespace {

constexpr int kAaThreads = 256;
constexpr int kAaMax = 8;

struct AaArgs {
    long long L;              // vector length
    int m;                    // depth
    const IterState* state;
    const double* u_even;     // state by parity of the step index
    const double* u_odd;
    double* out_even;         // g_k (the map's output) by parity of k + 1; u_{k+1} goes there too
    double* out_odd;
    double* fh;               // [(m+1) L] residual history
    double* gh;               // [(m+1) L] map-output history
    AaDev* dev;               // products and weights
    double* partial;          // [(m+1) * blocks]
};

__device__ __forceinline__ int step_index(const IterState* st) { return st->iter - 1; }

// Products of one problem over the elements start, start + stride, ...:
// block partials into a.partial at local block lb.  Every thread loads the
// same M history vectors whether or not the step has that many differences
// yet (a missing one is read from slot k, a valid vector, and left out of
// the sums), so that the loads issue back to back; M >= the problem's depth.
template <int M>
__device__ __forceinline__ void aa_dots_body(const AaArgs& a, long long start, long long stride, int lb)
{
    const int k = step_index(a.state), ns = a.m + 1, mk = k < a.m ? k : a.m;
    const double* __restrict__ u = (k & 1) ? a.u_odd : a.u_even;
    const double* __restrict__ g = ((k + 1) & 1) ? a.out_odd : a.out_even;
    double* __restrict__ fk = a.fh + (size_t)(k % ns) * a.L;
    double* __restrict__ gk = a.gh + (size_t)(k % ns) * a.L;
    const double* fj[M];
#pragma unroll
    for (int j = 1; j <= M; ++j) fj[j - 1] = a.fh + (size_t)((k - (j <= mk ? j : 0)) % ns) * a.L;
    double acc[M + 1];
#pragma unroll
    for (int j = 0; j <= M; ++j) acc[j] = 0.0;
    for (long long q = start; q < a.L; q += stride) {
        double h[M];
#pragma unroll
        for (int j = 0; j < M; ++j) h[j] = __ldg(fj[j] + q);
        const double gv = __ldg(g + q), f = gv - __ldg(u + q);
        fk[q] = f;
        gk[q] = gv;
        acc[0] = fma(f, f, acc[0]);
#pragma unroll
        for (int j = 1; j <= M; ++j) acc[j] = fma(f, h[j - 1], acc[j]);
    }
    __shared__ double red[M + 1][kAaThreads / 32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j <= M; ++j) {
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[j][w] = v;
    }
    __syncthreads();
    if (threadIdx.x <= mk) {
        double t = 0.0;
        for (int q = 0; q < kAaThreads / 32; ++q) t += red[threadIdx.x][q];
        a.partial[(size_t)lb * (kAaMax + 1) + threadIdx.x] = t;
    }
}

template <int M>
__global__ void __launch_bounds__(kAaThreads) k_aa_dots(AaArgs a)
{
    if (a.state->done || a.state->iter < 1) return;
    aa_dots_body<M>(a, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x,
                    blockIdx.x);
}

// the weights of one problem from its block partials (a block of
// 32 (kAaMax + 1) threads)
__device__ void aa_solve_body(const AaArgs& a, int nblocks)
{
    const int k = step_index(a.state), ns = a.m + 1, mk = k < a.m ? k : a.m;
    __shared__ double sums[kAaMax + 1];
    __shared__ double part[kAaMax + 1][32];
    // products: 32 threads per entry, a fixed order
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (j <= mk) {
        double t = 0.0;
        for (int b = lane; b < nblocks; b += 32) t += a.partial[(size_t)b * (kAaMax + 1) + j];
        part[j][lane] = t;
    }
    __syncthreads();
    if (threadIdx.x <= mk) {
        double t = 0.0;
        for (int q = 0; q < 32; ++q) t += part[threadIdx.x][q];
        sums[threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    AaDev& d = *a.dev;
    const int sk = k % ns;
    for (int jj = 0; jj <= mk; ++jj) {
        const int sj = (k - jj) % ns;
        d.R[sk][sj] = sums[jj];
        d.R[sj][sk] = sums[jj];
    }
    // the normal equations of the min(m, k) newest differences
    double A[kAaMax][kAaMax], rhs[kAaMax], Lc[kAaMax][kAaMax], y[kAaMax], gam[kAaMax];
    auto R = [&](int x, int z) { return d.R[x % ns][z % ns]; };
    for (int i = 1; i <= mk; ++i) {
        const int ai = k - i + 1, bi = k - i;
        rhs[i - 1] = R(ai, k) - R(bi, k);
        for (int jj = 1; jj <= i; ++jj) {
            const int aj = k - jj + 1, bj = k - jj;
            A[i - 1][jj - 1] = R(ai, aj) - R(ai, bj) - R(bi, aj) + R(bi, bj);
        }
    }
    int use = mk;
    for (int i = 0; i < mk; ++i) {
        double dd = A[i][i];
        for (int q = 0; q < i; ++q) dd -= Lc[i][q] * Lc[i][q];
        if (!(A[i][i] > 0.0) || !(dd > 1e-12 * A[i][i])) {
            use = i;
            break;
        }
        Lc[i][i] = sqrt(dd);
        for (int r = i + 1; r < mk; ++r) {
            double e = A[r][i];
            for (int q = 0; q < i; ++q) e -= Lc[r][q] * Lc[i][q];
            Lc[r][i] = e / Lc[i][i];
        }
    }
    for (int i = 0; i < use; ++i) {
        double e = rhs[i];
        for (int q = 0; q < i; ++q) e -= Lc[i][q] * y[q];
        y[i] = e / Lc[i][i];
    }
    for (int i = use - 1; i >= 0; --i) {
        double e = y[i];
        for (int q = i + 1; q < use; ++q) e -= Lc[q][i] * gam[q];
        gam[i] = e / Lc[i][i];
    }
    double c[kAaMax + 1];
    for (int q = 0; q <= kAaMax; ++q) c[q] = 0.0;
    c[0] = 1.0;
    for (int i = 1; i <= use; ++i) {
        c[i - 1] -= gam[i - 1];
        c[i] += gam[i - 1];
    }
    for (int q = 0; q <= kAaMax; ++q) d.c[q] = c[q];
    d.used = use;
}

__global__ void k_aa_solve(AaArgs a, int nblocks)
{
    if (a.state->done || a.state->iter < 1) return;
    aa_solve_body(a, nblocks);
}

template <int M>
__device__ __forceinline__ void aa_update_body(const AaArgs& a, long long start, long long stride)
{
    const int k = step_index(a.state), ns = a.m + 1, mk = k < a.m ? k : a.m;
    double* __restrict__ out = ((k + 1) & 1) ? a.out_odd : a.out_even;
    double c[M + 1];
    const double* gj[M + 1];
#pragma unroll
    for (int j = 0; j <= M; ++j) {
        c[j] = j <= mk ? a.dev->c[j] : 0.0;
        gj[j] = a.gh + (size_t)((k - (j <= mk ? j : 0)) % ns) * a.L;
    }
    for (long long q = start; q < a.L; q += stride) {
        double h[M + 1];
#pragma unroll
        for (int j = 0; j <= M; ++j) h[j] = __ldg(gj[j] + q);
        double v = c[0] * h[0];
#pragma unroll
        for (int j = 1; j <= M; ++j) v = fma(c[j], h[j], v);
        out[q] = v;
    }
}

template <int M>
__global__ void __launch_bounds__(kAaThreads) k_aa_update(AaArgs a)
{
    if (a.state->done || a.state->iter < 1) return;
    aa_update_body<M>(a, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------- batches
// One AaArgs per problem (depth 0: no extrapolation); the dots and update
// kernels walk the batch's active map blocks (problem, local block), as the
// batched map does, and the solve kernel takes one block per problem.

template <int M>
__global__ void __launch_bounds__(kAaThreads) k_aa_dots_batch(const AaArgs* __restrict__ table, AaBatchView v)
{
    const int cur = *v.sel;
    const int* list = v.act_blocks[cur];
    const int n_act = v.act_count[cur * 7 + 6];
    for (int ii = blockIdx.x; ii < n_act; ii += gridDim.x) {
        const int bk = list[ii], p = v.blk_prob[bk], lb = v.blk_local[bk];
        const AaArgs& a = table[p];
        if (a.m == 0 || a.state->done || a.state->iter < 1) continue;  // uniform per block
        aa_dots_body<M>(a, (long long)lb * blockDim.x + threadIdx.x, (long long)v.nblk[p] * blockDim.x, lb);
        __syncthreads();  // the reduction's shared arrays are reused
    }
}

__global__ void k_aa_solve_batch(const AaArgs* __restrict__ table, AaBatchView v)
{
    const AaArgs& a = table[blockIdx.x];
    if (a.m == 0 || a.state->done || a.state->iter < 1) return;
    aa_solve_body(a, v.nblk[blockIdx.x]);
}

template <int M>
__global__ void __launch_bounds__(kAaThreads) k_aa_update_batch(const AaArgs* __restrict__ table, AaBatchView v)
{
    const int cur = *v.sel;
    const int* list = v.act_blocks[cur];
    const int n_act = v.act_count[cur * 7 + 6];
    for (int ii = blockIdx.x; ii < n_act; ii += gridDim.x) {
        const int bk = list[ii], p = v.blk_prob[bk], lb = v.blk_local[bk];
        const AaArgs& a = table[p];
        if (a.m == 0 || a.state->done || a.state->iter < 1) continue;
        aa_update_body<M>(a, (long long)lb * blockDim.x + threadIdx.x, (long long)v.nblk[p] * blockDim.x);
    }
}

AaArgs aa_args(Problem* p)
{
    AaArgs a{};
    a.m = p->opts.anderson;
    a.state = p->state;
    if (p->opts.transfer) {
        a.L = p->fam[0].n_nodes;
        a.u_even = p->xu[0];
        a.u_odd = p->xu[1];
        a.out_even = p->xu[0];
        a.out_odd = p->xu[1];
    } else {
        a.L = p->N;
        a.u_even = p->ubuf[0];
        a.u_odd = p->ubuf[1];
        a.out_even = p->ubuf[0];
        a.out_odd = p->ubuf[1];
    }
    a.fh = p->aa_f;
    a.gh = p->aa_g;
    a.dev = p->aa_dev;
    a.partial = p->aa_partial;
    return a;
}

}  // namespace

int aa_blocks(const Problem* p) { return grid_map_blocks(p); }

// the three kernels of one extrapolation step (inside the solve's graph)
adr_status launch_anderson(Problem* p)
{
    const int m = p->opts.anderson;
    if (m <= 0) return ADR_OK;
    const AaArgs a = aa_args(p);
    const int nb = aa_blocks(p);
    cudaStream_t st = p->stream;
    switch (m) {
#define ADR_AA_CASE(M_)                                        \
    case M_:                                                   \
        k_aa_dots<M_><<<nb, kAaThreads, 0, st>>>(a);           \
        k_aa_solve<<<1, 32 * (kAaMax + 1), 0, st>>>(a, nb);    \
        k_aa_update<M_><<<nb, kAaThreads, 0, st>>>(a);         \
        break;
        ADR_AA_CASE(1)
        ADR_AA_CASE(2)
        ADR_AA_CASE(3)
        ADR_AA_CASE(4)
        ADR_AA_CASE(5)
        ADR_AA_CASE(6)
        ADR_AA_CASE(7)
        ADR_AA_CASE(8)
#undef ADR_AA_CASE
    default:
        set_error("internal: Anderson depth out of range");
        return ADR_EINVAL;
    }
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

// the extrapolation's buffers: two histories of m + 1 state vectors
adr_status alloc_anderson(Problem* p)
{
    const int m = p->opts.anderson;
    if (m <= 0) return ADR_OK;
    const size_t L = p->opts.transfer ? (size_t)p->fam[0].n_nodes : (size_t)p->N;
    int keep = p->map_blocks_per_sm;  // partials sized for the largest grid
    p->map_blocks_per_sm = 8;
    const int nb = aa_blocks(p);
    p->map_blocks_per_sm = keep;
    TRY_S(dev_alloc(p, &p->aa_f, (size_t)(m + 1) * L));
    TRY_S(dev_alloc(p, &p->aa_g, (size_t)(m + 1) * L));
    TRY_S(dev_alloc(p, &p->aa_dev, 1));
    TRY_S(dev_alloc(p, &p->aa_partial, (size_t)nb * (kAaMax + 1)));
    ADR_CUDA_TRY(cudaMemsetAsync(p->aa_dev, 0, sizeof(AaDev), p->stream));
    return ADR_OK;
}

}  // namespace adr

namespace adr {

// the batch's table of per-problem arguments (device memory from cudaMalloc,
// freed by the caller with cudaFree); *mmax = the largest depth (0: none)
adr_status anderson_batch_table(Problem* const* ps, int n, void** table, int* mmax)
{
    *table = nullptr;
    *mmax = 0;
    std::vector<AaArgs> t(n);
    for (int i = 0; i < n; ++i) {
        t[i] = aa_args(ps[i]);
        *mmax = std::max(*mmax, t[i].m);
    }
    if (*mmax == 0) return ADR_OK;
    ADR_CUDA_TRY(cudaMalloc(table, sizeof(AaArgs) * n));
    cudaError_t e = cudaMemcpy(*table, t.data(), sizeof(AaArgs) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(*table);
        *table = nullptr;
        return cuda_fail(e, "anderson batch table");
    }
    return ADR_OK;
}

// one extrapolation step of every active problem with a depth (batch graph)
adr_status launch_anderson_batch(const AaBatchView& v, cudaStream_t st)
{
    if (v.mmax <= 0 || !v.table) return ADR_OK;
    const AaArgs* t = static_cast<const AaArgs*>(v.table);
    switch (v.mmax) {
#define ADR_AA_CASE(M_)                                                   \
    case M_:                                                              \
        k_aa_dots_batch<M_><<<v.grid, kAaThreads, 0, st>>>(t, v);         \
        k_aa_solve_batch<<<v.n, 32 * (kAaMax + 1), 0, st>>>(t, v);        \
        k_aa_update_batch<M_><<<v.grid, kAaThreads, 0, st>>>(t, v);       \
        break;
        ADR_AA_CASE(1)
        ADR_AA_CASE(2)
        ADR_AA_CASE(3)
        ADR_AA_CASE(4)
        ADR_AA_CASE(5)
        ADR_AA_CASE(6)
        ADR_AA_CASE(7)
        ADR_AA_CASE(8)
#undef ADR_AA_CASE
    default:
        set_error("internal: Anderson depth out of range");
        return ADR_EINVAL;
    }
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

}  // namespace adr
