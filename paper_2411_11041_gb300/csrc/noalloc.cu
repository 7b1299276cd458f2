// adr_cross_substep_noalloc: one cross-flow (G family) substep whose work
// space is a fixed array in device memory, for callers that must not
// allocate.  See include/adr.h for the contract.
//
// The scratch below is a file-scope __device__ array: every GPU that loads
// this library holds it (kNoAllocMaxNodes curve nodes x 4 planes of doubles =
// 16 MiB) until the process exits.  Host code cannot use the array's name as a
// device address, so every call looks the address up on the current device
// with cudaGetSymbolAddress (a lookup, no allocation) and passes it to the
// kernels.  Looking it up each time keeps the address right even after a
// context reset has reloaded the module.
#include <cuda_runtime.h>

#include "adr_internal.cuh"

namespace {

constexpr int kNoAllocMaxNodes = 1 << 19;  // curve nodes of the G family

// planes: [0] c', [1] v', [2] r' of the partitioned elimination, [3] curve values
static __device__ __align__(256) double g_noalloc_scratch[4 * (size_t)kNoAllocMaxNodes];

__device__ __forceinline__ double gather_u(const double* __restrict__ u, int nx, int ny, double xi,
                                           double eta)
{
    int i = (int)floor(xi), r = (int)floor(eta);
    i = i > nx - 2 ? nx - 2 : (i < 0 ? 0 : i);
    r = r > ny - 2 ? ny - 2 : (r < 0 ? 0 : r);
    double lx = xi - i, ly = eta - r;
    const double* r0 = u + (size_t)r * nx + i;
    double b = r0[0] + lx * (r0[1] - r0[0]);
    double t = r0[nx] + lx * (r0[nx + 1] - r0[nx]);
    return b + ly * (t - b);
}

// One warp per G curve: (M + theta dt mu K) d = -mu K u on the curve, values
// u + dt d out into the curve-value plane (the same partitioned elimination
// as the library's curve solve, over the scratch planes).
__global__ void k_cross_curves(int nx, int ny, const double* __restrict__ u, int n_lines,
                               int n_nodes, const int* __restrict__ off, const double* __restrict__ hl,
                               const double* __restrict__ xs, const double* __restrict__ es,
                               double mu, double theta, double dt, double* scr)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n_lines) return;
    double* cpS = scr;
    double* vpS = scr + kNoAllocMaxNodes;
    double* rpS = scr + 2 * (size_t)kNoAllocMaxNodes;
    double* v = scr + 3 * (size_t)kNoAllocMaxNodes;
    int base = off[warp], end = off[warp + 1];
    if (base < 0 || end > n_nodes || end - base < 2) {
        // malformed curve: skipped, and the nodes of its range that lie in
        // [0, n_nodes) set to 0, so that no crossing reads an earlier call's value
        const int lo = base < 0 ? 0 : base, hi = end > n_nodes ? n_nodes : end;
        for (int k = lo + lane; k < hi; k += 32) v[k] = 0.0;
        return;
    }
    int n = end - base - 1;
    if (n < 2) {
        if (lane <= n) v[base + lane] = 0.0;
        return;
    }
    const int m = n - 1, c = (m + 31) >> 5, s = lane * c, e = min(m, s + c);
    const bool has = s < m;
    const double h = hl[warp];
    const double Mo = h / 6.0, Md = 2.0 * h / 3.0, Ko = -1.0 / h, Kd = 2.0 / h, td = theta * dt;
    double cpL = 0, vpL = 0, rpL = 0;
    if (has) {
        auto uat = [&](int k) {
            return (k == 0 || k == n) ? 0.0 : gather_u(u, nx, ny, xs[base + k], es[base + k]);
        };
        double u0 = uat(s), u1 = uat(s + 1);
        double cpp = 0, vpp = 0, rpp = 0;
        for (int q = s; q < e; ++q) {
            double u2 = uat(q + 2);
            double r = -(mu * Ko * u0 + mu * Kd * u1 + mu * Ko * u2);
            double A = (q == 0) ? 0.0 : Mo + td * mu * Ko;
            double B = Md + td * mu * Kd;
            double C = (q == m - 1) ? 0.0 : Mo + td * mu * Ko;
            double inv = 1.0 / (q == s ? B : B - A * cpp);
            double cp = C * inv, vp = (q == s ? A : -A * vpp) * inv, rp = (q == s ? r : r - A * rpp) * inv;
            int g = base + q;
            cpS[g] = cp;
            vpS[g] = vp;
            rpS[g] = rp;
            v[g + 1] = u1;
            cpp = cp;
            vpp = vp;
            rpp = rp;
            u0 = u1;
            u1 = u2;
        }
        cpL = cpp;
        vpL = vpp;
        rpL = rpp;
    }
    double rho = 0.0, kap = has ? -1.0 : 0.0, nu = 0.0;
    if (has)
        for (int q = e - 2; q >= s; --q) {
            int g = base + q;
            double cp = cpS[g];
            rho = rpS[g] - cp * rho;
            kap = -cp * kap;
            nu = vpS[g] - cp * nu;
        }
    double rhoN = __shfl_down_sync(0xffffffffu, rho, 1);
    double kapN = __shfl_down_sync(0xffffffffu, kap, 1);
    double nuN = __shfl_down_sync(0xffffffffu, nu, 1);
    if (lane == 31) rhoN = kapN = nuN = 0.0;
    double A = has ? vpL : 0.0, B = has ? 1.0 - cpL * nuN : 1.0;
    double C = has ? -cpL * kapN : 0.0, R = has ? rpL - cpL * rhoN : 0.0;
    for (int d = 1; d < 32; d <<= 1) {
        double Am = __shfl_up_sync(0xffffffffu, A, d), Bm = __shfl_up_sync(0xffffffffu, B, d);
        double Cm = __shfl_up_sync(0xffffffffu, C, d), Rm = __shfl_up_sync(0xffffffffu, R, d);
        double Ap = __shfl_down_sync(0xffffffffu, A, d), Bp = __shfl_down_sync(0xffffffffu, B, d);
        double Cp = __shfl_down_sync(0xffffffffu, C, d), Rp = __shfl_down_sync(0xffffffffu, R, d);
        bool lo = lane >= d, hi = lane + d < 32;
        double k1 = lo ? A / Bm : 0.0, k2 = hi ? C / Bp : 0.0;
        double nA = lo ? -Am * k1 : 0.0, nC = hi ? -Cp * k2 : 0.0;
        B = B - (lo ? Cm * k1 : 0.0) - (hi ? Ap * k2 : 0.0);
        R = R - (lo ? Rm * k1 : 0.0) - (hi ? Rp * k2 : 0.0);
        A = nA;
        C = nC;
    }
    double G = R / B;
    double Gm = __shfl_up_sync(0xffffffffu, G, 1);
    if (lane == 0) Gm = 0.0;
    if (has) {
        double x = G;
        int g = base + e - 1;
        v[g + 1] += dt * x;
        for (int q = e - 2; q >= s; --q) {
            g = base + q;
            x = rpS[g] - cpS[g] * x - vpS[g] * Gm;
            v[g + 1] += dt * x;
        }
    }
    if (lane == 0) {
        v[base] = 0.0;
        v[base + n] = 0.0;
    }
}

// curve values -> grid through the 4 crossings of every node (seg/t/pos as
// reported by adr_get_crossings; seg = -2 marks a non-interior node)
__global__ void k_cross_map(int nx, int ny, int n_nodes, const int* __restrict__ seg,
                            const double* __restrict__ t,
                            const double* __restrict__ pos, const double* __restrict__ v,
                            double* __restrict__ out)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= (long long)nx * ny) return;
    const int* g = seg + 4 * k;
    if (g[0] == -2) {
        out[k] = 0.0;
        return;
    }
    double val[4];
    for (int q = 0; q < 4; ++q) {
        int s = g[q];
        double tq = t[4 * k + q];
        bool ok = s >= 0 && s + 1 < n_nodes;  // boundary crossing or malformed index: 0
        val[q] = ok ? v[s] + tq * (v[s + 1] - v[s]) : 0.0;
    }
    const double* p = pos + 4 * k;
    double i = (double)(k % nx), r = (double)(k / nx);
    double wr = (p[1] == p[0]) ? 0.0 : (i - p[0]) / (p[1] - p[0]);
    double wc = (p[3] == p[2]) ? 0.0 : (r - p[2]) / (p[3] - p[2]);
    double row = val[0] + wr * (val[1] - val[0]);
    double col = val[2] + wc * (val[3] - val[2]);
    out[k] = 0.5 * (row + col);
}

}  // namespace

extern "C" adr_status adr_cross_substep_noalloc(int nx, int ny, double mu, double theta, double dt,
                                                const double* u_in, int n_lines, int n_nodes,
                                                const int* off, const double* h, const double* xi,
                                                const double* eta, const int* seg, const double* t,
                                                const double* pos, double* u_out, void* stream)
{
    if (nx < 3 || ny < 3 || (long long)nx * ny > 0x7fffffffLL || n_lines < 1 || n_nodes < 2 ||
        !u_in || !off || !h || !xi || !eta || !seg || !t || !pos || !u_out || !(mu > 0.0) ||
        !(theta > 0.0 && theta <= 1.0) || !(dt > 0.0)) {
        adr::set_error("adr_cross_substep_noalloc: bad arguments");
        return ADR_EINVAL;
    }
    if (n_nodes > kNoAllocMaxNodes) {
        adr::set_error("adr_cross_substep_noalloc: more than 524288 curve nodes (fixed work space)");
        return ADR_EINVAL;
    }
    // the array's address on the current device (the first call on a device
    // also loads the module there)
    double* scr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&scr), g_noalloc_scratch);
    if (e != cudaSuccess) return adr::cuda_fail(e, "cudaGetSymbolAddress");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_cross_curves<<<(n_lines + 3) / 4, 128, 0, st>>>(nx, ny, u_in, n_lines, n_nodes, off, h, xi,
                                                      eta, mu, theta, dt, scr);
    long long N = (long long)nx * ny;
    k_cross_map<<<(int)((N + 255) / 256), 256, 0, st>>>(nx, ny, n_nodes, seg, t, pos,
                                                       scr + 3 * (size_t)kNoAllocMaxNodes, u_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return adr::cuda_fail(e, "adr_cross_substep_noalloc launch");
    return ADR_OK;
}
