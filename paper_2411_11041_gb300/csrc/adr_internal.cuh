// Internal declarations of the GB300 directional-splitting library.
// Device data layout of one problem and the launchers shared by the .cu files.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "adr.h"

namespace adr {

// Geometry readings of §6 (the paper leaves them open):
constexpr double kSnapTol = 1e-9;   // index coordinates this close to an integer are snapped
constexpr double kNodeTol = 1e-9;   // elements per curve: ceil(|L| / h_s - kNodeTol)
constexpr int kTraceStepsPerH = 8;  // RK4 step h_s / 8 along traced curves
constexpr int kBisectIters = 60;    // exit point of a traced curve

enum NodeType : uint8_t { kOutside = 0, kDirichlet = 1, kInterior = 2 };

// Device view of the grid and its nodal data.
struct GridView {
    int nx, ny;
    double hx, hy, hs, W, H;  // spacings, curve spacing h_s = min(hx, hy), box size
    const uint8_t* cell;      // [(ny-1)*(nx-1)] active cells
    const uint8_t* ntype;     // [ny*nx] NodeType
    const double* beta1;      // [ny*nx]
    const double* beta2;
    const double* f;
};

// One curve family in structure-of-arrays form.  Curves are stored back to
// back: curve l owns nodes off[l] .. off[l+1]-1 (both ends on the boundary).
struct Family {
    int n_lines = 0;
    int n_nodes = 0;
    int max_nodes = 0;        // longest curve (nodes)
    int* off = nullptr;       // [n_lines+1]
    int* order = nullptr;     // [n_lines] curves sorted longest first (work order)
    double* h = nullptr;      // [n_lines] element length (physical)
    double* xi = nullptr;     // [n_nodes] index coordinates of the nodes
    double* eta = nullptr;
    double* bnorm = nullptr;  // [n_nodes] |beta| at the nodes
    double* fval = nullptr;   // [n_nodes] f at the nodes
    double* v = nullptr;      // [n_nodes] curve values u + dt d of the current substep
    double* scr = nullptr;    // [3*n_nodes] tridiagonal work space
    // curve -> grid map, per grid node: 4 crossings (row L, row R, col D, col U)
    int* cg = nullptr;        // [4*N] first node of the crossed segment (-1 boundary)
    double* ct = nullptr;     // [4*N] position in that segment
    double* cw = nullptr;     // [2*N] weight of the right / upper crossing
    double* cpos = nullptr;   // [4*N] crossing coordinate (inspection only)
};

// Result of a solve kept on the device: [0] rel update, [1] num, [2] den.
struct IterState {
    int iter;       // split steps done
    int done;       // 1 once converged or capped
    int converged;  // 1 if rel <= tol
    int pad;
    double rel;
};

struct Problem {
    adr_grid grid{};
    adr_opts opts{};
    double mu = 0, sigma = 0;
    cudaStream_t stream = nullptr;
    GridView gv{};
    int N = 0;             // nx*ny
    int n_interior = 0;
    bool const_beta = false;
    double bmax = 0;
    Family fam[2];
    // owned device buffers
    uint8_t* cell = nullptr;
    uint8_t* ntype = nullptr;
    double* beta1 = nullptr;
    double* beta2 = nullptr;
    double* f = nullptr;
    double* ubuf[3] = {nullptr, nullptr, nullptr};  // u_j / u_{j+1} ping-pong and u_{j+1/2}
    double* partial = nullptr;                      // per-block norm partial sums
    int n_partial_blocks = 0;
    IterState* state = nullptr;
    double* fextra = nullptr;                       // [N] extra load (parabolic slices)
    std::vector<void*> owned;
};

// error helpers
void set_error(const std::string& msg);
adr_status cuda_fail(cudaError_t e, const char* what);
#define ADR_CUDA_TRY(call)                                      \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return ::adr::cuda_fail(_e, #call); \
    } while (0)

template <typename T>
adr_status dev_alloc(Problem* p, T** ptr, size_t count)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        set_error(std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
        return ADR_ENOMEM;
    }
    p->owned.push_back(q);
    *ptr = static_cast<T*>(q);
    return ADR_OK;
}

// setup (geometry.cu)
adr_status build_geometry(Problem* p, const uint8_t* mask);

// sweeps (sweep.cu)
adr_status launch_mask_copy(Problem* p, const double* in, double* out);
adr_status launch_state_reset(Problem* p);

}  // namespace adr
