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
constexpr int kTraceStepsPerH = 2;  // RK4 step h_s / 2 along traced curves
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

// Work items of the curve solve: a block of BS threads takes BS/T curves of
// the same block size T.
constexpr int kItemSets = 3;
struct ItemSet {
    int BS = 0;
    int count = 0;
    int* T = nullptr;         // [count] block size of the item's curves
    int* curve = nullptr;     // [count * BS/32] curve indices (-1 empty)
    double* lanec = nullptr;  // [count * (2 log2 BS + 2) * BS] reduced-system constants
    float* lanec32 = nullptr; // the same in FP32 (reduced-precision mode)
};

// A factorisation of family 0's curve systems that is not the active one:
// the family keeps the steady start's (eq. u0stationary) and the iteration's
// side by side, so that switching between them costs no refactorisation.
// When allocated, its kind (paper) is always the other one than the active.
struct FacState {
    bool allocated = false;
    double* fac = nullptr;
    float* fac32 = nullptr;
    double* srow = nullptr;
    double* Fl = nullptr;
    double* lanec[3] = {nullptr, nullptr, nullptr};
    float* lanec32[3] = {nullptr, nullptr, nullptr};
    bool valid = false;
    double td = 0, dt = 0, sig = 0;
    int paper = 0, vform = 0;
    bool load_plain = false;
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
    // per-row data of the curve solve in slot layout (row (t, j) of a curve at
    // soff[curve] + j*T + t, T the curve's block size)
    int n_slots = 0;
    int cmax = 1;             // rows of the longest chunk (a thread's rows) of the family
    int* soff = nullptr;      // [n_lines+1]
    int* ncell = nullptr;     // [n_nodes] the same cells in node order (-1 at the curves' ends;
                              // FP64 through the grid: the separate gather pass)
    double* nw = nullptr;     // [4*n_nodes] the same corner weights in node order
    double* ug = nullptr;     // [n_nodes] the gathered grid state at the nodes
    int* gcell = nullptr;     // [n_slots] bilinear cell r*nx + i of the row's node
    double* gw = nullptr;     // [4 n_slots] bilinear corner weights (1-lx)(1-ly), lx(1-ly),
                              // (1-lx)ly, lx ly
    double* Fl = nullptr;     // [n_slots] load row of the right-hand side (B), times ip
    double* srow = nullptr;   // [3*n_slots] B / [n_slots] G: right-hand-side rows, times ip
    double* kap = nullptr;    // [n_lines] G: diagonal / off-diagonal ratio of the rhs stencil
    double* fac = nullptr;    // [4*n_slots] elimination factors cp, vp, ip, lp
    float* fac32 = nullptr;   // [4*n_slots] the same in FP32 (reduced-precision mode)
    ItemSet iset[3];          // BS = 256, 512, 1024
    int* mg = nullptr;        // [4*N] curve -> grid map: segment of each crossing
    double* mc = nullptr;     // [8*N] combined weights of the map
    // factorisation currently held in fac/lanec (theta dt, dt, sigma, steady flag,
    // right-hand-side form: 1 = FP64 new-value form, 0 = residual form / steady)
    bool prep_valid = false;
    double prep_td = 0, prep_dt = 0, prep_sig = 0;
    int prep_paper = 0, prep_vform = 0;
    bool load_plain = false;  // Fl holds M f without extra load
    FacState alt;             // family 0: the other factorisation (steady start / iteration)
    // curve -> grid map, per grid node: 4 crossings (row L, row R, col D, col U)
    int* cg = nullptr;        // [4*N] first node of the crossed segment (-1 boundary)
    double* ct = nullptr;     // [4*N] position in that segment
    double* cw = nullptr;     // [2*N] weight of the right / upper crossing
    double* cpos = nullptr;   // [4*N] crossing coordinate (inspection only)
    // direct transfer (opts.transfer = 1): per node of this family, the
    // nearest crossing with the other family on each side along its curve
    int* xseg = nullptr;      // [2*n_nodes] crossed segment (-1 the curve's end, -2 an end node)
    double* xtt = nullptr;    // [2*n_nodes] position in that segment
    double* xpos = nullptr;   // [2*n_nodes] position along the curve (element units)
    int* xg = nullptr;        // [2*n_nodes] the two source segments of the node's value
    double* xc = nullptr;     // [4*n_nodes] their coefficients
};

// Result of a solve kept on the device: [0] rel update, [1] num, [2] den.
// Reduced-precision mode: the corrections are solved in FP32 until the relative
// update reaches kHpSwitch * tol, and in FP64 from there on (the FP32 rounding
// of a correction does not vanish at the fixed point, where d != 0).
constexpr double kHpSwitch = 100.0;

struct IterState {
    int iter;       // split steps done
    int done;       // 1 once converged or capped
    int converged;  // 1 if rel <= tol
    int hp;         // reduced-precision mode: 1 once the corrections are solved in FP64
    double rel;
    unsigned long long corr_bits;  // running max |dt d| of the step's corrections (bits)
    double corr;                   // the last step's largest correction (reduced precision)
    int fp32_steps;                // steps done with FP32 corrections
    int pad;
};

// Anderson extrapolation's small state on the device: the raw products
// <f_a, f_b> of the last m + 1 residuals by history slot, and the weights of
// the next state
struct AaDev {
    double R[9][9];
    double c[9];
    int used;  // difference columns the last weights used
    int pad;
};

struct Problem {
    adr_grid grid{};
    adr_opts opts{};
    double mu = 0, sigma = 0;
    cudaStream_t stream = nullptr;
    GridView gv{};
    int N = 0;             // nx*ny
    int n_interior = 0;
    int n_sm = 0;
    int rows_per_thread = 16;   // launch shape of the curve solve (<= 16 rows per thread)
    int map_blocks_per_sm = 4;  // launch shape of the curve -> grid map
    bool const_beta = false;
    double bmax = 0;
    Family fam[2];
    // owned device buffers
    uint8_t* mask = nullptr;    // copy of the caller's node mask (warm-start features)
    uint8_t* cell = nullptr;
    uint8_t* ntype = nullptr;
    double* beta1 = nullptr;
    double* beta2 = nullptr;
    double* f = nullptr;
    double* ubuf[3] = {nullptr, nullptr, nullptr};  // u_j / u_{j+1} ping-pong and u_{j+1/2}
    double* partial = nullptr;                      // per-block norm partial sums
    int n_partial_blocks = 0;
    IterState* state = nullptr;
    double* pivmin = nullptr;   // [2] smallest |Thomas pivot| of each family's systems
    double* fextra = nullptr;                       // [N] extra load (parabolic slices)
    // direct transfer (opts.transfer = 1): the iteration state at the B nodes
    double* xu[2] = {nullptr, nullptr};  // u_j / u_{j+1} ping-pong at the B nodes
    double* xuG = nullptr;               // u_{j+1/2} at the G nodes
    double* xtmp = nullptr;              // B-node work array (midpoint output)
    bool xu_set = false;                 // xu[0] already holds the initial state
    // Anderson extrapolation (opts.anderson = m): histories of m + 1 state vectors
    double* aa_f = nullptr;              // residuals f = g - u
    double* aa_g = nullptr;              // map outputs g
    AaDev* aa_dev = nullptr;
    double* aa_partial = nullptr;        // per-block partial products
    std::vector<void*> owned;
};

// error helpers
void set_error(const std::string& msg);
adr_status cuda_fail(cudaError_t e, const char* what);
#define TRY_S(x)                      \
    do {                              \
        adr_status _st = (x);         \
        if (_st != ADR_OK) return _st; \
    } while (0)
#define ADR_CUDA_TRY(call)                                      \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return ::adr::cuda_fail(_e, #call); \
    } while (0)

// The library's stream-ordered memory pool on the current device (api.cu).
// Problem buffers and setup temporaries come from it and go back to it; it
// keeps up to kPoolKeepBytes of freed memory mapped, so that creating and
// destroying problems does not map and unmap device memory every time.
// NULL when no pool could be made (the device's default pool is used then).
constexpr unsigned long long kPoolKeepBytes = 8ull << 30;
cudaMemPool_t device_pool();

// stream-ordered allocation of n bytes from the library's pool
inline cudaError_t pool_alloc(void** q, size_t n, cudaStream_t st)
{
    cudaMemPool_t pool = device_pool();
    return pool ? cudaMallocFromPoolAsync(q, n, pool, st) : cudaMallocAsync(q, n, st);
}

// free a buffer owned by the problem (NULL is a no-op), in stream order
inline void dev_free(Problem* p, void* ptr)
{
    if (!ptr) return;
    for (size_t i = 0; i < p->owned.size(); ++i)
        if (p->owned[i] == ptr) {
            cudaFreeAsync(ptr, p->stream);
            p->owned.erase(p->owned.begin() + i);
            return;
        }
}

template <typename T>
adr_status dev_alloc(Problem* p, T** ptr, size_t count)
{
    void* q = nullptr;
    cudaError_t e = pool_alloc(&q, count * sizeof(T) + 16, p->stream);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        set_error(std::string("device allocation failed: ") + cudaGetErrorString(e));
        return ADR_ENOMEM;
    }
    p->owned.push_back(q);
    *ptr = static_cast<T*>(q);
    return ADR_OK;
}

// setup (geometry.cu)
adr_status build_geometry(Problem* p, const uint8_t* mask);
adr_status build_transfer(Problem* p);  // crossing tables of the direct transfer

// sweeps (sweep.cu)
adr_status setup_groups(Problem* p, int fam, const std::vector<int>& off);
void release_groups(Problem* p, int fam);
adr_status launch_map_coef(Problem* p, int fam);
int grid_map_blocks(const Problem* p);
adr_status prepare_family(Problem* p, int fam, double td, double dt, double sig, int paper);
adr_status load_family(Problem* p, const double* fextra, double fx_scale);
adr_status launch_line_solve(Problem* p, int fam, double dt, const double* u_even,
                             const double* u_odd, bool use_state, int paper);
adr_status launch_mask_copy(Problem* p, const double* in, double* out);
// make the iteration's factorisation family 0's active one (sweep.cu); a
// batch reads the active buffers once, when it is built
adr_status ensure_iteration_active(Problem* p);
// Anderson extrapolation (accel.cu)
adr_status launch_anderson(Problem* p);
adr_status alloc_anderson(Problem* p);
// a batch's view for the extrapolation: its per-problem table and the map's
// active block lists
struct AaBatchView {
    const void* table;           // per-problem arguments (anderson_batch_table)
    int n, mmax, grid;
    const int* blk_prob;
    const int* blk_local;
    const int* nblk;
    const int* const* act_blocks;
    const int* act_count;
    const int* sel;
};
adr_status anderson_batch_table(Problem* const* ps, int n, void** table, int* mmax);
adr_status launch_anderson_batch(const AaBatchView& v, cudaStream_t st);
// the curve solve of one substep through the grid (gather pass + solve in
// FP64, the solve's own gather otherwise), and its two passes apart
adr_status launch_substep_solve(Problem* p, int fam, double dt, const double* u_even, const double* u_odd,
                                bool use_state);
adr_status launch_gather_pass(Problem* p, int fam, const double* u);
adr_status launch_solve_pass(Problem* p, int fam, double dt, const double* u);
// direct transfer between the families (sweep.cu)
adr_status launch_line_solve_dir(Problem* p, int fam, double dt, const double* u_even,
                                 const double* u_odd, bool use_state);
adr_status launch_xfer(Problem* p, int to_fam, const double* v, double* out_even, double* out_odd,
                       int shift, const double* prev_even, const double* prev_odd, bool use_state,
                       bool norms);
adr_status launch_gather_nodes(Problem* p, int fam, const double* u, double* out);
adr_status launch_node_midpoint(Problem* p, const double* u_even, const double* u_odd, const double* vb,
                                double* out, bool use_state);
// batches of problems (sweep.cu)
struct BatchDev;
adr_status batch_dev_create(Problem* const* ps, int n, const double* dts, const double* tols,
                            const int* max_iters, BatchDev** out);
adr_status batch_dev_step(BatchDev* b, cudaStream_t st, cudaGraphConditionalHandle cond);
adr_status batch_dev_reset(BatchDev* b, cudaStream_t st);
void batch_dev_destroy(BatchDev* b);
adr_status launch_state_reset(Problem* p);
// warm-start network (cnn.cu): prediction [64][64][8] -> initial state on the grid
adr_status launch_cnn_upsample(Problem* p, const float* y, const double* u0, const double* scale,
                               double* u);
// one network forward on a problem's stream (cnn.cu)
adr_status cnn_forward_on(adr_cnn* c, int batch, const uint16_t* x, float* y, cudaStream_t st);

}  // namespace adr
