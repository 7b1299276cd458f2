// C ABI of the directional splitting solver: handle lifecycle, the outer
// iteration as one CUDA graph with a device-side WHILE loop, and the
// parabolic time stepping.  See include/adr.h for the contract.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "adr_internal.cuh"

namespace adr {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

cudaMemPool_t device_pool()
{
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        pool = nullptr;
    } else {
        unsigned long long keep = kPoolKeepBytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pools[dev] = pool;
    return pool;
}

adr_status cuda_fail(cudaError_t e, const char* what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return ADR_ECUDA;
}

// launchers defined in sweep.cu
adr_status launch_grid_map_ex(Problem* p, int fam, double* out_even, double* out_odd,
                              int parity_shift, const double* prev_even, const double* prev_odd,
                              bool use_state, bool norms, const double* vin = nullptr);
adr_status launch_check_ex(Problem* p, double tol, int max_iter,
                           cudaGraphConditionalHandle handle, bool use_cond);
adr_status launch_finish(Problem* p, double* out, double* iter_out, bool midpoint);

}  // namespace adr

using namespace adr;

// The handle: the problem plus the cached solve graph.
struct adr_problem {
    Problem p;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // parameters the cached graph was captured with
    double g_theta = 0, g_dt = 0, g_sig = 0, g_scale = 0, g_tol = 0;
    int g_max_iter = -1;
    bool g_accel = false;
    const double* g_fextra = nullptr;
    double line_unknowns[2] = {0, 0};
    std::vector<int> offs[2];  // host copies of the curve offsets
    bool diverged = false;     // the last iteration stopped on a non-finite norm
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // learned warm start (adr_set_warm_start): the network (not owned) and the
    // buffers of its chain
    adr_cnn* cnn = nullptr;
    uint16_t* ws_x = nullptr;    // features [64][64][40] (BF16 storage)
    float* ws_y = nullptr;       // prediction [64][64][8]
    double* ws_u0 = nullptr;     // the paper's initial state [ny][nx]
    double* ws_par = nullptr;    // mu, sigma, scale
};

#define TRY(x)                       \
    do {                             \
        adr_status _s = (x);         \
        if (_s != ADR_OK) return _s; \
    } while (0)

namespace {

double default_dt(const Problem& p, double sig)
{
    double hs = p.gv.hs;
    double lmax = 12.0 * p.mu / (hs * hs) + 2.0 * std::sqrt(3.0) * p.bmax / hs;
    return 2.0 / std::sqrt(sig * lmax);
}

void drop_graph(adr_problem* h)
{
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
    h->g_max_iter = -1;
}

// Capture one split step (B sweep, B map, G sweep, G map + norms, check) as
// the body of a conditional WHILE node; the check kernel clears the
// condition once the relative update reaches tol or max_iter steps ran.
adr_status build_graph(adr_problem* h, double theta, double dt, double sig,
                       const double* fextra, double fx_scale, double tol, int max_iter, bool accel)
{
    Problem* p = &h->p;
    drop_graph(h);
    ADR_CUDA_TRY(cudaGraphCreate(&h->graph, 0));
    cudaGraphConditionalHandle cond;
    ADR_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, h->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    ADR_CUDA_TRY(cudaGraphAddNode(&node, h->graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    TRY(prepare_family(p, 0, theta * dt, dt, sig, 0));
    TRY(prepare_family(p, 1, theta * dt, dt, sig, 0));
    cudaStream_t user = p->stream;
    p->stream = h->cap_stream;
    cudaError_t e = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed);
    adr_status s = ADR_OK;
    if (e != cudaSuccess) s = cuda_fail(e, "cudaStreamBeginCaptureToGraph");
    if (p->opts.transfer) {
        // B solve from the state at the B nodes, B -> G nodes, G solve,
        // G -> B nodes (u_{j+1}) with the norms of the update
        if (s == ADR_OK) s = launch_line_solve_dir(p, 0, dt, p->xu[0], p->xu[1], true);
        if (s == ADR_OK)
            s = launch_xfer(p, 1, p->fam[0].v, p->xuG, p->xuG, 0, nullptr, nullptr, true, false);
        if (s == ADR_OK) s = launch_line_solve_dir(p, 1, dt, p->xuG, p->xuG, true);
        if (s == ADR_OK)
            s = launch_xfer(p, 0, p->fam[1].v, p->xu[0], p->xu[1], 1, p->xu[0], p->xu[1], true, true);
    } else {
        if (s == ADR_OK) s = launch_substep_solve(p, 0, dt, p->ubuf[0], p->ubuf[1], true);
        if (s == ADR_OK)
            s = launch_grid_map_ex(p, 0, p->ubuf[2], p->ubuf[2], 0, nullptr, nullptr, true, false);
        if (s == ADR_OK) s = launch_substep_solve(p, 1, dt, p->ubuf[2], p->ubuf[2], true);
        if (s == ADR_OK)
            s = launch_grid_map_ex(p, 1, p->ubuf[0], p->ubuf[1], 1, p->ubuf[0], p->ubuf[1], true, true);
    }
    if (s == ADR_OK) s = launch_check_ex(p, tol, max_iter, cond, true);
    if (s == ADR_OK && accel) s = launch_anderson(p);  // u_{j+1} extrapolated unless done
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &out);
    p->stream = user;
    if (s != ADR_OK) return s;
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    ADR_CUDA_TRY(cudaGraphInstantiate(&h->exec, h->graph, 0));
    h->g_theta = theta;
    h->g_dt = dt;
    h->g_sig = sig;
    h->g_fextra = fextra;
    h->g_scale = fx_scale;
    h->g_tol = tol;
    h->g_max_iter = max_iter;
    h->g_accel = accel;
    return ADR_OK;
}

// Output of the direct-transfer iteration: theta = 1/2 the midpoint
// (u_j + u_{j+1/2}) / 2 at the B nodes, otherwise the last G curve values,
// mapped to the grid (iter_out: the G values); no step run: the initial state.
adr_status finish_direct(Problem* p, int max_iter, double* out, double* iter_out, bool midpoint)
{
    if (max_iter <= 0) {
        TRY(launch_grid_map_ex(p, 0, out, out, 0, nullptr, nullptr, false, false, p->xu[0]));
        if (iter_out) TRY(launch_grid_map_ex(p, 0, iter_out, iter_out, 0, nullptr, nullptr, false, false, p->xu[0]));
        return ADR_OK;
    }
    if (midpoint) {
        TRY(launch_node_midpoint(p, p->xu[0], p->xu[1], p->fam[0].v, p->xtmp, true));
        TRY(launch_grid_map_ex(p, 0, out, out, 0, nullptr, nullptr, false, false, p->xtmp));
    } else {
        TRY(launch_grid_map_ex(p, 1, out, out, 0, nullptr, nullptr, false, false));
    }
    if (iter_out) TRY(launch_grid_map_ex(p, 1, iter_out, iter_out, 0, nullptr, nullptr, false, false));
    return ADR_OK;
}

// the handle's capture stream and timing events, on first use
adr_status ensure_stream_events(adr_problem* h)
{
    if (!h->cap_stream) ADR_CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    if (!h->ev0) ADR_CUDA_TRY(cudaEventCreate(&h->ev0));
    if (!h->ev1) ADR_CUDA_TRY(cudaEventCreate(&h->ev1));
    return ADR_OK;
}

// Outer iteration from the state in ubuf[0] (the direct transfer: in xu[0]
// when xu_set, else gathered from ubuf[0]); results into out / iter_out.
adr_status run_iteration(adr_problem* h, double theta, double dt, double sig,
                         const double* fextra, double fx_scale, double tol, int max_iter,
                         bool midpoint, double* out, double* iter_out, adr_stats* stats,
                         bool* converged, bool accel = true)
{
    Problem* p = &h->p;
    accel = accel && p->opts.anderson > 0;
    TRY(ensure_stream_events(h));
    TRY(launch_state_reset(p));
    ADR_CUDA_TRY(cudaEventRecord(h->ev0, p->stream));
    if (p->opts.transfer) {
        // the initial state at the B nodes (unless the paper's u_0 put it there)
        if (!p->xu_set) TRY(launch_gather_nodes(p, 0, p->ubuf[0], p->xu[0]));
        p->xu_set = false;
    }
    if (max_iter > 0) {
        TRY(prepare_family(p, 0, theta * dt, dt, sig, 0));
        TRY(prepare_family(p, 1, theta * dt, dt, sig, 0));
        TRY(load_family(p, fextra, fx_scale));
        if (!h->exec || h->g_theta != theta || h->g_dt != dt || h->g_sig != sig ||
            h->g_fextra != fextra || h->g_scale != fx_scale || h->g_tol != tol ||
            h->g_max_iter != max_iter || h->g_accel != accel)
            TRY(build_graph(h, theta, dt, sig, fextra, fx_scale, tol, max_iter, accel));
        ADR_CUDA_TRY(cudaGraphLaunch(h->exec, p->stream));
    }
    if (p->opts.transfer) TRY(finish_direct(p, max_iter, out, iter_out, midpoint));
    else TRY(launch_finish(p, out, iter_out, midpoint));
    ADR_CUDA_TRY(cudaEventRecord(h->ev1, p->stream));
    IterState st;
    double piv[2] = {INFINITY, INFINITY};
    ADR_CUDA_TRY(cudaMemcpyAsync(&st, p->state, sizeof st, cudaMemcpyDeviceToHost, p->stream));
    if (max_iter > 0)
        ADR_CUDA_TRY(cudaMemcpyAsync(piv, p->pivmin, sizeof piv, cudaMemcpyDeviceToHost, p->stream));
    ADR_CUDA_TRY(cudaStreamSynchronize(p->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    *converged = st.converged != 0;
    if (st.iter > 0 && !std::isfinite(st.rel)) {
        *converged = false;
        h->diverged = true;
    }
    if (stats) {
        stats->iters += st.iter;
        stats->rel_update = st.rel;
        stats->ms += ms;
        stats->line_dofs += (double)st.iter * (h->line_unknowns[0] + h->line_unknowns[1]);
        stats->dt = dt;
        stats->min_pivot = std::fmin(stats->min_pivot, std::fmin(piv[0], piv[1]));
        stats->max_correction = st.iter > 0 ? st.corr : 0.0;
        if (p->opts.prec == ADR_FP32_REFINE) stats->fp32_steps += st.fp32_steps;
    }
    return ADR_OK;
}

adr_status init_state(adr_problem* h, int init, const double* u_init)
{
    Problem* p = &h->p;
    if (init == ADR_INIT_USER) {
        if (!u_init) {
            set_error("opts.init == ADR_INIT_USER needs u_init");
            return ADR_EINVAL;
        }
        return launch_mask_copy(p, u_init, p->ubuf[0]);
    }
    if (init == ADR_INIT_PAPER_U0) {
        TRY(prepare_family(p, 0, 1.0, 1.0, p->sigma, 1));
        TRY(load_family(p, nullptr, 0.0));
        TRY(launch_line_solve(p, 0, 1.0, nullptr, nullptr, false, 1));
        if (p->opts.transfer) {
            // the B curve solutions are the state at the B nodes as they stand
            ADR_CUDA_TRY(cudaMemcpyAsync(p->xu[0], p->fam[0].v, sizeof(double) * p->fam[0].n_nodes,
                                         cudaMemcpyDeviceToDevice, p->stream));
            p->xu_set = true;
            return ADR_OK;
        }
        return launch_grid_map_ex(p, 0, p->ubuf[0], p->ubuf[0], 0, nullptr, nullptr, false, false);
    }
    if (init == ADR_INIT_ZERO) return launch_mask_copy(p, nullptr, p->ubuf[0]);
    if (init == ADR_INIT_LEARNED) {
        if (!h->cnn) {
            set_error("opts.init == ADR_INIT_LEARNED needs a network (adr_set_warm_start)");
            return ADR_EINVAL;
        }
        // the paper's initial state (eq. u0stationary), the network's features
        // of the problem and of it, one forward pass, and the corrected state
        TRY(prepare_family(p, 0, 1.0, 1.0, p->sigma, 1));
        TRY(load_family(p, nullptr, 0.0));
        TRY(launch_line_solve(p, 0, 1.0, nullptr, nullptr, false, 1));
        TRY(launch_grid_map_ex(p, 0, h->ws_u0, h->ws_u0, 0, nullptr, nullptr, false, false));
        TRY(adr_cnn_features(1, p->grid.nx, p->f, p->beta1, p->beta2, p->mask, h->ws_par,
                             h->ws_par + 1, h->ws_u0, h->ws_x, h->ws_par + 2, p->stream));
        TRY(cnn_forward_on(h->cnn, 1, h->ws_x, h->ws_y, p->stream));
        return launch_cnn_upsample(p, h->ws_y, h->ws_u0, h->ws_par + 2, p->ubuf[0]);
    }
    set_error("unsupported opts.init");
    return ADR_EINVAL;
}

void clear_stats(adr_stats* s)
{
    if (!s) return;
    memset(s, 0, sizeof *s);
    s->min_pivot = INFINITY;
}

adr_status check_opts(const adr_opts* o)
{
    if (!o) return ADR_OK;
    if (o->prec != ADR_FP64 && o->prec != ADR_FP32_REFINE) {
        set_error("opts.prec must be ADR_FP64 or ADR_FP32_REFINE");
        return ADR_EINVAL;
    }
    if (!(o->theta > 0.0 && o->theta <= 1.0)) {
        set_error("opts.theta must lie in (0, 1]");
        return ADR_EINVAL;
    }
    if (o->interp_weights != 0 && o->interp_weights != 1) {
        set_error("opts.interp_weights must be 0 or 1");
        return ADR_EINVAL;
    }
    if (o->stabilize != 0 && o->stabilize != 1) {
        set_error("opts.stabilize must be 0 or 1");
        return ADR_EINVAL;
    }
    if (o->stabilize && o->prec != ADR_FP64) {
        set_error("opts.stabilize needs opts.prec == ADR_FP64");
        return ADR_EINVAL;
    }
    if (o->max_iter < 0 || !std::isfinite(o->dt) || std::isnan(o->tol)) {
        set_error("opts.max_iter must be >= 0 and dt, tol finite");
        return ADR_EINVAL;
    }
    if (o->init < ADR_INIT_ZERO || o->init > ADR_INIT_LEARNED) {
        set_error("unsupported opts.init");
        return ADR_EINVAL;
    }
    if (o->transfer != 0 && o->transfer != 1) {
        set_error("opts.transfer must be 0 or 1");
        return ADR_EINVAL;
    }
    if (o->transfer && o->prec != ADR_FP64) {
        set_error("opts.transfer == 1 needs opts.prec == ADR_FP64");
        return ADR_EINVAL;
    }
    if (o->anderson < 0 || o->anderson > 8) {
        set_error("opts.anderson must be 0..8");
        return ADR_EINVAL;
    }
    if (o->anderson && o->prec != ADR_FP64) {
        set_error("opts.anderson > 0 needs opts.prec == ADR_FP64");
        return ADR_EINVAL;
    }
    if ((o->rows_per_thread != 0 && o->rows_per_thread != 2 && o->rows_per_thread != 4 &&
         o->rows_per_thread != 8 && o->rows_per_thread != 16) ||
        o->map_blocks_per_sm < 0 || o->map_blocks_per_sm > 8) {
        set_error("opts.rows_per_thread must be 0, 2, 4, 8 or 16 and map_blocks_per_sm 0..8");
        return ADR_EINVAL;
    }
    return ADR_OK;
}

}  // namespace

extern "C" {

void adr_default_opts(adr_opts* o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->prec = ADR_FP64;
    o->theta = 0.5;
    o->dt = 0.0;
    o->tol = 1e-10;
    o->max_iter = 100000;
    o->init = ADR_INIT_ZERO;
}

adr_status adr_cnn_initial_state(adr_problem* h, const float* y, const double* u0,
                                 const double* scale, double* u_out)
{
    if (!h || !y || !u_out) {
        set_error("adr_cnn_initial_state: NULL argument");
        return ADR_EINVAL;
    }
    if (h->p.grid.nx != 256 || h->p.grid.ny != 256) {
        set_error("adr_cnn_initial_state: the network predicts 256 x 256 grids");
        return ADR_EINVAL;
    }
    return launch_cnn_upsample(&h->p, y, u0, scale, u_out);
}

const char* adr_last_error(void) { return g_err.c_str(); }

adr_status adr_create(const adr_grid* grid, const uint8_t* mask, double mu, double sigma,
                      const double* beta1, const double* beta2, const double* f,
                      const adr_opts* opts, void* stream, adr_problem** out)
{
    g_err.clear();
    if (!out) {
        set_error("out is NULL");
        return ADR_EINVAL;
    }
    *out = nullptr;
    if (!grid || !mask || !beta1 || !beta2 || !f) {
        set_error("NULL argument");
        return ADR_EINVAL;
    }
    if (grid->nx < 3 || grid->ny < 3 || !(grid->x1 > grid->x0) || !(grid->y1 > grid->y0) ||
        (long long)grid->nx * grid->ny > 0x7fffffffLL) {
        set_error("grid needs nx, ny >= 3, x1 > x0, y1 > y0 and nx*ny < 2^31");
        return ADR_EINVAL;
    }
    if (!(mu > 0.0) || !(sigma > 0.0) || !std::isfinite(mu) || !std::isfinite(sigma)) {
        set_error("mu and sigma must be positive constants");
        return ADR_EINVAL;
    }
    TRY(check_opts(opts));
    adr_problem* h = new (std::nothrow) adr_problem;
    if (!h) {
        set_error("out of host memory");
        return ADR_ENOMEM;
    }
    Problem* p = &h->p;
    p->grid = *grid;
    if (opts) p->opts = *opts;
    else adr_default_opts(&p->opts);
    p->mu = mu;
    p->sigma = sigma;
    p->stream = static_cast<cudaStream_t>(stream);
    if (p->opts.rows_per_thread > 0) p->rows_per_thread = p->opts.rows_per_thread;
    if (p->opts.map_blocks_per_sm > 0) p->map_blocks_per_sm = p->opts.map_blocks_per_sm;
    p->N = grid->nx * grid->ny;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev);
    }
    adr_status s = ADR_OK;
    auto fail = [&](adr_status st) {
        adr_destroy(h);
        return st;
    };
    size_t N = p->N;
    if ((s = dev_alloc(p, &p->beta1, N)) || (s = dev_alloc(p, &p->beta2, N)) ||
        (s = dev_alloc(p, &p->f, N)) || (s = dev_alloc(p, &p->mask, N)))
        return fail(s);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(p->mask, mask, N, cudaMemcpyDeviceToDevice, p->stream)) ||
        (e = cudaMemcpyAsync(p->beta1, beta1, N * 8, cudaMemcpyDeviceToDevice, p->stream)) ||
        (e = cudaMemcpyAsync(p->beta2, beta2, N * 8, cudaMemcpyDeviceToDevice, p->stream)) ||
        (e = cudaMemcpyAsync(p->f, f, N * 8, cudaMemcpyDeviceToDevice, p->stream)))
        return fail(cuda_fail(e, "cudaMemcpyAsync"));
    if ((s = build_geometry(p, mask))) return fail(s);
    for (int k = 0; k < 3; ++k)
        if ((s = dev_alloc(p, &p->ubuf[k], N))) return fail(s);
    {
        int keep = p->map_blocks_per_sm;  // partial sums sized for the largest map grid
        p->map_blocks_per_sm = 8;
        p->n_partial_blocks = grid_map_blocks(p);
        p->map_blocks_per_sm = keep;
    }
    if (p->opts.transfer) {
        if ((s = build_transfer(p)) || (s = dev_alloc(p, &p->xu[0], p->fam[0].n_nodes)) ||
            (s = dev_alloc(p, &p->xu[1], p->fam[0].n_nodes)) ||
            (s = dev_alloc(p, &p->xtmp, p->fam[0].n_nodes)) ||
            (s = dev_alloc(p, &p->xuG, p->fam[1].n_nodes)))
            return fail(s);
        if ((e = cudaMemsetAsync(p->xu[0], 0, sizeof(double) * p->fam[0].n_nodes, p->stream)))
            return fail(cuda_fail(e, "cudaMemsetAsync"));
    }
    if ((s = alloc_anderson(p))) return fail(s);
    if ((s = dev_alloc(p, &p->partial, 2 * (size_t)p->n_partial_blocks)) ||
        (s = dev_alloc(p, &p->state, 1)) || (s = dev_alloc(p, &p->fextra, N)) ||
        (s = dev_alloc(p, &p->pivmin, 2)))
        return fail(s);
    for (int fam = 0; fam < 2; ++fam) {
        std::vector<int>& off = h->offs[fam];
        off.resize(p->fam[fam].n_lines + 1);
        if ((e = cudaMemcpyAsync(off.data(), p->fam[fam].off, off.size() * sizeof(int),
                                 cudaMemcpyDeviceToHost, p->stream)) ||
            (e = cudaStreamSynchronize(p->stream)))
            return fail(cuda_fail(e, "cudaMemcpyAsync"));
        double u = 0;
        for (int l = 0; l < p->fam[fam].n_lines; ++l) u += std::max(0, off[l + 1] - off[l] - 2);
        h->line_unknowns[fam] = u;
        if ((s = setup_groups(p, fam, off))) return fail(s);
    }
    // the capture stream and the timing events come with the handle's first
    // own solve: a handle solved only inside batches never needs them, and
    // thousands of handles would otherwise hold thousands of streams
    if ((e = cudaStreamSynchronize(p->stream))) return fail(cuda_fail(e, "adr_create"));
    *out = h;
    return ADR_OK;
}

void adr_destroy(adr_problem* h)
{
    if (!h) return;
    // a batch may still use the buffers on its own stream
    cudaDeviceSynchronize();
    drop_graph(h);
    for (void* q : h->p.owned) cudaFreeAsync(q, h->p.stream);
    cudaStreamSynchronize(h->p.stream);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
}

adr_status adr_set_warm_start(adr_problem* h, adr_cnn* cnn)
{
    g_err.clear();
    if (!h) {
        set_error("adr_set_warm_start: NULL handle");
        return ADR_EINVAL;
    }
    Problem* p = &h->p;
    if (cnn && (p->grid.nx != 256 || p->grid.ny != 256)) {
        set_error("adr_set_warm_start: the network predicts 256 x 256 grids");
        return ADR_EINVAL;
    }
    if (cnn && !h->ws_x) {
        TRY(dev_alloc(p, &h->ws_x, (size_t)64 * 64 * 40));
        TRY(dev_alloc(p, &h->ws_y, (size_t)64 * 64 * 8));
        TRY(dev_alloc(p, &h->ws_u0, (size_t)p->N));
        TRY(dev_alloc(p, &h->ws_par, 3));
        // mu and sigma of the features, next to the scale the features write
        const double par[2] = {p->mu, p->sigma};
        ADR_CUDA_TRY(cudaMemcpyAsync(h->ws_par, par, sizeof par, cudaMemcpyHostToDevice, p->stream));
        ADR_CUDA_TRY(cudaStreamSynchronize(p->stream));
    }
    h->cnn = cnn;
    return ADR_OK;
}

adr_status adr_solve_stationary(adr_problem* h, const double* u_init, double* u_out,
                                double* u_iter_out, adr_stats* stats)
{
    g_err.clear();
    if (!h || !u_out) {
        set_error("NULL handle or output");
        return ADR_EINVAL;
    }
    Problem* p = &h->p;
    const adr_opts& o = p->opts;
    clear_stats(stats);
    double dt = o.dt > 0 ? o.dt : default_dt(*p, p->sigma);
    TRY(init_state(h, o.init, u_init));
    bool conv = false;
    TRY(run_iteration(h, o.theta, dt, p->sigma, nullptr, 0.0, o.tol, o.max_iter,
                      o.theta == 0.5, u_out, u_iter_out, stats, &conv));
    if (h->diverged) {
        h->diverged = false;
        set_error("the iteration diverged (a norm stopped being finite)");
        return ADR_ENOCONV;
    }
    if (!conv && o.tol > 0.0) {
        set_error("max_iter reached before tol");
        return ADR_ENOCONV;
    }
    return ADR_OK;
}

adr_status adr_step_parabolic(adr_problem* h, double dt, int nsteps, int mode, double* u,
                              adr_stats* stats)
{
    g_err.clear();
    if (!h || !u || !(dt > 0.0) || nsteps < 0 || (mode != 0 && mode != 1)) {
        set_error("bad arguments to adr_step_parabolic");
        return ADR_EINVAL;
    }
    Problem* p = &h->p;
    const adr_opts& o = p->opts;
    clear_stats(stats);
    if (nsteps == 0) return launch_mask_copy(p, u, u);
    bool conv = false;
    if (mode == 0) {
        TRY(launch_mask_copy(p, u, p->ubuf[0]));
        TRY(run_iteration(h, o.theta, dt, p->sigma, nullptr, 0.0, -1.0, nsteps, false, u, nullptr,
                          stats, &conv, false));
        return ADR_OK;
    }
    double sig = p->sigma + 1.0 / dt;
    double pdt = o.dt > 0 ? o.dt : default_dt(*p, sig);
    adr_status result = ADR_OK;
    for (int k = 0; k < nsteps; ++k) {
        TRY(launch_mask_copy(p, u, p->fextra));
        TRY(launch_mask_copy(p, u, p->ubuf[0]));
        TRY(run_iteration(h, o.theta, pdt, sig, p->fextra, 1.0 / dt, o.tol, o.max_iter,
                          o.theta == 0.5, u, nullptr, stats, &conv));
        if (!conv && o.tol > 0.0) result = ADR_ENOCONV;
    }
    if (result != ADR_OK) set_error("a time slice reached max_iter before tol");
    return result;
}

adr_status adr_split_step(adr_problem* h, double dt, const double* u, double* u_half,
                          double* u_next)
{
    g_err.clear();
    if (!h || !u || !u_next) {
        set_error("NULL argument");
        return ADR_EINVAL;
    }
    Problem* p = &h->p;
    double* half = u_half ? u_half : p->ubuf[2];
    double th = p->opts.theta;
    TRY(prepare_family(p, 0, th * dt, dt, p->sigma, 0));
    TRY(prepare_family(p, 1, th * dt, dt, p->sigma, 0));
    TRY(load_family(p, nullptr, 0.0));
    if (p->opts.transfer) {
        // u onto the B nodes, B solve, B -> G nodes, G solve; both halves to the grid
        TRY(launch_gather_nodes(p, 0, u, p->xtmp));
        TRY(launch_line_solve_dir(p, 0, dt, p->xtmp, p->xtmp, false));
        TRY(launch_grid_map_ex(p, 0, half, half, 0, nullptr, nullptr, false, false));
        TRY(launch_xfer(p, 1, p->fam[0].v, p->xuG, p->xuG, 0, nullptr, nullptr, false, false));
        TRY(launch_line_solve_dir(p, 1, dt, p->xuG, p->xuG, false));
        TRY(launch_grid_map_ex(p, 1, u_next, u_next, 0, nullptr, nullptr, false, false));
    } else {
        TRY(launch_substep_solve(p, 0, dt, u, u, false));
        TRY(launch_grid_map_ex(p, 0, half, half, 0, nullptr, nullptr, false, false));
        TRY(launch_substep_solve(p, 1, dt, half, half, false));
        TRY(launch_grid_map_ex(p, 1, u_next, u_next, 0, nullptr, nullptr, false, false));
    }
    ADR_CUDA_TRY(cudaStreamSynchronize(p->stream));
    return ADR_OK;
}

adr_status adr_paper_u0(adr_problem* h, double* u0)
{
    g_err.clear();
    if (!h || !u0) {
        set_error("NULL argument");
        return ADR_EINVAL;
    }
    Problem* p = &h->p;
    TRY(prepare_family(p, 0, 1.0, 1.0, p->sigma, 1));
    TRY(load_family(p, nullptr, 0.0));
    TRY(launch_line_solve(p, 0, 1.0, nullptr, nullptr, false, 1));
    TRY(launch_grid_map_ex(p, 0, u0, u0, 0, nullptr, nullptr, false, false));
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;  // enqueued on the handle's stream
}

int adr_num_lines(const adr_problem* h, int fam)
{
    return (h && (fam == 0 || fam == 1)) ? h->p.fam[fam].n_lines : -1;
}

int adr_num_line_nodes(const adr_problem* h, int fam)
{
    return (h && (fam == 0 || fam == 1)) ? h->p.fam[fam].n_nodes : -1;
}

adr_status adr_get_lines(const adr_problem* h, int fam, int* off, double* xi, double* eta,
                         double* hh)
{
    if (!h || (fam != 0 && fam != 1)) {
        set_error("bad handle or family");
        return ADR_EINVAL;
    }
    const Family& F = h->p.fam[fam];
    if (off) ADR_CUDA_TRY(cudaMemcpy(off, F.off, sizeof(int) * (F.n_lines + 1), cudaMemcpyDeviceToHost));
    if (xi) ADR_CUDA_TRY(cudaMemcpy(xi, F.xi, sizeof(double) * F.n_nodes, cudaMemcpyDeviceToHost));
    if (eta) ADR_CUDA_TRY(cudaMemcpy(eta, F.eta, sizeof(double) * F.n_nodes, cudaMemcpyDeviceToHost));
    if (hh) ADR_CUDA_TRY(cudaMemcpy(hh, F.h, sizeof(double) * F.n_lines, cudaMemcpyDeviceToHost));
    return ADR_OK;
}

adr_status adr_get_crossings(const adr_problem* h, int fam, int* seg, double* t, double* pos)
{
    if (!h || (fam != 0 && fam != 1)) {
        set_error("bad handle or family");
        return ADR_EINVAL;
    }
    const Family& F = h->p.fam[fam];
    size_t n = 4 * (size_t)h->p.N;
    if (seg) ADR_CUDA_TRY(cudaMemcpy(seg, F.cg, sizeof(int) * n, cudaMemcpyDeviceToHost));
    if (t) ADR_CUDA_TRY(cudaMemcpy(t, F.ct, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (pos) ADR_CUDA_TRY(cudaMemcpy(pos, F.cpos, sizeof(double) * n, cudaMemcpyDeviceToHost));
    return ADR_OK;
}

adr_status adr_get_transfer(const adr_problem* h, int fam, int* seg, double* t, double* pos)
{
    if (!h || (fam != 0 && fam != 1)) {
        set_error("bad handle or family");
        return ADR_EINVAL;
    }
    const Family& F = h->p.fam[fam];
    if (!h->p.opts.transfer || !F.xseg) {
        set_error("adr_get_transfer: the handle was created with opts.transfer == 0");
        return ADR_EINVAL;
    }
    size_t n = 2 * (size_t)F.n_nodes;
    if (seg) ADR_CUDA_TRY(cudaMemcpy(seg, F.xseg, sizeof(int) * n, cudaMemcpyDeviceToHost));
    if (t) ADR_CUDA_TRY(cudaMemcpy(t, F.xtt, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (pos) ADR_CUDA_TRY(cudaMemcpy(pos, F.xpos, sizeof(double) * n, cudaMemcpyDeviceToHost));
    return ADR_OK;
}

adr_status adr_autotune(adr_problem* h, int reps, int* rows_out, int* blocks_out, double* ms_out)
{
    g_err.clear();
    if (!h || reps < 1) {
        set_error("bad arguments to adr_autotune");
        return ADR_EINVAL;
    }
    Problem* p = &h->p;
    const int rows[3] = {4, 8, 16}, blocks[3] = {2, 4, 8};
    double best = 1e300;
    int bR = p->rows_per_thread, bM = p->map_blocks_per_sm;
    double ms[6];
    for (int R : rows) {
        p->rows_per_thread = R;
        drop_graph(h);
        for (int fam = 0; fam < 2; ++fam) {
            release_groups(p, fam);
            TRY(setup_groups(p, fam, h->offs[fam]));
        }
        for (int M : blocks) {
            p->map_blocks_per_sm = M;
            TRY(adr_time_kernels(h, reps, ms));
            double t = ms[0] + ms[1] + ms[2] + ms[3] + ms[4] + ms[5];
            if (t < best) {
                best = t;
                bR = R;
                bM = M;
            }
        }
    }
    p->rows_per_thread = bR;
    p->map_blocks_per_sm = bM;
    drop_graph(h);
    for (int fam = 0; fam < 2; ++fam) {
        release_groups(p, fam);
        TRY(setup_groups(p, fam, h->offs[fam]));
    }
    if (rows_out) *rows_out = bR;
    if (blocks_out) *blocks_out = bM;
    if (ms_out) *ms_out = best;
    return ADR_OK;
}

adr_status adr_time_kernels(adr_problem* h, int reps, double* ms_out)
{
    g_err.clear();
    if (!h || reps < 1 || !ms_out) {
        set_error("bad arguments to adr_time_kernels");
        return ADR_EINVAL;
    }
    Problem* p = &h->p;
    const adr_opts& o = p->opts;
    double dt = o.dt > 0 ? o.dt : default_dt(*p, p->sigma);
    TRY(prepare_family(p, 0, o.theta * dt, dt, p->sigma, 0));
    TRY(prepare_family(p, 1, o.theta * dt, dt, p->sigma, 0));
    TRY(load_family(p, nullptr, 0.0));
    // stages: B gather, B solve, B map (or transfer), G gather, G solve, G map
    // (or transfer) with the norms; a stage without a kernel of its own (the
    // gathers inside the solves of the other modes) reads 0
    const bool split = p->fam[0].ug != nullptr;
    cudaEvent_t ev[7];
    for (int k = 0; k < 7; ++k) ADR_CUDA_TRY(cudaEventCreate(&ev[k]));
    adr_status s = ADR_OK;
    for (int stage = 0; stage < 6 && s == ADR_OK; ++stage) {
        cudaEventRecord(ev[stage], p->stream);
        for (int r = 0; r < reps && s == ADR_OK; ++r) {
            if (o.transfer) {
                // B solve, B -> G transfer, G solve, G -> B transfer with norms
                switch (stage) {
                case 1:
                    s = launch_line_solve_dir(p, 0, dt, p->xu[0], p->xu[0], false);
                    break;
                case 2:
                    s = launch_xfer(p, 1, p->fam[0].v, p->xuG, p->xuG, 0, nullptr, nullptr, false, false);
                    break;
                case 4:
                    s = launch_line_solve_dir(p, 1, dt, p->xuG, p->xuG, false);
                    break;
                case 5:
                    s = launch_xfer(p, 0, p->fam[1].v, p->xu[1], p->xu[1], 0, p->xu[0], p->xu[0], false,
                                    true);
                    break;
                default:
                    break;
                }
                continue;
            }
            switch (stage) {
            case 0:
                if (split) s = launch_gather_pass(p, 0, p->ubuf[0]);
                break;
            case 1:
                s = launch_solve_pass(p, 0, dt, p->ubuf[0]);
                break;
            case 2:
                s = launch_grid_map_ex(p, 0, p->ubuf[2], p->ubuf[2], 0, nullptr, nullptr, false, false);
                break;
            case 3:
                if (split) s = launch_gather_pass(p, 1, p->ubuf[2]);
                break;
            case 4:
                s = launch_solve_pass(p, 1, dt, p->ubuf[2]);
                break;
            default:
                s = launch_grid_map_ex(p, 1, p->ubuf[1], p->ubuf[1], 0, p->ubuf[0], p->ubuf[0], false,
                                       true);
            }
        }
    }
    cudaEventRecord(ev[6], p->stream);
    cudaError_t e = cudaEventSynchronize(ev[6]);
    if (s == ADR_OK && e != cudaSuccess) s = cuda_fail(e, "adr_time_kernels");
    const bool has[6] = {split && !o.transfer, true, true, split && !o.transfer, true, true};
    for (int k = 0; k < 6 && s == ADR_OK; ++k) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
        ms_out[k] = has[k] ? ms / reps : 0.0;
    }
    for (int k = 0; k < 7; ++k) cudaEventDestroy(ev[k]);
    return s;
}

// ---------------------------------------------------------------- batches

}  // extern "C"

struct adr_batch {
    std::vector<adr_problem*> hs;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    BatchDev* dev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<double> dts;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

// run f with every handle's stream set to the batch stream
template <typename F>
adr_status on_batch_stream(adr_batch* b, F f)
{
    std::vector<cudaStream_t> saved;
    for (adr_problem* h : b->hs) {
        saved.push_back(h->p.stream);
        h->p.stream = b->stream;
    }
    adr_status s = f();
    for (size_t i = 0; i < b->hs.size(); ++i) b->hs[i]->p.stream = saved[i];
    return s;
}

// the batch's device tables and its loop graph: WHILE(any problem active)
// { batched split step }; an earlier build of them is released first
adr_status build_batch(adr_batch* b, const double* tols, const int* maxit);

adr_status prepare_batch(adr_batch* b)
{
    for (size_t i = 0; i < b->hs.size(); ++i) {
        Problem* p = &b->hs[i]->p;
        double td = p->opts.theta * b->dts[i];
        TRY(prepare_family(p, 0, td, b->dts[i], p->sigma, 0));
        TRY(prepare_family(p, 1, td, b->dts[i], p->sigma, 0));
        TRY(load_family(p, nullptr, 0.0));
    }
    return ADR_OK;
}

adr_status build_batch(adr_batch* b, const double* tols, const int* maxit)
{
    const int n = (int)b->hs.size();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (b->dev) {
        cudaStreamSynchronize(b->stream);
        batch_dev_destroy(b->dev);
        b->dev = nullptr;
    }
    std::vector<Problem*> ps(n);
    for (int i = 0; i < n; ++i) ps[i] = &b->hs[i]->p;
    TRY(batch_dev_create(ps.data(), n, b->dts.data(), tols, maxit, &b->dev));
    TRY(on_batch_stream(b, [&] { return prepare_batch(b); }));
    ADR_CUDA_TRY(cudaGraphCreate(&b->graph, 0));
    cudaGraphConditionalHandle cond;
    ADR_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, b->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    ADR_CUDA_TRY(cudaGraphAddNode(&node, b->graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    ADR_CUDA_TRY(cudaStreamBeginCaptureToGraph(b->cap_stream, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeRelaxed));
    adr_status s = batch_dev_step(b->dev, b->cap_stream, cond);
    cudaGraph_t cap = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &cap);
    if (s) return s;
    if (e) return cuda_fail(e, "cudaStreamEndCapture");
    ADR_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    ADR_CUDA_TRY(cudaStreamSynchronize(b->stream));
    return ADR_OK;
}

}  // namespace

extern "C" {

void adr_batch_destroy(adr_batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    batch_dev_destroy(b->dev);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
}

adr_status adr_batch_create(adr_problem* const* probs, int n, void* stream, adr_batch** out)
{
    g_err.clear();
    if (!out || !probs || n < 1) {
        set_error("adr_batch_create needs n >= 1 handles and an output");
        return ADR_EINVAL;
    }
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!probs[i] || probs[i]->p.opts.prec != probs[0]->p.opts.prec) {
            set_error("adr_batch_create: NULL handle or mixed precision modes");
            return ADR_EINVAL;
        }
        if (probs[i]->p.opts.transfer) {
            set_error("adr_batch_create: problems with opts.transfer == 1 are solved one by one");
            return ADR_EINVAL;
        }
    }
    adr_batch* b = new (std::nothrow) adr_batch;
    if (!b) {
        set_error("out of host memory");
        return ADR_ENOMEM;
    }
    auto fail = [&](adr_status st) {
        adr_batch_destroy(b);
        return st;
    };
    b->hs.assign(probs, probs + n);
    b->stream = static_cast<cudaStream_t>(stream);
    std::vector<double> tols(n);
    std::vector<int> maxit(n);
    for (int i = 0; i < n; ++i) {
        const Problem& p = probs[i]->p;
        b->dts.push_back(p.opts.dt > 0 ? p.opts.dt : default_dt(p, p.sigma));
        tols[i] = p.opts.tol;
        maxit[i] = p.opts.max_iter;
    }
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) ||
        (e = cudaEventCreate(&b->ev0)) || (e = cudaEventCreate(&b->ev1)))
        return fail(cuda_fail(e, "batch stream/events"));
    adr_status s = build_batch(b, tols.data(), maxit.data());
    if (s) return fail(s);
    *out = b;
    return ADR_OK;
}

adr_status adr_batch_solve(adr_batch* b, const double* const* u_init, double* const* u_out,
                           double* const* u_iter_out, adr_stats* stats)
{
    g_err.clear();
    if (!b || !u_out) {
        set_error("NULL batch or output array");
        return ADR_EINVAL;
    }
    const int n = (int)b->hs.size();
    for (int i = 0; i < n; ++i)
        if (!u_out[i]) {
            set_error("NULL output grid in adr_batch_solve");
            return ADR_EINVAL;
        }
    std::vector<IterState> st(n);
    std::vector<double> piv(2 * (size_t)n, INFINITY);
    float ms = 0.f;
    adr_status s = on_batch_stream(b, [&]() -> adr_status {
        for (int i = 0; i < n; ++i) {
            adr_problem* h = b->hs[i];
            TRY(init_state(h, h->p.opts.init, u_init ? u_init[i] : nullptr));
            TRY(launch_state_reset(&h->p));
        }
        TRY(prepare_batch(b));
        TRY(batch_dev_reset(b->dev, b->stream));
        ADR_CUDA_TRY(cudaEventRecord(b->ev0, b->stream));
        ADR_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
        for (int i = 0; i < n; ++i)
            TRY(launch_finish(&b->hs[i]->p, u_out[i], u_iter_out ? u_iter_out[i] : nullptr,
                              b->hs[i]->p.opts.theta == 0.5));
        ADR_CUDA_TRY(cudaEventRecord(b->ev1, b->stream));
        for (int i = 0; i < n; ++i) {
            ADR_CUDA_TRY(cudaMemcpyAsync(&st[i], b->hs[i]->p.state, sizeof(IterState),
                                         cudaMemcpyDeviceToHost, b->stream));
            ADR_CUDA_TRY(cudaMemcpyAsync(&piv[2 * i], b->hs[i]->p.pivmin, 2 * sizeof(double),
                                         cudaMemcpyDeviceToHost, b->stream));
        }
        ADR_CUDA_TRY(cudaStreamSynchronize(b->stream));
        cudaEventElapsedTime(&ms, b->ev0, b->ev1);
        return ADR_OK;
    });
    if (s) return s;
    bool all = true;
    for (int i = 0; i < n; ++i) {
        adr_problem* h = b->hs[i];
        if ((!st[i].converged && h->p.opts.tol > 0.0) || !std::isfinite(st[i].rel)) all = false;
        if (stats) {
            stats[i].iters = st[i].iter;
            stats[i].rel_update = st[i].rel;
            stats[i].ms = ms;
            stats[i].line_dofs = (double)st[i].iter * (h->line_unknowns[0] + h->line_unknowns[1]);
            stats[i].dt = b->dts[i];
            stats[i].min_pivot = std::fmin(piv[2 * i], piv[2 * i + 1]);
            stats[i].max_correction = st[i].iter > 0 ? st[i].corr : 0.0;
            stats[i].fp32_steps = h->p.opts.prec == ADR_FP32_REFINE ? st[i].fp32_steps : 0;
        }
    }
    if (!all) {
        set_error("a problem of the batch reached max_iter before tol");
        return ADR_ENOCONV;
    }
    return ADR_OK;
}

adr_status adr_batch_autotune(adr_batch* b, int reps, int* rows_out, double* ms_out)
{
    g_err.clear();
    if (!b || reps < 1) {
        set_error("bad arguments to adr_batch_autotune");
        return ADR_EINVAL;
    }
    const int n = (int)b->hs.size();
    // every candidate runs exactly reps batched split steps from u = 0
    std::vector<double> tol0(n, 0.0), tols(n);
    std::vector<int> capped(n, reps), maxit(n);
    for (int i = 0; i < n; ++i) {
        tols[i] = b->hs[i]->p.opts.tol;
        maxit[i] = b->hs[i]->p.opts.max_iter;
    }
    auto set_rows = [&](int R) -> adr_status {
        for (adr_problem* h : b->hs) {
            Problem* p = &h->p;
            if (p->rows_per_thread == R && p->fam[0].iset[0].BS) continue;
            p->rows_per_thread = R;
            drop_graph(h);
            for (int fam = 0; fam < 2; ++fam) {
                release_groups(p, fam);
                TRY(setup_groups(p, fam, h->offs[fam]));
            }
        }
        return ADR_OK;
    };
    const int rows[3] = {4, 8, 16};
    int best_r = b->hs[0]->p.rows_per_thread;
    double best = 1e300;
    for (int R : rows) {
        TRY(set_rows(R));
        TRY(build_batch(b, tol0.data(), capped.data()));
        float ms = 0.f;
        adr_status s = on_batch_stream(b, [&]() -> adr_status {
            for (adr_problem* h : b->hs) {
                TRY(init_state(h, ADR_INIT_ZERO, nullptr));
                TRY(launch_state_reset(&h->p));
            }
            TRY(batch_dev_reset(b->dev, b->stream));
            ADR_CUDA_TRY(cudaEventRecord(b->ev0, b->stream));
            ADR_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
            ADR_CUDA_TRY(cudaEventRecord(b->ev1, b->stream));
            ADR_CUDA_TRY(cudaStreamSynchronize(b->stream));
            cudaEventElapsedTime(&ms, b->ev0, b->ev1);
            return ADR_OK;
        });
        TRY(s);
        if (ms < best) {
            best = ms;
            best_r = R;
        }
    }
    TRY(set_rows(best_r));
    TRY(build_batch(b, tols.data(), maxit.data()));
    if (rows_out) *rows_out = best_r;
    if (ms_out) *ms_out = best / reps;
    return ADR_OK;
}

adr_status adr_solve_batch(adr_problem* const* probs, int n, double* const* u_out, adr_stats* stats)
{
    adr_batch* b = nullptr;
    void* stream = (n > 0 && probs && probs[0]) ? (void*)probs[0]->p.stream : nullptr;
    adr_status s = adr_batch_create(probs, n, stream, &b);
    if (s) return s;
    s = adr_batch_solve(b, nullptr, u_out, nullptr, stats);
    std::string keep = g_err;
    adr_batch_destroy(b);
    g_err = keep;
    return s;
}

}  // extern "C"
