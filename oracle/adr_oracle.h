/*
 * FP64 CPU oracle of the directional diffusion splitting method for the 2D
 * advection-diffusion-reaction problem (Drebotiy & Shynkarenko, arXiv
 * 2411.11041).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may load it; the product library never links it and
 * shares no code, header or table with it.
 *
 * Conventions: grids are row-major [ny][nx] over nodes, boundary included.
 * Geometry is held in "index space" (xi, eta) = ((x-x0)/hx, (y-y0)/hy), so that
 * grid lines sit at integer coordinates.  Family 0 = B (integral curves of beta,
 * oriented along b), family 1 = G (integral curves of gamma, oriented along p).
 */
#ifndef ADR_ORACLE_H
#define ADR_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_problem orc_problem;

/* node classes */
enum { ORC_OUTSIDE = 0, ORC_DIRICHLET = 1, ORC_INTERIOR = 2 };
/* status codes (same meaning as the library's, own definitions) */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENOCONV = 4, ORC_EGEOM = 5 };

int orc_create(int nx, int ny, double x0, double y0, double x1, double y1,
               const unsigned char* mask, double mu, double sigma,
               const double* beta1, const double* beta2, const double* f,
               orc_problem** out);
void orc_destroy(orc_problem* p);

/* curve -> grid weighting: 0 = plain average (default), 1 = inverse gaps */
void orc_set_interp_weights(orc_problem* p, int mode);
/* 1D problems on the B lines: 0 = Galerkin (the paper, default), 1 = SUPG */
void orc_set_stabilization(orc_problem* p, int mode);

/* values between the families: 0 = through the grid (§6, default),
   1 = directly through the curves' crossings (the paper's conclusions);
   builds the crossing tables on first use.  Returns ORC_OK / ORC_EINVAL. */
int orc_set_transfer(orc_problem* p, int mode);
/* direct transfer: values at the nodes of to_fam from the other family's
   curve values */
void orc_transfer(const orc_problem* p, int to_fam, const double* from_vals, double* to_vals);
/* the crossing table of fam: per node (left, right) crossings with the other
   family along its curve: seg[2 n_nodes] (first node of the crossed segment,
   -1 = the curve's end, -2 = an end node of the curve), t, pos (element units
   along the curve) */
void orc_transfer_table(const orc_problem* p, int fam, int* seg, double* t, double* pos);
/* one substep's increments on family fam from values at its nodes */
double orc_sweep_line_values(const orc_problem* p, int fam, double theta, double dt,
                             const double* u_vals, double sig, const double* f_extra,
                             double fx_scale, double* d);

/* acceleration of the stationary iteration: 0 = none (default), 1..8 = the
   depth m of Anderson extrapolation over the last m steps.  Returns ORC_OK /
   ORC_EINVAL. */
int orc_set_anderson(orc_problem* p, int m);
/* the same extrapolation on a linear fixed-point map g(x) = T x + c of size n
   (T row-major n*n): iterates from x (overwritten) until |g(x) - x| / |g(x)|
   <= tol or max_iter maps; returns the number of maps applied, res[k] the
   relative update at map k */
int orc_anderson_linear(int n, int m, const double* T, const double* c, double* x, int max_iter,
                        double tol, double* res);

/* geometry queries */
int orc_const_beta(const orc_problem* p);
void orc_node_types(const orc_problem* p, unsigned char* out /* [ny*nx] */);
int orc_num_lines(const orc_problem* p, int fam);
int orc_num_line_nodes(const orc_problem* p, int fam);
/* off[n_lines+1], xi/eta/bnorm/fval[n_nodes], h[n_lines] */
void orc_lines(const orc_problem* p, int fam, int* off, double* xi, double* eta,
               double* bnorm, double* fval, double* h);
/* per grid node, 4 crossings (row left, row right, col down, col up):
   seg[4*ny*nx] (global index of the segment's first node, -1 = boundary),
   t[4*ny*nx], pos[4*ny*nx] (index coordinate of the crossing along the row/col) */
void orc_crossings(const orc_problem* p, int fam, int* seg, double* t, double* pos);

/* building blocks (each is one step of the method) */
double orc_bilinear(const orc_problem* p, const double* grid, double xi, double eta);
void orc_gather(const orc_problem* p, int fam, const double* grid, double* line_vals);
void orc_map_to_grid(const orc_problem* p, int fam, const double* line_vals, double* grid);
/* assemble the tridiagonal system of one line: rows 1..n-1 of the line (n-1 rows) */
int orc_line_system(const orc_problem* p, int fam, int line, double theta, double dt,
                    const double* u_line, double sigma_eff, const double* f_line,
                    double* a, double* b, double* c, double* r);
int orc_thomas(int n, const double* a, const double* b, const double* c,
               const double* r, double* x);
int orc_dense_lu_solve(int n, double* A /* n*n row-major, overwritten */, double* b);
/* d = line increments for a sweep (0 at line ends); returns min |pivot| */
double orc_sweep_lines(const orc_problem* p, int fam, double theta, double dt,
                       const double* u_grid, double sigma_eff, const double* f_grid,
                       const double* f_extra, double f_extra_scale, double* d);

/* one split step  u -> u_half -> u_next  (eq. SemiDiscrSplit) */
void orc_split_step(const orc_problem* p, double theta, double dt, double sigma_eff,
                    const double* f_extra, double f_extra_scale,
                    const double* u, double* u_half, double* u_next);

double orc_default_dt(const orc_problem* p, double sigma_eff);

/* stationary solve by pseudo-time marching.  init: 0 zero, 1 user, 2 paper u0 */
int orc_solve_stationary(const orc_problem* p, double theta, double dt, double tol,
                         int max_iter, int init, const double* u_init,
                         double sigma_eff, const double* f_extra, double f_extra_scale,
                         double* u_out, double* u_iter_out, int* iters, double* rel);
/* paper's initial state s(u0, v) = <l, v> (eq. u0stationary) */
void orc_paper_u0(const orc_problem* p, double* u0);

/* parabolic problem: mode 0 = one split step per time step (eq. SemiDiscrSplit),
   mode 1 = each implicit-Euler slice solved by the stationary iteration */
int orc_step_parabolic(const orc_problem* p, double dt, int nsteps, int mode,
                       double theta, double pseudo_dt, double tol, int max_iter,
                       double* u_inout, int* total_iters);

/* brute-force references */
int orc_q1_dense(int nx, int ny, double x0, double y0, double x1, double y1,
                 const unsigned char* mask, double mu, double sigma,
                 const double* beta1, const double* beta2, const double* f, double* u);
int orc_p1_dense(int nx, int ny, double x0, double y0, double x1, double y1,
                 const unsigned char* mask, double mu, double sigma,
                 const double* beta1, const double* beta2, const double* f, double* u);

#ifdef __cplusplus
}
#endif
#endif
