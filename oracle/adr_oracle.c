/*
 * FP64 CPU oracle of the directional diffusion splitting method
 * (Drebotiy & Shynkarenko, "Directional diffusion splitting method for
 * advection-diffusion-reaction model", arXiv 2411.11041).
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow, single-threaded reference that the
 * CUDA library is checked against.  Only the tests, the smoke check and the
 * bench's CPU-baseline leg load it.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * Each function follows one step of the method in the paper's order:
 *   domain and grid               §6 eq. BndBox and the M x N mesh
 *   fields b, gamma, p            §3
 *   curve families B and G        §6 eqs. cauchyStartSets, CauchyBeta, CauchyGamma
 *   1D FEM on every curve         §6 eqs. SemiDiscrSplit1Dbeta(1), SemiDiscrSplit1Dgamma(1)
 *   grid -> curve interpolation   §6.1 eqs. bilinInd, bilinInterp, bilinInterpComp
 *   curve -> grid interpolation   §6 (min/max crossing per grid-line segment)
 *   split time step               §5 eq. SemiDiscrSplit
 *   stationary start              §5 eq. u0stationary
 * Readings where the paper is silent are stated at the point of use.
 *
 * Parity unpinned: none of the functions below lacks a pin; the convergence
 * RATE of the converged iterate toward the 2D FEM solution is not fixed by the
 * paper and is only measured.
 */
#include "adr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* coordinates within SNAP_TOL (index units) of an integer are snapped to it */
#define SNAP_TOL 1e-9
/* element count n = ceil(|L| / h_s - NODE_TOL) */
#define NODE_TOL 1e-9
/* RK4 steps per curve spacing h_s along traced curves (step h_s / 2) */
#define TRACE_STEPS_PER_H 2
#define BISECT_ITERS 60

typedef struct {
    int g;      /* global index of the segment's first node; -1 = boundary */
    double t;   /* position inside the segment, 0..1 */
    double pos; /* index coordinate of the crossing along the grid line */
    int valid;
} crossing;

typedef struct {
    int n_lines, n_nodes, cap_lines, cap_nodes;
    int* off;
    double* h;
    double *xi, *eta, *bnorm, *fval;
    /* four crossings per grid node: row-left, row-right, col-down, col-up */
    crossing* cross;
    /* direct transfer (built on request): per node of this family, the
       nearest crossing with the other family's curves before and after it
       along its own curve (pos in element units along the curve) */
    crossing* xf;
} family;

struct orc_problem {
    int nx, ny;
    double x0, y0, x1, y1, hx, hy, hs;
    double mu, sigma;
    double *beta1, *beta2, *f;
    unsigned char* cell;  /* [(ny-1)*(nx-1)] active cells */
    unsigned char* ntype; /* [ny*nx] node classes */
    int const_beta;
    double bmax;
    int interp_weights; /* 0: plain average of the row and column values; 1: inverse-gap weights */
    int stabilize;      /* 0: Galerkin on the B lines (the paper); 1: SUPG on the B lines */
    int transfer;       /* 0: values between the families through the grid (§6); 1: directly */
    int anderson;       /* 0: plain stationary iteration; m >= 1: Anderson extrapolation, depth m */
    family fam[2];
};

/* ------------------------------------------------------------------ helpers */

static double snap(double v)
{
    double r = rint(v);
    return fabs(v - r) <= SNAP_TOL ? r : v;
}

static int cell_active(const orc_problem* p, int i, int r)
{
    if (i < 0 || r < 0 || i >= p->nx - 1 || r >= p->ny - 1) return 0;
    return p->cell[(size_t)r * (p->nx - 1) + i];
}

/* A point (snapped index coordinates) is interior to the staircase domain
 * Omega_h iff every grid cell whose closure contains it is active. */
static int interior_point(const orc_problem* p, double xi, double eta)
{
    if (!isfinite(xi) || !isfinite(eta)) return 0;
    if (xi < -1.0 || eta < -1.0 || xi > p->nx || eta > p->ny) return 0;
    double fx = floor(xi), fy = floor(eta);
    int i0 = (int)fx, i1 = (int)fx, r0 = (int)fy, r1 = (int)fy;
    if (xi == fx) i0 = (int)fx - 1;
    if (eta == fy) r0 = (int)fy - 1;
    for (int r = r0; r <= r1; ++r)
        for (int i = i0; i <= i1; ++i)
            if (!cell_active(p, i, r)) return 0;
    return 1;
}

/* §6.1 eqs. bilinInd, bilinInterp, bilinInterpComp.  The printed cell index
 * uses a ceiling (and x in place of y for i_y); read as i = min(floor(xi), k-1)
 * with lambda = xi - i, which picks the same cell off the grid lines and is
 * continuous on them.  Points outside the box extrapolate from the edge cell. */
static double bilin(const orc_problem* p, const double* g, double xi, double eta)
{
    int nx = p->nx, ny = p->ny;
    int i = (int)floor(xi), r = (int)floor(eta);
    if (i > nx - 2) i = nx - 2;
    if (i < 0) i = 0;
    if (r > ny - 2) r = ny - 2;
    if (r < 0) r = 0;
    double lx = xi - i, ly = eta - r;
    const double* r0 = g + (size_t)r * nx;
    const double* r1 = r0 + nx;
    double p11 = r0[i], p12 = r0[i + 1], p21 = r1[i], p22 = r1[i + 1];
    return (1.0 - ly) * (1.0 - lx) * p11 + (1.0 - ly) * lx * p12 +
           ly * (1.0 - lx) * p21 + ly * lx * p22;
}

double orc_bilinear(const orc_problem* p, const double* grid, double xi, double eta)
{
    return bilin(p, grid, xi, eta);
}

/* §3: b = beta/|beta|, gamma = (beta2, -beta1), p = gamma/|gamma|.  Family 0
 * follows b, family 1 follows p.  beta at a point is the bilinear interpolant
 * of the nodal field.  The point is given in index coordinates (xi, eta); the
 * returned direction is the physical unit vector. */
static int direction(const orc_problem* p, int fam, double xi, double eta,
                     double* dx, double* dy)
{
    double b1 = bilin(p, p->beta1, xi, eta), b2 = bilin(p, p->beta2, xi, eta);
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

/* one classical Runge-Kutta step of x' = dir(x) over an arc length ds
 * (eqs. CauchyBeta / CauchyGamma with the field normalised, so that the
 * curve parameter is arc length), carried out in index coordinates: the step
 * is (sx, sy) = (ds / hx, ds / hy) along the two axes. */
static int rk4(const orc_problem* p, int fam, double X, double Y, double sx, double sy,
               double* Xo, double* Yo)
{
    double k1x, k1y, k2x, k2y, k3x, k3y, k4x, k4y;
    if (direction(p, fam, X, Y, &k1x, &k1y)) return -1;
    if (direction(p, fam, X + 0.5 * sx * k1x, Y + 0.5 * sy * k1y, &k2x, &k2y)) return -1;
    if (direction(p, fam, X + 0.5 * sx * k2x, Y + 0.5 * sy * k2y, &k3x, &k3y)) return -1;
    if (direction(p, fam, X + sx * k3x, Y + sy * k3y, &k4x, &k4y)) return -1;
    *Xo = X + sx / 6.0 * (k1x + 2.0 * k2x + 2.0 * k3x + k4x);
    *Yo = Y + sy / 6.0 * (k1y + 2.0 * k2y + 2.0 * k3y + k4y);
    return 0;
}

/* ---------------------------------------------------------- line storage */

static int fam_reserve(family* F, int add_lines, int add_nodes)
{
    if (F->n_lines + add_lines + 1 > F->cap_lines) {
        int cap = (F->cap_lines ? F->cap_lines * 2 : 256);
        while (cap < F->n_lines + add_lines + 1) cap *= 2;
        int* off = realloc(F->off, sizeof(int) * cap);
        double* h = realloc(F->h, sizeof(double) * cap);
        if (!off || !h) return -1;
        F->off = off;
        F->h = h;
        F->cap_lines = cap;
    }
    if (F->n_nodes + add_nodes > F->cap_nodes) {
        int cap = (F->cap_nodes ? F->cap_nodes * 2 : 4096);
        while (cap < F->n_nodes + add_nodes) cap *= 2;
        double* a = realloc(F->xi, sizeof(double) * cap);
        if (!a) return -1;
        F->xi = a;
        a = realloc(F->eta, sizeof(double) * cap);
        if (!a) return -1;
        F->eta = a;
        a = realloc(F->bnorm, sizeof(double) * cap);
        if (!a) return -1;
        F->bnorm = a;
        a = realloc(F->fval, sizeof(double) * cap);
        if (!a) return -1;
        F->fval = a;
        F->cap_nodes = cap;
    }
    return 0;
}

/* nodal |beta| and f at a line node (O2: from the bilinear fields) */
static void node_data(const orc_problem* p, family* F, int k)
{
    double b1 = bilin(p, p->beta1, F->xi[k], F->eta[k]);
    double b2 = bilin(p, p->beta2, F->xi[k], F->eta[k]);
    F->bnorm[k] = sqrt(b1 * b1 + b2 * b2);
    F->fval[k] = bilin(p, p->f, F->xi[k], F->eta[k]);
}

static int elements_for(const orc_problem* p, double L)
{
    int n = (int)ceil(L / p->hs - NODE_TOL);
    return n < 1 ? 1 : n;
}

/* ------------------------------------------------ straight lines (const beta)
 * Reading of §6 (the paper leaves the number and spacing of the curves open):
 * for a constant field the integral curves are the lines
 *    B: { x : p.(x - x_ref) = k h_s },  G: { x : b.(x - x_ref) = k h_s },
 * x_ref = (x0, y0), h_s = min(hx, hy), each oriented along its own direction and
 * cut into the maximal sub-intervals that lie inside Omega_h; every sub-interval
 * is one 1D problem.  The parameter s is physical arc length along the line. */
static int emit_straight(orc_problem* p, family* F, double ox, double oy,
                         double dx, double dy, double sa, double sb)
{
    double L = sb - sa;
    int n = elements_for(p, L);
    if (fam_reserve(F, 1, n + 1)) return -1;
    int base = F->n_nodes;
    for (int j = 0; j <= n; ++j) {
        double s = (j == n) ? sb : sa + j * (L / n);
        F->xi[base + j] = snap((ox + s * dx) / p->hx);
        F->eta[base + j] = snap((oy + s * dy) / p->hy);
        node_data(p, F, base + j);
    }
    F->off[F->n_lines] = base;
    F->h[F->n_lines] = L / n;
    F->n_lines += 1;
    F->n_nodes += n + 1;
    F->off[F->n_lines] = F->n_nodes;
    return 0;
}

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

static int build_straight(orc_problem* p, int fam)
{
    family* F = &p->fam[fam];
    double b1 = 0, b2 = 0;
    for (size_t k = 0; k < (size_t)p->nx * p->ny; ++k)
        if (p->ntype[k] != ORC_OUTSIDE) {
            b1 = p->beta1[k];
            b2 = p->beta2[k];
            break;
        }
    double nb = sqrt(b1 * b1 + b2 * b2);
    double bx = b1 / nb, by = b2 / nb, px = by, py = -bx;
    double dx = fam == 0 ? bx : px, dy = fam == 0 ? by : py;
    double nx_ = fam == 0 ? px : bx, ny_ = fam == 0 ? py : by;
    double W = p->x1 - p->x0, H = p->y1 - p->y0;
    double qc[4] = {0.0, nx_ * W, ny_ * H, nx_ * W + ny_ * H};
    double qmin = qc[0], qmax = qc[0];
    for (int c = 1; c < 4; ++c) {
        if (qc[c] < qmin) qmin = qc[c];
        if (qc[c] > qmax) qmax = qc[c];
    }
    long kmin = (long)ceil(qmin / p->hs - 1e-9), kmax = (long)floor(qmax / p->hs + 1e-9);
    double* bp = malloc(sizeof(double) * (size_t)(p->nx + p->ny + 4));
    if (!bp) return -1;
    F->off = NULL;
    if (fam_reserve(F, 1, 0)) return -1;
    F->off[0] = 0;
    for (long k = kmin; k <= kmax; ++k) {
        double ox = k * p->hs * nx_, oy = k * p->hs * ny_; /* offset of the base point */
        /* clip to the box in s */
        double slo = -INFINITY, shi = INFINITY;
        double lim[2][2] = {{0.0, W}, {0.0, H}};
        double o[2] = {ox, oy}, d[2] = {dx, dy};
        int empty = 0;
        for (int a = 0; a < 2; ++a) {
            if (d[a] == 0.0) {
                double c = snap(o[a] / (a == 0 ? p->hx : p->hy));
                double top = (a == 0 ? p->nx - 1 : p->ny - 1);
                if (c < 0.0 || c > top) empty = 1;
            } else {
                double s0 = (lim[a][0] - o[a]) / d[a], s1 = (lim[a][1] - o[a]) / d[a];
                if (s0 > s1) {
                    double t = s0;
                    s0 = s1;
                    s1 = t;
                }
                if (s0 > slo) slo = s0;
                if (s1 < shi) shi = s1;
            }
        }
        if (empty || !(shi > slo)) continue;
        /* breakpoints: crossings with every grid line inside [slo, shi] */
        int nb_ = 0;
        bp[nb_++] = slo;
        bp[nb_++] = shi;
        for (int a = 0; a < 2; ++a) {
            if (d[a] == 0.0) continue;
            double hh = (a == 0 ? p->hx : p->hy);
            double c0 = (o[a] + slo * d[a]) / hh, c1 = (o[a] + shi * d[a]) / hh;
            double lo = c0 < c1 ? c0 : c1, hi = c0 < c1 ? c1 : c0;
            for (long g = (long)ceil(lo - 1e-9); g <= (long)floor(hi + 1e-9); ++g) {
                double s = (g * hh - o[a]) / d[a];
                if (s > slo && s < shi) bp[nb_++] = s;
            }
        }
        qsort(bp, nb_, sizeof(double), cmp_double);
        double run_a = 0.0, run_b = 0.0;
        int open = 0;
        for (int m = 0; m + 1 < nb_; ++m) {
            double s0 = bp[m], s1 = bp[m + 1];
            if (!(s1 - s0 > 1e-9 * p->hs)) continue;
            double sm = 0.5 * (s0 + s1);
            double xi = snap((ox + sm * dx) / p->hx), eta = snap((oy + sm * dy) / p->hy);
            if (interior_point(p, xi, eta)) {
                if (!open) {
                    run_a = s0;
                    open = 1;
                }
                run_b = s1;
            } else if (open) {
                if (emit_straight(p, F, ox, oy, dx, dy, run_a, run_b)) return -1;
                open = 0;
            }
        }
        if (open && emit_straight(p, F, ox, oy, dx, dy, run_a, run_b)) return -1;
    }
    free(bp);
    return 0;
}

/* ------------------------------------------------------ curved families
 * §6 eq. cauchyStartSets: inflow parts of the boundary, n.beta < 0 (B) or
 * n.gamma < 0 (G).  Reading (the paper leaves the seeds open): the boundary of
 * the staircase domain is walked loop by loop, counter-clockwise (domain on
 * the left), each loop starting at its lowest-leftmost bottom edge, loops in
 * order of that edge.  Every boundary edge e carries the transverse inflow
 * measure w_e = max(0, -n_e . dir(mid_e)) |e| with dir from the nodal mean of
 * beta over the edge; seeds sit where the cumulative measure reaches
 * (k + 1/2) h_s, linearly inside the edge.  From each seed the curve is traced
 * (eqs. CauchyBeta / CauchyGamma) with RK4 steps of h_s/2 in arc length until
 * it leaves the interior of Omega_h; the exit is located by bisection. */

/* boundary edge orientation: +1 / -1 along the axis, 0 = not a boundary edge */
static int hedge_dir(const orc_problem* p, int i, int r)
{
    int up = cell_active(p, i, r), dn = cell_active(p, i, r - 1);
    return up && !dn ? 1 : (dn && !up ? -1 : 0);
}
static int vedge_dir(const orc_problem* p, int i, int r)
{
    int lf = cell_active(p, i - 1, r), rt = cell_active(p, i, r);
    return lf && !rt ? 1 : (rt && !lf ? -1 : 0);
}

/* does a boundary edge leave node (i, r) in direction d (0:+x 1:+y 2:-x 3:-y)? */
static int out_edge(const orc_problem* p, int i, int r, int d)
{
    switch (d) {
    case 0: return i <= p->nx - 2 && hedge_dir(p, i, r) == 1;
    case 1: return r <= p->ny - 2 && vedge_dir(p, i, r) == 1;
    case 2: return i >= 1 && hedge_dir(p, i - 1, r) == -1;
    default: return r >= 1 && vedge_dir(p, i, r - 1) == -1;
    }
}

static const int DXI[4] = {1, 0, -1, 0}, DETA[4] = {0, 1, 0, -1};

typedef struct {
    int i, r, d;
} bedge;

static int boundary_loops(const orc_problem* p, bedge** out, int* count)
{
    int nx = p->nx, ny = p->ny;
    unsigned char* vis_h = calloc((size_t)ny * (nx - 1), 1);
    unsigned char* vis_v = calloc((size_t)nx * (ny - 1), 1);
    int cap = 4 * (nx + ny) + 16, n = 0;
    bedge* E = malloc(sizeof(bedge) * cap);
    if (!vis_h || !vis_v || !E) return -1;
    long total = 0;
    for (int r = 0; r < ny; ++r)
        for (int i = 0; i < nx - 1; ++i)
            if (hedge_dir(p, i, r)) total++;
    for (int r = 0; r < ny - 1; ++r)
        for (int i = 0; i < nx; ++i)
            if (vedge_dir(p, i, r)) total++;
    for (int r0 = 0; r0 < ny; ++r0)
        for (int i0 = 0; i0 < nx - 1; ++i0) {
            if (hedge_dir(p, i0, r0) != 1 || vis_h[(size_t)r0 * (nx - 1) + i0]) continue;
            int i = i0, r = r0, d = 0;
            long steps = 0;
            for (;;) {
                unsigned char* mark;
                if (d == 0) mark = &vis_h[(size_t)r * (nx - 1) + i];
                else if (d == 2) mark = &vis_h[(size_t)r * (nx - 1) + i - 1];
                else if (d == 1) mark = &vis_v[(size_t)r * nx + i];
                else mark = &vis_v[(size_t)(r - 1) * nx + i];
                if (*mark) break; /* back at an edge already walked: loop closed */
                *mark = 1;
                if (n == cap) {
                    cap *= 2;
                    bedge* e2 = realloc(E, sizeof(bedge) * cap);
                    if (!e2) return -1;
                    E = e2;
                }
                E[n].i = i;
                E[n].r = r;
                E[n].d = d;
                n++;
                i += DXI[d];
                r += DETA[d];
                /* turn preference at the end node: left, straight, right */
                int nd = -1;
                int pref[3] = {(d + 1) & 3, d, (d + 3) & 3};
                for (int q = 0; q < 3; ++q)
                    if (out_edge(p, i, r, pref[q])) {
                        nd = pref[q];
                        break;
                    }
                if (nd < 0 || ++steps > total + 4) break;
                d = nd;
            }
        }
    free(vis_h);
    free(vis_v);
    *out = E;
    *count = n;
    return 0;
}

/* trace one curve from a seed; stores the RK4 points (index coordinates) */
typedef struct {
    double *X, *Y;
    int n, cap;
} trace_buf;

static int trace_curve(const orc_problem* p, int fam, double X0, double Y0,
                       trace_buf* tb, double* Lout)
{
    double ds = p->hs / TRACE_STEPS_PER_H;
    double sx = ds / p->hx, sy = ds / p->hy; /* the step in index units */
    double cap_len = 10.0 * 2.0 * ((p->x1 - p->x0) + (p->y1 - p->y0));
    tb->n = 0;
    double X = X0, Y = Y0;
    for (;;) {
        if (tb->n == tb->cap) {
            tb->cap = tb->cap ? tb->cap * 2 : 1024;
            double* a = realloc(tb->X, sizeof(double) * tb->cap);
            double* b = realloc(tb->Y, sizeof(double) * tb->cap);
            if (!a || !b) return -1;
            tb->X = a;
            tb->Y = b;
        }
        tb->X[tb->n] = X;
        tb->Y[tb->n] = Y;
        tb->n++;
        double Xn, Yn;
        if (rk4(p, fam, X, Y, sx, sy, &Xn, &Yn)) return ORC_EGEOM;
        if (interior_point(p, snap(Xn), snap(Yn))) {
            X = Xn;
            Y = Yn;
            if ((tb->n) * ds > cap_len) return ORC_EGEOM; /* closed curve */
            continue;
        }
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < BISECT_ITERS; ++it) {
            double mid = 0.5 * (lo + hi);
            if (rk4(p, fam, X, Y, mid * sx, mid * sy, &Xn, &Yn)) return ORC_EGEOM;
            if (interior_point(p, snap(Xn), snap(Yn))) lo = mid;
            else hi = mid;
        }
        double Xe = X, Ye = Y;
        if (lo > 0.0 && rk4(p, fam, X, Y, lo * sx, lo * sy, &Xe, &Ye)) return ORC_EGEOM;
        if (tb->n == tb->cap) {
            tb->cap *= 2;
            double* a = realloc(tb->X, sizeof(double) * tb->cap);
            double* b = realloc(tb->Y, sizeof(double) * tb->cap);
            if (!a || !b) return -1;
            tb->X = a;
            tb->Y = b;
        }
        tb->X[tb->n] = Xe;
        tb->Y[tb->n] = Ye;
        tb->n++;
        *Lout = (tb->n - 2) * ds + lo * ds;
        return 0;
    }
}

static int build_curved(orc_problem* p, int fam)
{
    family* F = &p->fam[fam];
    bedge* E = NULL;
    int ne = 0;
    if (boundary_loops(p, &E, &ne)) return -1;
    if (fam_reserve(F, 1, 0)) return -1;
    F->off[0] = 0;
    double ds = p->hs / TRACE_STEPS_PER_H;
    double cum = 0.0;
    long k = 0;
    trace_buf tb = {0};
    for (int e = 0; e < ne; ++e) {
        int i = E[e].i, r = E[e].r, d = E[e].d;
        int ib = i + DXI[d], rb = r + DETA[d];
        size_t A = (size_t)r * p->nx + i, B = (size_t)rb * p->nx + ib;
        double m1 = 0.5 * (p->beta1[A] + p->beta1[B]), m2 = 0.5 * (p->beta2[A] + p->beta2[B]);
        double nm = sqrt(m1 * m1 + m2 * m2);
        if (!(nm > 0.0)) return ORC_EGEOM;
        double vx = fam == 0 ? m1 / nm : m2 / nm, vy = fam == 0 ? m2 / nm : -m1 / nm;
        double nxo = (double)DETA[d], nyo = (double)(-DXI[d]); /* outward normal */
        double len = (d & 1) ? p->hy : p->hx;
        double w = -(nxo * vx + nyo * vy) * len;
        if (!(w > 0.0)) continue;
        while ((k + 0.5) * p->hs < cum + w) {
            double phi = ((k + 0.5) * p->hs - cum) / w;
            double X0 = i + phi * DXI[d], Y0 = r + phi * DETA[d]; /* index coordinates */
            double L = 0.0;
            int st = trace_curve(p, fam, X0, Y0, &tb, &L);
            if (st) return st;
            int n = elements_for(p, L);
            if (fam_reserve(F, 1, n + 1)) return -1;
            int base = F->n_nodes, M = tb.n - 2; /* tb holds P_0..P_M and the exit */
            for (int j = 0; j <= n; ++j) {
                double X, Y;
                if (j == n) {
                    X = tb.X[tb.n - 1];
                    Y = tb.Y[tb.n - 1];
                } else {
                    double s = j * (L / n);
                    int q = (int)floor(s / ds);
                    if (q > M) q = M;
                    double s0 = q * ds, s1 = (q < M) ? (q + 1) * ds : L;
                    double fr = (s1 > s0) ? (s - s0) / (s1 - s0) : 0.0;
                    X = tb.X[q] + fr * (tb.X[q + 1] - tb.X[q]);
                    Y = tb.Y[q] + fr * (tb.Y[q + 1] - tb.Y[q]);
                }
                F->xi[base + j] = snap(X);
                F->eta[base + j] = snap(Y);
                node_data(p, F, base + j);
            }
            F->off[F->n_lines] = base;
            F->h[F->n_lines] = L / n;
            F->n_lines += 1;
            F->n_nodes += n + 1;
            F->off[F->n_lines] = F->n_nodes;
            k++;
        }
        cum += w;
    }
    free(tb.X);
    free(tb.Y);
    free(E);
    return 0;
}

/* ------------------------------------------------ curve -> grid structure
 * §6 (interpolation through the intermediate grid): every grid line is cut
 * into segments by the grid nodes; each segment keeps its crossing with the
 * smallest and with the largest coordinate.  A crossing exactly on a grid node
 * is recorded on both adjacent segments.  Reading where a segment holds no
 * crossing: the search moves on to the next segment; a non-interior grid node
 * met first stands for the boundary, value 0. */

static int key_less_min(const crossing* a, const crossing* b)
{
    if (a->pos != b->pos) return a->pos < b->pos;
    if (a->g != b->g) return a->g < b->g;
    return a->t < b->t;
}
static int key_less_max(const crossing* a, const crossing* b)
{
    if (a->pos != b->pos) return a->pos > b->pos;
    if (a->g != b->g) return a->g < b->g;
    return a->t < b->t;
}

typedef struct {
    crossing mn, mx;
} seg_slot;

static void record(seg_slot* slots, int nseg, double pos, int g, double t)
{
    crossing c = {g, t, pos, 1};
    double fp = floor(pos);
    int e0 = (int)fp, e1 = (int)fp;
    if (pos == fp) e0 = (int)fp - 1;
    for (int e = e0; e <= e1; ++e) {
        if (e < 0 || e >= nseg) continue;
        seg_slot* s = &slots[e];
        if (!s->mn.valid || key_less_min(&c, &s->mn)) s->mn = c;
        if (!s->mx.valid || key_less_max(&c, &s->mx)) s->mx = c;
    }
}

static int build_crossings(orc_problem* p, int fam)
{
    family* F = &p->fam[fam];
    int nx = p->nx, ny = p->ny;
    seg_slot* rows = calloc((size_t)ny * (nx - 1), sizeof(seg_slot));
    seg_slot* cols = calloc((size_t)nx * (ny - 1), sizeof(seg_slot));
    F->cross = calloc((size_t)4 * nx * ny, sizeof(crossing));
    int uncovered = 0;
    if (!rows || !cols || !F->cross) {
        free(rows);
        free(cols);
        return -1;
    }
    for (int l = 0; l < F->n_lines; ++l)
        for (int g = F->off[l]; g + 1 < F->off[l + 1]; ++g) {
            double xa = F->xi[g], xb = F->xi[g + 1], ea = F->eta[g], eb = F->eta[g + 1];
            /* crossings with grid rows eta = r */
            if (ea == eb) {
                if (ea == floor(ea) && ea >= 0 && ea <= ny - 1) {
                    int r = (int)ea;
                    record(rows + (size_t)r * (nx - 1), nx - 1, xa, g, 0.0);
                    record(rows + (size_t)r * (nx - 1), nx - 1, xb, g, 1.0);
                }
            } else {
                double lo = ea < eb ? ea : eb, hi = ea < eb ? eb : ea;
                for (long r = (long)ceil(lo); r <= (long)floor(hi); ++r) {
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
                    record(rows + (size_t)r * (nx - 1), nx - 1, pos, g, t);
                }
            }
            /* crossings with grid columns xi = i */
            if (xa == xb) {
                if (xa == floor(xa) && xa >= 0 && xa <= nx - 1) {
                    int i = (int)xa;
                    record(cols + (size_t)i * (ny - 1), ny - 1, ea, g, 0.0);
                    record(cols + (size_t)i * (ny - 1), ny - 1, eb, g, 1.0);
                }
            } else {
                double lo = xa < xb ? xa : xb, hi = xa < xb ? xb : xa;
                for (long i = (long)ceil(lo); i <= (long)floor(hi); ++i) {
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
                    record(cols + (size_t)i * (ny - 1), ny - 1, pos, g, t);
                }
            }
        }
    /* nearest crossing on each side of every interior node */
    for (int r = 1; r < ny - 1; ++r)
        for (int i = 1; i < nx - 1; ++i) {
            size_t node = (size_t)r * nx + i;
            if (p->ntype[node] != ORC_INTERIOR) continue;
            crossing* c = &F->cross[4 * node];
            crossing bnd = {-1, 0.0, 0.0, 1};
            const seg_slot* row = rows + (size_t)r * (nx - 1);
            const seg_slot* col = cols + (size_t)i * (ny - 1);
            for (int e = i - 1;; --e) { /* row, left */
                if (row[e].mx.valid) { c[0] = row[e].mx; break; }
                if (p->ntype[(size_t)r * nx + e] != ORC_INTERIOR) { c[0] = bnd; c[0].pos = e; break; }
            }
            for (int e = i;; ++e) { /* row, right */
                if (row[e].mn.valid) { c[1] = row[e].mn; break; }
                if (p->ntype[(size_t)r * nx + e + 1] != ORC_INTERIOR) { c[1] = bnd; c[1].pos = e + 1; break; }
            }
            for (int e = r - 1;; --e) { /* column, down */
                if (col[e].mx.valid) { c[2] = col[e].mx; break; }
                if (p->ntype[(size_t)e * nx + i] != ORC_INTERIOR) { c[2] = bnd; c[2].pos = e; break; }
            }
            for (int e = r;; ++e) { /* column, up */
                if (col[e].mn.valid) { c[3] = col[e].mn; break; }
                if (p->ntype[(size_t)(e + 1) * nx + i] != ORC_INTERIOR) { c[3] = bnd; c[3].pos = e + 1; break; }
            }
            /* no curve of the family on either grid line through the node
               before the boundary: the family does not cover the node (the
               curves of each family must cover the domain, §3 and §6) */
            if (c[0].g == -1 && c[1].g == -1 && c[2].g == -1 && c[3].g == -1) uncovered = 1;
        }
    free(rows);
    free(cols);
    return uncovered;
}

/* ------------------------------------ direct transfer between the families
 * The paper's conclusions propose to carry values between the two sets of
 * orthogonal curves through the points where they cross, without the
 * intermediate grid and its bilinear interpolation.  Reading: every crossing
 * of a target curve's polyline with a source curve's polyline is found (the
 * two segments share a grid cell: each source segment is listed in the cells
 * its bounding box covers, and a pair is taken in the cell that holds its
 * crossing point, so that it counts once).  Along the target curve every
 * element keeps its crossing of smallest and of largest position (ties: the
 * smaller source segment, then the smaller position inside it), a crossing on
 * a node counting for both of its elements.  A target node takes the value
 * linear in arc length between the nearest crossing at or before it and the
 * nearest at or after it; an element without a crossing passes the search
 * on, and the curve's end (on the boundary, u = 0) stands in where a side has
 * none.  The value at a crossing is linear along the source segment. */

static double cross_value(const crossing* c, const double* v);

/* crossing of the segments A-B and C-D (index coordinates):
 * A + a (B - A) = C + b (D - C) with 0 <= a, b <= 1; parallel segments give none */
static int seg_cross(double ax, double ay, double bx, double by, double cx, double cy,
                     double dx, double dy, double* a, double* b)
{
    double ex = bx - ax, ey = by - ay, fx = dx - cx, fy = dy - cy;
    double det = ex * fy - ey * fx;
    if (det == 0.0) return 0;
    double gx = cx - ax, gy = cy - ay;
    double aa = (gx * fy - gy * fx) / det;
    double bb = (gx * ey - gy * ex) / det;
    if (!(aa >= 0.0 && aa <= 1.0 && bb >= 0.0 && bb <= 1.0)) return 0;
    *a = aa;
    *b = bb;
    return 1;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* crossing tables of the target family tf with the source family 1 - tf */
static int build_transfer(orc_problem* p, int tf)
{
    family* T = &p->fam[tf];
    const family* S = &p->fam[1 - tf];
    int ncx = p->nx - 1, ncy = p->ny - 1;
    size_t ncell = (size_t)ncx * ncy;
    int* cnt = calloc(ncell + 1, sizeof(int));
    if (!cnt) return -1;
    /* source segments by cell (CSR), in segment order within a cell */
    for (int l = 0; l < S->n_lines; ++l)
        for (int g = S->off[l]; g + 1 < S->off[l + 1]; ++g) {
            int i0 = clampi((int)floor(fmin(S->xi[g], S->xi[g + 1])), 0, ncx - 1);
            int i1 = clampi((int)floor(fmax(S->xi[g], S->xi[g + 1])), 0, ncx - 1);
            int r0 = clampi((int)floor(fmin(S->eta[g], S->eta[g + 1])), 0, ncy - 1);
            int r1 = clampi((int)floor(fmax(S->eta[g], S->eta[g + 1])), 0, ncy - 1);
            for (int r = r0; r <= r1; ++r)
                for (int i = i0; i <= i1; ++i) cnt[(size_t)r * ncx + i + 1]++;
        }
    for (size_t c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
    int* fill = malloc(sizeof(int) * (ncell + 1));
    int* list = malloc(sizeof(int) * ((size_t)cnt[ncell] + 1));
    if (!fill || !list) {
        free(cnt);
        free(fill);
        free(list);
        return -1;
    }
    memcpy(fill, cnt, sizeof(int) * (ncell + 1));
    for (int l = 0; l < S->n_lines; ++l)
        for (int g = S->off[l]; g + 1 < S->off[l + 1]; ++g) {
            int i0 = clampi((int)floor(fmin(S->xi[g], S->xi[g + 1])), 0, ncx - 1);
            int i1 = clampi((int)floor(fmax(S->xi[g], S->xi[g + 1])), 0, ncx - 1);
            int r0 = clampi((int)floor(fmin(S->eta[g], S->eta[g + 1])), 0, ncy - 1);
            int r1 = clampi((int)floor(fmax(S->eta[g], S->eta[g + 1])), 0, ncy - 1);
            for (int r = r0; r <= r1; ++r)
                for (int i = i0; i <= i1; ++i) list[fill[(size_t)r * ncx + i]++] = g;
        }
    free(fill);
    int nmax = 1;
    for (int l = 0; l < T->n_lines; ++l)
        if (T->off[l + 1] - T->off[l] > nmax) nmax = T->off[l + 1] - T->off[l];
    seg_slot* slots = calloc((size_t)nmax, sizeof(seg_slot));
    free(T->xf);
    T->xf = calloc((size_t)2 * T->n_nodes + 2, sizeof(crossing));
    if (!slots || !T->xf) {
        free(cnt);
        free(list);
        free(slots);
        return -1;
    }
    for (int l = 0; l < T->n_lines; ++l) {
        int base = T->off[l], n = T->off[l + 1] - base - 1; /* n elements */
        if (n < 2) continue;
        memset(slots, 0, sizeof(seg_slot) * n);
        for (int e = 0; e < n; ++e) {
            int a0 = base + e;
            double ax = T->xi[a0], ay = T->eta[a0], bx = T->xi[a0 + 1], by = T->eta[a0 + 1];
            int i0 = clampi((int)floor(fmin(ax, bx)), 0, ncx - 1), i1 = clampi((int)floor(fmax(ax, bx)), 0, ncx - 1);
            int r0 = clampi((int)floor(fmin(ay, by)), 0, ncy - 1), r1 = clampi((int)floor(fmax(ay, by)), 0, ncy - 1);
            for (int r = r0; r <= r1; ++r)
                for (int i = i0; i <= i1; ++i) {
                    size_t c = (size_t)r * ncx + i;
                    for (int q = cnt[c]; q < cnt[c + 1]; ++q) {
                        int g = list[q];
                        double a, b;
                        if (!seg_cross(ax, ay, bx, by, S->xi[g], S->eta[g], S->xi[g + 1], S->eta[g + 1], &a, &b))
                            continue;
                        double px = ax + a * (bx - ax), py = ay + a * (by - ay);
                        if (clampi((int)floor(px), 0, ncx - 1) != i || clampi((int)floor(py), 0, ncy - 1) != r)
                            continue; /* counted in the cell that holds the crossing */
                        record(slots, n, e + a, g, b);
                    }
                }
        }
        /* nearest crossing on each side of every interior node of the curve */
        for (int k = 1; k < n; ++k) {
            crossing* c = &T->xf[2 * (size_t)(base + k)];
            crossing bnd = {-1, 0.0, 0.0, 1};
            c[0] = bnd;
            c[1] = bnd;
            c[1].pos = n;
            for (int e = k - 1; e >= 0; --e)
                if (slots[e].mx.valid) {
                    c[0] = slots[e].mx;
                    break;
                }
            for (int e = k; e < n; ++e)
                if (slots[e].mn.valid) {
                    c[1] = slots[e].mn;
                    break;
                }
        }
    }
    free(cnt);
    free(list);
    free(slots);
    return 0;
}

int orc_set_transfer(orc_problem* p, int mode)
{
    if (mode != 0 && mode != 1) return ORC_EINVAL;
    if (mode == 1 && (!p->fam[0].xf || !p->fam[1].xf)) {
        if (build_transfer(p, 0) || build_transfer(p, 1)) return ORC_ENOMEM;
    }
    p->transfer = mode;
    return ORC_OK;
}

/* values at the nodes of family to_fam from the curve values of the other
 * family, through the crossing tables (both ends of a curve get 0) */
void orc_transfer(const orc_problem* p, int to_fam, const double* from_vals, double* to_vals)
{
    const family* T = &p->fam[to_fam];
    for (int l = 0; l < T->n_lines; ++l) {
        int a = T->off[l], b = T->off[l + 1] - 1;
        for (int k = a; k <= b; ++k) {
            if (k == a || k == b || !T->xf) {
                to_vals[k] = 0.0;
                continue;
            }
            const crossing* c = &T->xf[2 * (size_t)k];
            double vL = cross_value(&c[0], from_vals), vR = cross_value(&c[1], from_vals);
            if (c[1].pos == c[0].pos) {
                to_vals[k] = vL;
            } else {
                double w = ((k - a) - c[0].pos) / (c[1].pos - c[0].pos);
                to_vals[k] = (1.0 - w) * vL + w * vR;
            }
        }
    }
}

void orc_transfer_table(const orc_problem* p, int fam, int* seg, double* t, double* pos)
{
    const family* F = &p->fam[fam];
    for (size_t k = 0; k < 2 * (size_t)F->n_nodes; ++k) {
        const crossing* c = F->xf ? &F->xf[k] : NULL;
        seg[k] = (c && c->valid) ? c->g : -2;
        t[k] = (c && c->valid) ? c->t : 0.0;
        pos[k] = (c && c->valid) ? c->pos : 0.0;
    }
}

/* ------------------------------------------------------------- create */

int orc_create(int nx, int ny, double x0, double y0, double x1, double y1,
               const unsigned char* mask, double mu, double sigma,
               const double* beta1, const double* beta2, const double* f,
               orc_problem** out)
{
    *out = NULL;
    if (nx < 3 || ny < 3 || !(x1 > x0) || !(y1 > y0) || !(mu > 0) || !(sigma > 0))
        return ORC_EINVAL;
    orc_problem* p = calloc(1, sizeof(orc_problem));
    if (!p) return ORC_ENOMEM;
    size_t N = (size_t)nx * ny;
    p->nx = nx;
    p->ny = ny;
    p->x0 = x0;
    p->y0 = y0;
    p->x1 = x1;
    p->y1 = y1;
    p->hx = (x1 - x0) / (nx - 1);
    p->hy = (y1 - y0) / (ny - 1);
    p->hs = p->hx < p->hy ? p->hx : p->hy;
    p->mu = mu;
    p->sigma = sigma;
    p->beta1 = malloc(N * sizeof(double));
    p->beta2 = malloc(N * sizeof(double));
    p->f = malloc(N * sizeof(double));
    p->cell = calloc((size_t)(nx - 1) * (ny - 1), 1);
    p->ntype = calloc(N, 1);
    if (!p->beta1 || !p->beta2 || !p->f || !p->cell || !p->ntype) {
        orc_destroy(p);
        return ORC_ENOMEM;
    }
    memcpy(p->beta1, beta1, N * sizeof(double));
    memcpy(p->beta2, beta2, N * sizeof(double));
    memcpy(p->f, f, N * sizeof(double));
    /* domain: a cell is active when its four corners are in the mask; Omega_h
       is their union; a node of Omega_h is interior when all four cells around
       it are active, otherwise it carries the Dirichlet condition (§2, BVP1). */
    int any = 0;
    for (int r = 0; r < ny - 1; ++r)
        for (int i = 0; i < nx - 1; ++i) {
            size_t a = (size_t)r * nx + i;
            int on = mask[a] && mask[a + 1] && mask[a + nx] && mask[a + nx + 1];
            p->cell[(size_t)r * (nx - 1) + i] = (unsigned char)on;
            any |= on;
        }
    if (!any) {
        orc_destroy(p);
        return ORC_EINVAL;
    }
    for (int r = 0; r < ny; ++r)
        for (int i = 0; i < nx; ++i) {
            int c00 = cell_active(p, i - 1, r - 1), c10 = cell_active(p, i, r - 1);
            int c01 = cell_active(p, i - 1, r), c11 = cell_active(p, i, r);
            int t = ORC_OUTSIDE;
            if (c00 || c10 || c01 || c11) t = (c00 && c10 && c01 && c11) ? ORC_INTERIOR : ORC_DIRICHLET;
            p->ntype[(size_t)r * nx + i] = (unsigned char)t;
        }
    /* constant field test and max |beta| over the nodes of Omega_h */
    int first = 1, cst = 1;
    double c1 = 0, c2 = 0, bmax = 0;
    for (size_t k = 0; k < N; ++k) {
        if (p->ntype[k] == ORC_OUTSIDE) continue;
        double nb = sqrt(beta1[k] * beta1[k] + beta2[k] * beta2[k]);
        if (!(nb > 0) || !isfinite(nb) || !isfinite(f[k])) {
            orc_destroy(p);
            return ORC_EINVAL;
        }
        if (nb > bmax) bmax = nb;
        if (first) {
            c1 = beta1[k];
            c2 = beta2[k];
            first = 0;
        } else if (beta1[k] != c1 || beta2[k] != c2) cst = 0;
    }
    p->const_beta = cst;
    p->bmax = bmax;
    for (int fam = 0; fam < 2; ++fam) {
        int st = cst ? build_straight(p, fam) : build_curved(p, fam);
        if (st) {
            orc_destroy(p);
            return st > 0 ? st : ORC_ENOMEM;
        }
        if (p->fam[fam].n_lines == 0) { /* no inflow boundary: no curve of the family */
            orc_destroy(p);
            return ORC_EGEOM;
        }
        st = build_crossings(p, fam);
        if (st) {
            orc_destroy(p);
            return st < 0 ? ORC_ENOMEM : ORC_EGEOM;
        }
    }
    *out = p;
    return ORC_OK;
}

void orc_destroy(orc_problem* p)
{
    if (!p) return;
    for (int k = 0; k < 2; ++k) {
        family* F = &p->fam[k];
        free(F->off);
        free(F->h);
        free(F->xi);
        free(F->eta);
        free(F->bnorm);
        free(F->fval);
        free(F->cross);
        free(F->xf);
    }
    free(p->beta1);
    free(p->beta2);
    free(p->f);
    free(p->cell);
    free(p->ntype);
    free(p);
}

int orc_const_beta(const orc_problem* p) { return p->const_beta; }
void orc_set_interp_weights(orc_problem* p, int mode) { p->interp_weights = mode ? 1 : 0; }
void orc_set_stabilization(orc_problem* p, int mode) { p->stabilize = mode ? 1 : 0; }

void orc_node_types(const orc_problem* p, unsigned char* out)
{
    memcpy(out, p->ntype, (size_t)p->nx * p->ny);
}
int orc_num_lines(const orc_problem* p, int fam) { return p->fam[fam].n_lines; }
int orc_num_line_nodes(const orc_problem* p, int fam) { return p->fam[fam].n_nodes; }

void orc_lines(const orc_problem* p, int fam, int* off, double* xi, double* eta,
               double* bnorm, double* fval, double* h)
{
    const family* F = &p->fam[fam];
    memcpy(off, F->off, sizeof(int) * (F->n_lines + 1));
    memcpy(xi, F->xi, sizeof(double) * F->n_nodes);
    memcpy(eta, F->eta, sizeof(double) * F->n_nodes);
    memcpy(bnorm, F->bnorm, sizeof(double) * F->n_nodes);
    memcpy(fval, F->fval, sizeof(double) * F->n_nodes);
    memcpy(h, F->h, sizeof(double) * F->n_lines);
}

void orc_crossings(const orc_problem* p, int fam, int* seg, double* t, double* pos)
{
    const family* F = &p->fam[fam];
    size_t N = (size_t)p->nx * p->ny;
    for (size_t k = 0; k < 4 * N; ++k) {
        int inter = p->ntype[k / 4] == ORC_INTERIOR;
        seg[k] = inter ? F->cross[k].g : -2;
        t[k] = inter ? F->cross[k].t : 0.0;
        pos[k] = inter ? F->cross[k].pos : 0.0;
    }
}

/* ------------------------------------------------- interpolation steps */

/* grid -> line nodes by bilinear interpolation (§6.1); the two end nodes of a
 * line lie on the boundary of Omega_h, where u = 0 (§2, BVP1). */
void orc_gather(const orc_problem* p, int fam, const double* grid, double* vals)
{
    const family* F = &p->fam[fam];
    for (int l = 0; l < F->n_lines; ++l) {
        int a = F->off[l], b = F->off[l + 1] - 1;
        for (int k = a; k <= b; ++k)
            vals[k] = (k == a || k == b) ? 0.0 : bilin(p, grid, F->xi[k], F->eta[k]);
    }
}

static double cross_value(const crossing* c, const double* v)
{
    if (c->g < 0) return 0.0;
    return (1.0 - c->t) * v[c->g] + c->t * v[c->g + 1];
}

/* line values -> grid (§6): linear interpolation between the nearest crossing
 * on each side along the node's row and along its column, then the average of
 * the two (the paper's rule).  Optional reading for flow nearly parallel to a
 * grid axis, where the crossings on one grid direction are sparse: weight the
 * row value by the column gap and the column value by the row gap,
 * (g_c row + g_r col) / (g_r + g_c), g = distance between the two crossings
 * (a zero gap takes that direction's value alone).  Non-interior nodes get 0. */
void orc_map_to_grid(const orc_problem* p, int fam, const double* vals, double* grid)
{
    const family* F = &p->fam[fam];
    int nx = p->nx, ny = p->ny;
    for (int r = 0; r < ny; ++r)
        for (int i = 0; i < nx; ++i) {
            size_t node = (size_t)r * nx + i;
            if (p->ntype[node] != ORC_INTERIOR) {
                grid[node] = 0.0;
                continue;
            }
            const crossing* c = &F->cross[4 * node];
            double vL = cross_value(&c[0], vals), vR = cross_value(&c[1], vals);
            double vD = cross_value(&c[2], vals), vU = cross_value(&c[3], vals);
            double row, col;
            if (c[1].pos == c[0].pos) row = vL;
            else {
                double w = (i - c[0].pos) / (c[1].pos - c[0].pos);
                row = (1.0 - w) * vL + w * vR;
            }
            if (c[3].pos == c[2].pos) col = vD;
            else {
                double w = (r - c[2].pos) / (c[3].pos - c[2].pos);
                col = (1.0 - w) * vD + w * vU;
            }
            double gr = c[1].pos - c[0].pos, gc = c[3].pos - c[2].pos;
            if (p->interp_weights && gr + gc > 0.0) grid[node] = (gc * row + gr * col) / (gr + gc);
            else grid[node] = 0.5 * (row + col);
        }
}

/* ----------------------------------------------------------- 1D FEM */

/* Rows 1..n-1 of one line's system (§6 eqs. SemiDiscrSplit1Dbeta/1Dgamma with
 * linear elements):  (M + theta dt S) d = F - S u  on B lines, S = mu K + C + sigma M;
 *                    (M + theta dt mu K) d = -mu K u on G lines.
 * M = h/6 [2 1; 1 2], K = 1/h [1 -1; -1 1]; C is the advection form
 * int |beta| u' w dl with |beta| linear on the element and integrated exactly;
 * F = M f (f linear on the element).  Row q of the outputs is line row q+1;
 * a[0] and c[n-2] are set to 0. */
/* SUPG parameter of an element of length h with mean |beta| b (the
 * stabilisation the paper's conclusions propose for the 1D problems along
 * beta): tau = h / (2 b) (coth Pe - 1 / Pe), Pe = b h / (2 mu), the choice that
 * makes the 1D solution of -mu u'' + b u' = f nodally exact; the small-Pe
 * branch is the series Pe / 3 - Pe^3 / 45 of coth Pe - 1 / Pe. */
static double supg_tau(double h, double b, double mu)
{
    if (!(b > 0.0)) return 0.0;
    double pe = b * h / (2.0 * mu);
    double xi = pe < 1e-3 ? pe / 3.0 - pe * pe * pe / 45.0 : 1.0 / tanh(pe) - 1.0 / pe;
    return h / (2.0 * b) * xi;
}

/* One row k (1 <= k <= n-1) of a line's mass M, operator S and load F.
 * B lines (eq. SemiDiscrSplit1Dbeta1): S = mu K + C + sigma M,
 *   s_i(u, w) = int (mu u' w' + |beta| u' w + sigma u w) dl, F = M f.
 * G lines (eq. SemiDiscrSplit1Dgamma1): S = mu K, m_i(u, w) = int mu u' w' dl.
 * Linear elements of length h: M = h/6 [2 1; 1 2], K = 1/h [1 -1; -1 1];
 * C integrates |beta| u' w exactly with |beta| linear on the element
 * (reading: the paper does not say how the coefficient is integrated).
 * With SUPG on the B lines the test function w + tau |beta| w' adds, per
 * element (tau from the element's mean |beta|; |beta| and f linear, the
 * integrals exact): tau int u_t |beta| w' to M, tau int (|beta|^2 u' w' +
 * sigma u |beta| w') to S and tau int f |beta| w' to F. */
static void line_row(const orc_problem* p, int fam, int line, int k, double sig,
                     const double* fl, double* Msub, double* Mdia, double* Msup,
                     double* Ssub, double* Sdia, double* Ssup, double* Fk)
{
    const family* F = &p->fam[fam];
    const double* bn = F->bnorm + F->off[line];
    double h = F->h[line], mu = p->mu;
    double Mo = h / 6.0, Md = 2.0 * h / 3.0, Ko = -1.0 / h, Kd = 2.0 / h;
    *Msub = Mo;
    *Mdia = Md;
    *Msup = Mo;
    if (fam == 0) {
        double Csub = -(bn[k - 1] / 6.0 + bn[k] / 3.0);
        double Cdia = (bn[k - 1] - bn[k + 1]) / 6.0;
        double Csup = bn[k] / 3.0 + bn[k + 1] / 6.0;
        *Ssub = mu * Ko + Csub + sig * Mo;
        *Sdia = mu * Kd + Cdia + sig * Md;
        *Ssup = mu * Ko + Csup + sig * Mo;
        *Fk = h / 6.0 * (fl[k - 1] + 4.0 * fl[k] + fl[k + 1]);
        if (p->stabilize) {
            double bm = bn[k - 1], b0 = bn[k], bp = bn[k + 1];
            double fm = fl[k - 1], f0 = fl[k], fp = fl[k + 1];
            double tl = supg_tau(h, 0.5 * (bm + b0), mu), tr = supg_tau(h, 0.5 * (b0 + bp), mu);
            /* int phi_j |beta| phi_n' over the left (phi_n' = 1/h) and right
               (phi_n' = -1/h) element */
            double mb_sub = tl * (2.0 * bm + b0) / 6.0;
            double mb_dia = tl * (bm + 2.0 * b0) / 6.0 - tr * (2.0 * b0 + bp) / 6.0;
            double mb_sup = -tr * (b0 + 2.0 * bp) / 6.0;
            /* int |beta|^2 phi_j' phi_n' */
            double al = tl * (bm * bm + bm * b0 + b0 * b0) / (3.0 * h);
            double ar = tr * (b0 * b0 + b0 * bp + bp * bp) / (3.0 * h);
            *Msub += mb_sub;
            *Mdia += mb_dia;
            *Msup += mb_sup;
            *Ssub += -al + sig * mb_sub;
            *Sdia += al + ar + sig * mb_dia;
            *Ssup += -ar + sig * mb_sup;
            *Fk += tl * (2.0 * fm * bm + fm * b0 + f0 * bm + 2.0 * f0 * b0) / 6.0 -
                   tr * (2.0 * f0 * b0 + f0 * bp + fp * b0 + 2.0 * fp * bp) / 6.0;
        }
    } else {
        *Ssub = mu * Ko;
        *Sdia = mu * Kd;
        *Ssup = mu * Ko;
        *Fk = 0.0;
    }
}

/* Rows 1..n-1 of one line's substep system (§6 eqs. SemiDiscrSplit1Dbeta and
 * SemiDiscrSplit1Dgamma with linear elements):
 *   (M + theta dt S) d = F - S u   (the G lines carry no load).
 * Row q of the outputs is line row q+1; a[0] and c[n-2] are set to 0. */
int orc_line_system(const orc_problem* p, int fam, int line, double theta, double dt,
                    const double* u, double sig, const double* fl,
                    double* a, double* b, double* c, double* r)
{
    const family* F = &p->fam[fam];
    int n = F->off[line + 1] - F->off[line] - 1;
    if (n < 2) return 0;
    for (int k = 1; k < n; ++k) {
        double Msub, Mdia, Msup, Ssub, Sdia, Ssup, Fk;
        line_row(p, fam, line, k, sig, fl, &Msub, &Mdia, &Msup, &Ssub, &Sdia, &Ssup, &Fk);
        a[k - 1] = (k == 1) ? 0.0 : Msub + theta * dt * Ssub;
        b[k - 1] = Mdia + theta * dt * Sdia;
        c[k - 1] = (k == n - 1) ? 0.0 : Msup + theta * dt * Ssup;
        r[k - 1] = Fk - (Ssub * u[k - 1] + Sdia * u[k] + Ssup * u[k + 1]);
    }
    return n - 1;
}

/* Thomas algorithm (Gaussian elimination without pivoting for tridiagonal
 * systems); a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = r[i].  Returns 0, or -1 on a
 * zero pivot. */
static double g_min_pivot;
int orc_thomas(int n, const double* a, const double* b, const double* c,
               const double* r, double* x)
{
    if (n <= 0) return 0;
    double* cp = malloc(sizeof(double) * n);
    double* rp = malloc(sizeof(double) * n);
    if (!cp || !rp) return -1;
    double piv = b[0];
    if (piv == 0.0) return -1;
    if (fabs(piv) < g_min_pivot) g_min_pivot = fabs(piv);
    cp[0] = c[0] / piv;
    rp[0] = r[0] / piv;
    for (int i = 1; i < n; ++i) {
        piv = b[i] - a[i] * cp[i - 1];
        if (piv == 0.0) return -1;
        if (fabs(piv) < g_min_pivot) g_min_pivot = fabs(piv);
        cp[i] = c[i] / piv;
        rp[i] = (r[i] - a[i] * rp[i - 1]) / piv;
    }
    x[n - 1] = rp[n - 1];
    for (int i = n - 2; i >= 0; --i) x[i] = rp[i] - cp[i] * x[i + 1];
    free(cp);
    free(rp);
    return 0;
}

/* dense LU with partial pivoting (row-major A, solution overwrites b) */
int orc_dense_lu_solve(int n, double* A, double* b)
{
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = fabs(A[(size_t)i * n + k]);
            if (v > best) {
                best = v;
                piv = i;
            }
        }
        if (best == 0.0) return -1;
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[(size_t)k * n + j];
                A[(size_t)k * n + j] = A[(size_t)piv * n + j];
                A[(size_t)piv * n + j] = t;
            }
            double t = b[k];
            b[k] = b[piv];
            b[piv] = t;
        }
        double inv = 1.0 / A[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            double m = A[(size_t)i * n + k] * inv;
            if (m == 0.0) continue;
            A[(size_t)i * n + k] = m;
            for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= m * A[(size_t)k * n + j];
            b[i] -= m * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[(size_t)i * n + j] * b[j];
        b[i] = s / A[(size_t)i * n + i];
    }
    return 0;
}

/* One directional substep on every line of family fam: the increment d
 * (0 at the line ends).  f_extra (nullable, scaled) is added to f on the
 * B lines (the u_n/dt term of an implicit-Euler slice).  Returns the smallest
 * |pivot| met. */
static double sweep_core(const orc_problem* p, int fam, double theta, double dt,
                         const double* u_grid, const double* u_vals, double sig,
                         const double* f_grid, const double* f_extra, double fx_scale, double* d);

double orc_sweep_lines(const orc_problem* p, int fam, double theta, double dt,
                       const double* u_grid, double sig, const double* f_grid,
                       const double* f_extra, double fx_scale, double* d)
{
    return sweep_core(p, fam, theta, dt, u_grid, NULL, sig, f_grid, f_extra, fx_scale, d);
}

/* the same with the state given as values at the line nodes (u_vals) instead
 * of interpolated from the grid (the direct transfer) */
double orc_sweep_line_values(const orc_problem* p, int fam, double theta, double dt,
                             const double* u_vals, double sig, const double* f_extra,
                             double fx_scale, double* d)
{
    return sweep_core(p, fam, theta, dt, NULL, u_vals, sig, p->f, f_extra, fx_scale, d);
}

static double sweep_core(const orc_problem* p, int fam, double theta, double dt,
                         const double* u_grid, const double* u_vals, double sig,
                         const double* f_grid, const double* f_extra, double fx_scale, double* d)
{
    const family* F = &p->fam[fam];
    int nmax = 0;
    for (int l = 0; l < F->n_lines; ++l) {
        int n = F->off[l + 1] - F->off[l];
        if (n > nmax) nmax = n;
    }
    double* u = malloc(sizeof(double) * (nmax + 1));
    double* fl = malloc(sizeof(double) * (nmax + 1));
    double* a = malloc(sizeof(double) * (nmax + 1));
    double* b = malloc(sizeof(double) * (nmax + 1));
    double* c = malloc(sizeof(double) * (nmax + 1));
    double* r = malloc(sizeof(double) * (nmax + 1));
    g_min_pivot = INFINITY;
    for (int l = 0; l < F->n_lines; ++l) {
        int base = F->off[l], n = F->off[l + 1] - base - 1;
        for (int k = 0; k <= n; ++k) d[base + k] = 0.0;
        if (n < 2) continue;
        for (int k = 0; k <= n; ++k) {
            if (k == 0 || k == n) u[k] = 0.0;
            else if (u_vals) u[k] = u_vals[base + k];
            else u[k] = bilin(p, u_grid, F->xi[base + k], F->eta[base + k]);
            double fv = (f_grid == p->f) ? F->fval[base + k]
                                         : bilin(p, f_grid, F->xi[base + k], F->eta[base + k]);
            if (f_extra) fv += fx_scale * bilin(p, f_extra, F->xi[base + k], F->eta[base + k]);
            fl[k] = fv;
        }
        int m = orc_line_system(p, fam, l, theta, dt, u, sig, fl, a, b, c, r);
        orc_thomas(m, a, b, c, r, d + base + 1);
    }
    free(u);
    free(fl);
    free(a);
    free(b);
    free(c);
    free(r);
    return g_min_pivot;
}

/* ------------------------------------------------------- split step */

/* One directional substep of eq. SemiDiscrSplit reduced to the curves of one
 * family (§6): the grid state is interpolated onto the curves (§6.1), every
 * curve's 1D problem gives its increment d, the curve values
 * u^i + dt d are formed, and those VALUES are interpolated back onto the grid
 * (§6: the values of u_{j+1/2} are carried from one set of curves to the
 * other through the intermediate grid).  Non-interior grid nodes stay 0. */
static void substep(const orc_problem* p, int fam, double theta, double dt, double sig,
                    const double* f_extra, double fx_scale, const double* u_in,
                    double* u_out, double* d, double* v)
{
    const family* F = &p->fam[fam];
    orc_sweep_lines(p, fam, theta, dt, u_in, sig, p->f, fam == 0 ? f_extra : NULL,
                    fx_scale, d);
    orc_gather(p, fam, u_in, v);
    for (int k = 0; k < F->n_nodes; ++k) v[k] += dt * d[k];
    orc_map_to_grid(p, fam, v, u_out);
}

/* §5 eq. SemiDiscrSplit: u_j -> u_{j+1/2} (B curves, form s, load l)
 *                        u_{j+1/2} -> u_{j+1} (G curves, form m, no load). */
static void direct_step(const orc_problem* p, double theta, double dt, double sig,
                        const double* f_extra, double fx_scale, const double* uB, double* vB,
                        double* uG, double* vG, double* d);
static void paper_u0_values(const orc_problem* p, double* v);

void orc_split_step(const orc_problem* p, double theta, double dt, double sig,
                    const double* f_extra, double fx_scale,
                    const double* u, double* u_half, double* u_next)
{
    int nmax = p->fam[0].n_nodes > p->fam[1].n_nodes ? p->fam[0].n_nodes : p->fam[1].n_nodes;
    double* d = malloc(sizeof(double) * (nmax + 1));
    double* v = malloc(sizeof(double) * (nmax + 1));
    if (p->transfer) {
        /* the grid state onto the B nodes, one direct step, both halves back
           to the grid for the output */
        double* uB = malloc(sizeof(double) * (p->fam[0].n_nodes + 1));
        double* uG = malloc(sizeof(double) * (p->fam[1].n_nodes + 1));
        double* vG = malloc(sizeof(double) * (p->fam[1].n_nodes + 1));
        orc_gather(p, 0, u, uB);
        direct_step(p, theta, dt, sig, f_extra, fx_scale, uB, v, uG, vG, d);
        orc_map_to_grid(p, 0, v, u_half);
        orc_map_to_grid(p, 1, vG, u_next);
        free(uB);
        free(uG);
        free(vG);
    } else {
        substep(p, 0, theta, dt, sig, f_extra, fx_scale, u, u_half, d, v);
        substep(p, 1, theta, dt, sig, NULL, 0.0, u_half, u_next, d, v);
    }
    free(d);
    free(v);
}

/* one split step with the direct transfer: uB (state on the B nodes) -> vB
 * (B curve values u + dt d) -> uG (their transfer to the G nodes) -> vG (G
 * curve values); d is work space */
static void direct_step(const orc_problem* p, double theta, double dt, double sig,
                        const double* f_extra, double fx_scale, const double* uB, double* vB,
                        double* uG, double* vG, double* d)
{
    const family *B = &p->fam[0], *G = &p->fam[1];
    sweep_core(p, 0, theta, dt, NULL, uB, sig, p->f, f_extra, fx_scale, d);
    for (int k = 0; k < B->n_nodes; ++k) vB[k] = uB[k] + dt * d[k];
    orc_transfer(p, 1, vB, uG);
    sweep_core(p, 1, theta, dt, NULL, uG, sig, p->f, NULL, 0.0, d);
    for (int k = 0; k < G->n_nodes; ++k) vG[k] = uG[k] + dt * d[k];
}

/* ------------------------------------- accelerated stationary iteration
 * The multi-parameter pseudo-steps the method's stationary iteration invites
 * (a cycle of Δt values, as in cyclic ADI) do not keep its fixed point: the
 * split step's fixed point depends on Δt (only its midpoint does not, and only
 * for aligned flow), so a cycle converges to another state.  Reading: the
 * parameters vary per step as Anderson extrapolation weights instead.  With
 * g_k = Φ(u_k) the split step's output and f_k = g_k - u_k, the next state is
 * u_{k+1} = g_k - Σ_i γ_i (g_{k-i+1} - g_{k-i}), i = 1..min(m, k), where γ
 * minimises |f_k - Σ_i γ_i (f_{k-i+1} - f_{k-i})|.  Any γ leaves the fixed
 * points of Φ in place (f = 0 there gives γ = 0).  γ comes from the normal
 * equations A γ = b, A_ij = <Δf_i, Δf_j>, b_i = <Δf_i, f_k>, both formed from
 * the raw products <f_a, f_b> of the last m + 1 residuals, by Cholesky with
 * the columns newest first; a column whose pivot falls to 1e-12 of its
 * diagonal entry (or below) ends the factorisation, and only the columns
 * before it are used. */

#define AA_MAX 8

typedef struct {
    int m;
    size_t L;
    double* f;                          /* [(m+1) L] residuals by slot k mod (m+1) */
    double* g;                          /* [(m+1) L] map outputs by slot */
    double R[AA_MAX + 1][AA_MAX + 1];   /* <f_a, f_b> by slot */
} aa_state;

static int aa_init(aa_state* s, int m, size_t L)
{
    memset(s, 0, sizeof *s);
    s->m = m;
    s->L = L;
    s->f = calloc((size_t)(m + 1) * L, sizeof(double));
    s->g = calloc((size_t)(m + 1) * L, sizeof(double));
    return (s->f && s->g) ? 0 : -1;
}

static void aa_free(aa_state* s)
{
    free(s->f);
    free(s->g);
}

/* the mixing weights c_0..c_m of u_{k+1} = Σ_j c_j g_{k-j} from the raw
 * products of step k (mk = min(m, k) difference columns) */
static void aa_weights(const aa_state* s, int k, int mk, double* c)
{
    const int ns = s->m + 1;
#define AA_R(a, b) (s->R[(a) % ns][(b) % ns])
    double A[AA_MAX][AA_MAX], b[AA_MAX], Lc[AA_MAX][AA_MAX], y[AA_MAX], gam[AA_MAX];
    for (int i = 1; i <= mk; ++i) {
        int ai = k - i + 1, bi = k - i;
        b[i - 1] = AA_R(ai, k) - AA_R(bi, k);
        for (int j = 1; j <= i; ++j) {
            int aj = k - j + 1, bj = k - j;
            A[i - 1][j - 1] = AA_R(ai, aj) - AA_R(ai, bj) - AA_R(bi, aj) + AA_R(bi, bj);
        }
    }
#undef AA_R
    int use = mk;
    for (int i = 0; i < mk; ++i) {
        double d = A[i][i];
        for (int q = 0; q < i; ++q) d -= Lc[i][q] * Lc[i][q];
        if (!(A[i][i] > 0.0) || !(d > 1e-12 * A[i][i])) {
            use = i;
            break;
        }
        Lc[i][i] = sqrt(d);
        for (int j = i + 1; j < mk; ++j) {
            double e = A[j][i];
            for (int q = 0; q < i; ++q) e -= Lc[j][q] * Lc[i][q];
            Lc[j][i] = e / Lc[i][i];
        }
    }
    for (int i = 0; i < use; ++i) {
        double e = b[i];
        for (int q = 0; q < i; ++q) e -= Lc[i][q] * y[q];
        y[i] = e / Lc[i][i];
    }
    for (int i = use - 1; i >= 0; --i) {
        double e = y[i];
        for (int q = i + 1; q < use; ++q) e -= Lc[q][i] * gam[q];
        gam[i] = e / Lc[i][i];
    }
    for (int j = 0; j <= s->m; ++j) c[j] = 0.0;
    c[0] = 1.0;
    for (int i = 1; i <= use; ++i) {
        c[i - 1] -= gam[i - 1];
        c[i] += gam[i - 1];
    }
}

/* step k: records f_k = g - u and g_k, then u_next = the extrapolated state */
static void aa_next(aa_state* s, int k, const double* u, const double* g, double* u_next)
{
    const int ns = s->m + 1, sl = k % ns, mk = k < s->m ? k : s->m;
    double* fk = s->f + (size_t)sl * s->L;
    double* gk = s->g + (size_t)sl * s->L;
    for (size_t q = 0; q < s->L; ++q) {
        fk[q] = g[q] - u[q];
        gk[q] = g[q];
    }
    for (int j = 0; j <= mk; ++j) {
        const double* fj = s->f + (size_t)((k - j) % ns) * s->L;
        double acc = 0.0;
        for (size_t q = 0; q < s->L; ++q) acc += fk[q] * fj[q];
        s->R[sl][(k - j) % ns] = acc;
        s->R[(k - j) % ns][sl] = acc;
    }
    double c[AA_MAX + 1];
    aa_weights(s, k, mk, c);
    for (size_t q = 0; q < s->L; ++q) {
        double v = 0.0;
        for (int j = 0; j <= mk; ++j) v += c[j] * s->g[(size_t)((k - j) % ns) * s->L + q];
        u_next[q] = v;
    }
}

int orc_set_anderson(orc_problem* p, int m)
{
    if (m < 0 || m > AA_MAX) return ORC_EINVAL;
    p->anderson = m;
    return ORC_OK;
}

int orc_anderson_linear(int n, int m, const double* T, const double* c, double* x, int max_iter,
                        double tol, double* res)
{
    if (n < 1 || m < 0 || m > AA_MAX) return -1;
    aa_state s;
    double* g = malloc(sizeof(double) * n);
    if (!g || aa_init(&s, m, (size_t)n)) {
        free(g);
        return -1;
    }
    int k = 0;
    for (; k < max_iter; ++k) {
        double num = 0.0, den = 0.0;
        for (int i = 0; i < n; ++i) {
            double v = c[i];
            for (int j = 0; j < n; ++j) v += T[(size_t)i * n + j] * x[j];
            g[i] = v;
            num += (v - x[i]) * (v - x[i]);
            den += v * v;
        }
        double rel = den > 0.0 ? sqrt(num / den) : 0.0;
        if (res) res[k] = rel;
        if (rel <= tol) {
            ++k;
            break;
        }
        if (m == 0) memcpy(x, g, sizeof(double) * n);
        else aa_next(&s, k, x, g, x);
    }
    aa_free(&s);
    free(g);
    return k;
}

/* Stationary iteration with the direct transfer: the state lives on the B
 * nodes (u_j there), each step is direct_step followed by the transfer of the
 * G curve values back to the B nodes (u_{j+1}); the relative update is taken
 * over the interior B nodes.  Output: theta = 1/2 the midpoint
 * (u_j + u_{j+1/2}) / 2 on the B nodes mapped to the grid, otherwise the G
 * curve values of the last step mapped to the grid (also u_iter_out). */
static int solve_direct(const orc_problem* p, double theta, double dt, double tol, int max_iter,
                        int init, const double* u_init, double sig, const double* f_extra,
                        double fx_scale, double* u_out, double* u_iter_out, int* iters,
                        double* rel_out, int accel)
{
    const family *B = &p->fam[0], *G = &p->fam[1];
    size_t N = (size_t)p->nx * p->ny, nb = (size_t)B->n_nodes + 1, ng = (size_t)G->n_nodes + 1;
    double *uB = calloc(nb, sizeof(double)), *vB = calloc(nb, sizeof(double)),
           *uBn = calloc(nb, sizeof(double)), *uG = calloc(ng, sizeof(double)),
           *vG = calloc(ng, sizeof(double)), *d = calloc(nb > ng ? nb : ng, sizeof(double)),
           *tmp = calloc(N, sizeof(double));
    aa_state aa;
    const int m = accel ? p->anderson : 0;
    if (!uB || !vB || !uBn || !uG || !vG || !d || !tmp || aa_init(&aa, m, nb))
        return ORC_ENOMEM;
    if (dt <= 0.0) dt = orc_default_dt(p, sig);
    if (init == 1 && u_init) {
        for (size_t k = 0; k < N; ++k) tmp[k] = p->ntype[k] == ORC_INTERIOR ? u_init[k] : 0.0;
        orc_gather(p, 0, tmp, uB);
    } else if (init == 2) {
        paper_u0_values(p, uB);
    }
    int status = ORC_ENOCONV, j = 0;
    double rel = INFINITY;
    for (j = 0; j < max_iter; ++j) {
        direct_step(p, theta, dt, sig, f_extra, fx_scale, uB, vB, uG, vG, d);
        orc_transfer(p, 0, vG, uBn);
        double num = 0.0, den = 0.0;
        for (int l = 0; l < B->n_lines; ++l)
            for (int k = B->off[l] + 1; k < B->off[l + 1] - 1; ++k) {
                double dl = uBn[k] - uB[k];
                num += dl * dl;
                den += uBn[k] * uBn[k];
            }
        if (!isfinite(num) || !isfinite(den)) rel = INFINITY;
        else rel = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
        if (tol > 0.0 && rel <= tol) {
            status = ORC_OK;
            break;
        }
        if (!isfinite(rel)) break; /* diverged */
        if (j + 1 < max_iter) {
            if (m) aa_next(&aa, j, uB, uBn, uB);
            else memcpy(uB, uBn, sizeof(double) * nb);
        }
    }
    int done = (j < max_iter) ? j + 1 : max_iter;
    if (tol <= 0.0 && isfinite(rel)) status = ORC_OK;
    if (max_iter <= 0) {
        orc_map_to_grid(p, 0, uB, u_out);
        if (u_iter_out) memcpy(u_iter_out, u_out, N * sizeof(double));
    } else {
        if (theta == 0.5) {
            for (size_t k = 0; k < nb; ++k) d[k] = 0.5 * (uB[k] + vB[k]);
            orc_map_to_grid(p, 0, d, u_out);
        } else {
            orc_map_to_grid(p, 1, vG, u_out);
        }
        if (u_iter_out) orc_map_to_grid(p, 1, vG, u_iter_out);
    }
    if (iters) *iters = done;
    if (rel_out) *rel_out = rel;
    free(uB);
    free(vB);
    free(uBn);
    free(uG);
    free(vG);
    free(d);
    free(tmp);
    aa_free(&aa);
    return status;
}

/* Pseudo-time step (the paper gives none for the stationary problem): the
 * Peaceman-Rachford-optimal single parameter dt = 2 / sqrt(lmin lmax) with
 * lmin = sigma, lmax = 12 mu / h_s^2 + 2 sqrt(3) max|beta| / h_s. */
double orc_default_dt(const orc_problem* p, double sig)
{
    double lmax = 12.0 * p->mu / (p->hs * p->hs) + 2.0 * sqrt(3.0) * p->bmax / p->hs;
    return 2.0 / sqrt(sig * lmax);
}

/* §5 eq. u0stationary: s(u0, v) = <l, v>, i.e. one steady solve on every B
 * line (mu K + C + sigma M) u0 = F, mapped to the grid as values. */
void orc_paper_u0(const orc_problem* p, double* u0)
{
    double* v = calloc((size_t)p->fam[0].n_nodes + 1, sizeof(double));
    paper_u0_values(p, v);
    orc_map_to_grid(p, 0, v, u0);
    free(v);
}

/* the B-line solutions of eq. u0stationary (values at the B nodes) */
static void paper_u0_values(const orc_problem* p, double* v)
{
    const family* F = &p->fam[0];
    int nmax = 0;
    for (int l = 0; l < F->n_lines; ++l) {
        int n = F->off[l + 1] - F->off[l];
        if (n > nmax) nmax = n;
    }
    for (int k = 0; k < F->n_nodes; ++k) v[k] = 0.0;
    double* a = malloc(sizeof(double) * (nmax + 1));
    double* b = malloc(sizeof(double) * (nmax + 1));
    double* c = malloc(sizeof(double) * (nmax + 1));
    double* r = malloc(sizeof(double) * (nmax + 1));
    for (int l = 0; l < F->n_lines; ++l) {
        int base = F->off[l], n = F->off[l + 1] - base - 1;
        if (n < 2) continue;
        for (int k = 1; k < n; ++k) {
            double Msub, Mdia, Msup, Ssub, Sdia, Ssup, Fk;
            line_row(p, 0, l, k, p->sigma, F->fval + base, &Msub, &Mdia, &Msup, &Ssub, &Sdia, &Ssup,
                     &Fk);
            a[k - 1] = (k == 1) ? 0.0 : Ssub;
            b[k - 1] = Sdia;
            c[k - 1] = (k == n - 1) ? 0.0 : Ssup;
            r[k - 1] = Fk;
        }
        orc_thomas(n - 1, a, b, c, r, v + base + 1);
    }
    free(a);
    free(b);
    free(c);
    free(r);
}

/* relative update; a norm that is not finite (a diverging iteration) gives
 * rel = infinity, which ends the iteration without convergence */
static void relative_update(const orc_problem* p, const double* u, const double* un,
                            double* rel)
{
    double num = 0.0, den = 0.0;
    for (size_t k = 0; k < (size_t)p->nx * p->ny; ++k) {
        if (p->ntype[k] != ORC_INTERIOR) continue;
        double dlt = un[k] - u[k];
        num += dlt * dlt;
        den += un[k] * un[k];
    }
    if (!isfinite(num) || !isfinite(den)) *rel = INFINITY;
    else *rel = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
}

/* Stationary problem (BVP1) as the large-time limit of Parabolic1 (§2),
 * marched with the split scheme until the relative update
 * |u_{j+1} - u_j| / |u_{j+1}| (interior nodes, 2-norm) is <= tol.
 * Output: for theta = 1/2 the midpoint (u_j + u_{j+1/2}) / 2 of the last step
 * (the fixed point of the Crank-Nicolson split step sits there), otherwise
 * u_{j+1}; u_iter_out (nullable) receives u_{j+1}.  tol <= 0 runs exactly
 * max_iter steps and reports success. */
int orc_solve_stationary(const orc_problem* p, double theta, double dt, double tol,
                         int max_iter, int init, const double* u_init, double sig,
                         const double* f_extra, double fx_scale, double* u_out,
                         double* u_iter_out, int* iters, double* rel_out)
{
    if (p->transfer)
        return solve_direct(p, theta, dt, tol, max_iter, init, u_init, sig, f_extra, fx_scale, u_out,
                            u_iter_out, iters, rel_out, 1);
    size_t N = (size_t)p->nx * p->ny;
    double* u = calloc(N, sizeof(double));
    double* uh = calloc(N, sizeof(double));
    double* un = calloc(N, sizeof(double));
    aa_state aa;
    if (!u || !uh || !un || aa_init(&aa, p->anderson, N)) return ORC_ENOMEM;
    if (dt <= 0.0) dt = orc_default_dt(p, sig);
    if (init == 1 && u_init)
        for (size_t k = 0; k < N; ++k) u[k] = p->ntype[k] == ORC_INTERIOR ? u_init[k] : 0.0;
    else if (init == 2)
        orc_paper_u0(p, u);
    int status = ORC_ENOCONV, j = 0;
    double rel = INFINITY;
    for (j = 0; j < max_iter; ++j) {
        orc_split_step(p, theta, dt, sig, f_extra, fx_scale, u, uh, un);
        relative_update(p, u, un, &rel);
        if (tol > 0.0 && rel <= tol) {
            status = ORC_OK;
            break;
        }
        if (!isfinite(rel)) break; /* diverged */
        if (j + 1 < max_iter) {
            if (p->anderson) aa_next(&aa, j, u, un, u);
            else memcpy(u, un, N * sizeof(double));
        }
    }
    int done = (j < max_iter) ? j + 1 : max_iter;
    if (tol <= 0.0 && isfinite(rel)) status = ORC_OK; /* a fixed number of steps was asked for */
    if (max_iter <= 0) memcpy(un, u, N * sizeof(double)), memcpy(uh, u, N * sizeof(double));
    for (size_t k = 0; k < N; ++k)
        u_out[k] = (theta == 0.5) ? 0.5 * (u[k] + uh[k]) : un[k];
    if (u_iter_out) memcpy(u_iter_out, un, N * sizeof(double));
    if (iters) *iters = done;
    if (rel_out) *rel_out = rel;
    free(u);
    free(uh);
    free(un);
    aa_free(&aa);
    return status;
}

/* Parabolic1 (§2).  mode 0: the paper's scheme, one split step per time step
 * (eq. SemiDiscrSplit with the physical dt and theta).  mode 1: implicit Euler
 * in time, each slice -mu Lap u + beta.grad u + (sigma + 1/dt) u = f + u_n/dt
 * solved by the stationary iteration (theta, pseudo_dt, tol, max_iter).  The
 * Anderson extrapolation, when set, applies to the slices' solves of mode 1,
 * never to the time steps of mode 0. */
int orc_step_parabolic(const orc_problem* p, double dt, int nsteps, int mode,
                       double theta, double pseudo_dt, double tol, int max_iter,
                       double* u, int* total_iters)
{
    size_t N = (size_t)p->nx * p->ny;
    double* a = malloc(N * sizeof(double));
    double* b = malloc(N * sizeof(double));
    if (!a || !b) return ORC_ENOMEM;
    int st = ORC_OK, tot = 0;
    for (size_t k = 0; k < N; ++k)
        if (p->ntype[k] != ORC_INTERIOR) u[k] = 0.0;
    for (int s = 0; s < nsteps; ++s) {
        if (mode == 0 && p->transfer) {
            /* with the direct transfer the state stays on the B nodes: the
               time steps are the iteration's steps from the gathered u */
            int r = solve_direct(p, theta, dt, -1.0, nsteps, 1, u, p->sigma, NULL, 0.0, a, b, NULL, NULL,
                                 0);
            if (r != ORC_OK) st = r;
            memcpy(u, b, N * sizeof(double));
            tot += nsteps;
            break;
        } else if (mode == 0) {
            orc_split_step(p, theta, dt, p->sigma, NULL, 0.0, u, a, b);
            memcpy(u, b, N * sizeof(double));
            tot += 1;
        } else {
            double sig = p->sigma + 1.0 / dt;
            int it = 0;
            memcpy(a, u, N * sizeof(double));
            int r = orc_solve_stationary(p, theta, pseudo_dt, tol, max_iter, 1, a, sig, a,
                                         1.0 / dt, b, NULL, &it, NULL);
            if (r != ORC_OK) st = r;
            memcpy(u, b, N * sizeof(double));
            tot += it;
        }
    }
    if (total_iters) *total_iters = tot;
    free(a);
    free(b);
    return st;
}

/* -------------------------------------------------- brute-force references */

/* Dense Q1 (bilinear) Galerkin solution of a(u, v) = <l, v> (§4 eqs. VP1,
 * VP1a) on the active cells, beta and f bilinear, 2x2 Gauss quadrature (exact
 * for these integrands), Dirichlet on the non-interior nodes. */
int orc_q1_dense(int nx, int ny, double x0, double y0, double x1, double y1,
                 const unsigned char* mask, double mu, double sigma,
                 const double* beta1, const double* beta2, const double* f, double* u)
{
    orc_problem tmp;
    memset(&tmp, 0, sizeof tmp);
    tmp.nx = nx;
    tmp.ny = ny;
    size_t N = (size_t)nx * ny;
    tmp.cell = calloc((size_t)(nx - 1) * (ny - 1), 1);
    int* idx = malloc(sizeof(int) * N);
    if (!tmp.cell || !idx) return ORC_ENOMEM;
    for (int r = 0; r < ny - 1; ++r)
        for (int i = 0; i < nx - 1; ++i) {
            size_t a = (size_t)r * nx + i;
            tmp.cell[(size_t)r * (nx - 1) + i] = mask[a] && mask[a + 1] && mask[a + nx] && mask[a + nx + 1];
        }
    int n = 0;
    for (int r = 0; r < ny; ++r)
        for (int i = 0; i < nx; ++i) {
            int in = cell_active(&tmp, i - 1, r - 1) && cell_active(&tmp, i, r - 1) &&
                     cell_active(&tmp, i - 1, r) && cell_active(&tmp, i, r);
            idx[(size_t)r * nx + i] = in ? n++ : -1;
        }
    double* A = calloc((size_t)n * n, sizeof(double));
    double* F = calloc((size_t)n, sizeof(double));
    if (!A || !F) return ORC_ENOMEM;
    double hx = (x1 - x0) / (nx - 1), hy = (y1 - y0) / (ny - 1);
    double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
    for (int r = 0; r < ny - 1; ++r)
        for (int i = 0; i < nx - 1; ++i) {
            if (!cell_active(&tmp, i, r)) continue;
            size_t nd[4] = {(size_t)r * nx + i, (size_t)r * nx + i + 1, (size_t)(r + 1) * nx + i,
                            (size_t)(r + 1) * nx + i + 1};
            for (int qy = 0; qy < 2; ++qy)
                for (int qx = 0; qx < 2; ++qx) {
                    double sx = gp[qx], sy = gp[qy], w = 0.25 * hx * hy;
                    double ph[4] = {(1 - sx) * (1 - sy), sx * (1 - sy), (1 - sx) * sy, sx * sy};
                    double dxp[4] = {-(1 - sy) / hx, (1 - sy) / hx, -sy / hx, sy / hx};
                    double dyp[4] = {-(1 - sx) / hy, -sx / hy, (1 - sx) / hy, sx / hy};
                    double b1 = 0, b2 = 0, fv = 0;
                    for (int k = 0; k < 4; ++k) {
                        b1 += ph[k] * beta1[nd[k]];
                        b2 += ph[k] * beta2[nd[k]];
                        fv += ph[k] * f[nd[k]];
                    }
                    for (int ta = 0; ta < 4; ++ta) {
                        int I = idx[nd[ta]];
                        if (I < 0) continue;
                        F[I] += w * fv * ph[ta];
                        for (int tb = 0; tb < 4; ++tb) {
                            int J = idx[nd[tb]];
                            if (J < 0) continue;
                            double v = mu * (dxp[tb] * dxp[ta] + dyp[tb] * dyp[ta]) +
                                       (b1 * dxp[tb] + b2 * dyp[tb]) * ph[ta] + sigma * ph[tb] * ph[ta];
                            A[(size_t)I * n + J] += w * v;
                        }
                    }
                }
        }
    int st = orc_dense_lu_solve(n, A, F);
    for (size_t k = 0; k < N; ++k) u[k] = idx[k] >= 0 ? F[idx[k]] : 0.0;
    free(A);
    free(F);
    free(idx);
    free(tmp.cell);
    return st ? ORC_EINVAL : ORC_OK;
}

/* Dense P1 (linear triangles) Galerkin solution of the same problem; each
 * active cell is cut by its diagonal from (i, r) to (i+1, r+1).  Quadrature at
 * the edge midpoints (exact for the quadratic integrands). */
int orc_p1_dense(int nx, int ny, double x0, double y0, double x1, double y1,
                 const unsigned char* mask, double mu, double sigma,
                 const double* beta1, const double* beta2, const double* f, double* u)
{
    orc_problem tmp;
    memset(&tmp, 0, sizeof tmp);
    tmp.nx = nx;
    tmp.ny = ny;
    size_t N = (size_t)nx * ny;
    tmp.cell = calloc((size_t)(nx - 1) * (ny - 1), 1);
    int* idx = malloc(sizeof(int) * N);
    if (!tmp.cell || !idx) return ORC_ENOMEM;
    for (int r = 0; r < ny - 1; ++r)
        for (int i = 0; i < nx - 1; ++i) {
            size_t a = (size_t)r * nx + i;
            tmp.cell[(size_t)r * (nx - 1) + i] = mask[a] && mask[a + 1] && mask[a + nx] && mask[a + nx + 1];
        }
    int n = 0;
    for (int r = 0; r < ny; ++r)
        for (int i = 0; i < nx; ++i) {
            int in = cell_active(&tmp, i - 1, r - 1) && cell_active(&tmp, i, r - 1) &&
                     cell_active(&tmp, i - 1, r) && cell_active(&tmp, i, r);
            idx[(size_t)r * nx + i] = in ? n++ : -1;
        }
    double* A = calloc((size_t)n * n, sizeof(double));
    double* F = calloc((size_t)n, sizeof(double));
    if (!A || !F) return ORC_ENOMEM;
    double hx = (x1 - x0) / (nx - 1), hy = (y1 - y0) / (ny - 1);
    for (int r = 0; r < ny - 1; ++r)
        for (int i = 0; i < nx - 1; ++i) {
            if (!cell_active(&tmp, i, r)) continue;
            size_t n00 = (size_t)r * nx + i, n10 = n00 + 1, n01 = n00 + nx, n11 = n01 + 1;
            size_t tri[2][3] = {{n00, n10, n11}, {n00, n11, n01}};
            double cx[2][3] = {{0, hx, hx}, {0, hx, 0}}, cy[2][3] = {{0, 0, hy}, {0, hy, hy}};
            for (int t = 0; t < 2; ++t) {
                double xa = cx[t][0], ya = cy[t][0], xb = cx[t][1], yb = cy[t][1], xc = cx[t][2], yc = cy[t][2];
                double det = (xb - xa) * (yc - ya) - (xc - xa) * (yb - ya);
                double area = 0.5 * fabs(det);
                /* gradients of the barycentric functions */
                double gx[3] = {(yb - yc) / det, (yc - ya) / det, (ya - yb) / det};
                double gy[3] = {(xc - xb) / det, (xa - xc) / det, (xb - xa) / det};
                /* quadrature at edge midpoints: barycentric (1/2,1/2,0) etc. */
                double qb[3][3] = {{0.5, 0.5, 0.0}, {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}};
                for (int q = 0; q < 3; ++q) {
                    double b1 = 0, b2 = 0, fv = 0;
                    for (int k = 0; k < 3; ++k) {
                        b1 += qb[q][k] * beta1[tri[t][k]];
                        b2 += qb[q][k] * beta2[tri[t][k]];
                        fv += qb[q][k] * f[tri[t][k]];
                    }
                    double w = area / 3.0;
                    for (int ta = 0; ta < 3; ++ta) {
                        int I = idx[tri[t][ta]];
                        if (I < 0) continue;
                        F[I] += w * fv * qb[q][ta];
                        for (int tb = 0; tb < 3; ++tb) {
                            int J = idx[tri[t][tb]];
                            if (J < 0) continue;
                            double v = mu * (gx[tb] * gx[ta] + gy[tb] * gy[ta]) +
                                       (b1 * gx[tb] + b2 * gy[tb]) * qb[q][ta] +
                                       sigma * qb[q][tb] * qb[q][ta];
                            A[(size_t)I * n + J] += w * v;
                        }
                    }
                }
            }
        }
    int st = orc_dense_lu_solve(n, A, F);
    for (size_t k = 0; k < N; ++k) u[k] = idx[k] >= 0 ? F[idx[k]] : 0.0;
    free(A);
    free(F);
    free(idx);
    free(tmp.cell);
    return st ? ORC_EINVAL : ORC_OK;
}
