/*
 * FP64 CPU oracle of the warm-start network (forward, loss, backward).
 *
 * TEST INFRASTRUCTURE ONLY: the plain reference the GPU network kernels are
 * checked against; only the tests and the smoke check load it.
 *
 * The network maps a problem on a 256 x 256 node grid, and a first initial
 * state u0 of it (the state of eq. u0stationary), to the smooth part of the
 * correction u - u0, u the converged iterate of the stationary solve.  The
 * grid is read as 64 x 64 cells of 4 x 4 nodes; cell (r, c) holds the nodes
 * (4 r + a, 4 c + b), a, b = 0..3.  Every problem is scaled by
 * s = max |u0| (1 when u0 is absent or zero).  Features, NHWC, 40 channels:
 *   4 a + b: f at node (4 r + a, 4 c + b)      16 + 4 a + b: u0 / s there
 *   32, 33: cell means of beta1, beta2          34: (log10(mu) + 2.5) / 1.5
 *   35: sigma - 1                               36: cell mean of the mask
 *   37..39: 0
 * Eight 3 x 3 convolutions, zero padding, dilations 1 2 4 8 16 32 1 1,
 * channels 40 64 64 128 128 128 64 64 8, bias, ReLU after all but the last.
 * Output channel 0 predicts the cell mean of (u - u0) / s (channels 1..7 are
 * not used); the loss is 1/2 of the mean squared error of channel 0 over all
 * cells of the batch.  The initial state is u0 + s * (bilinear interpolation
 * of the cell values, cell centres at node 4 k + 1.5).
 * Weights of layer l: W[(tap * Cin + ci) * Cout + co], tap = 3 ky + kx.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define CNN_LAYERS 8
#define SUB 4     /* nodes per cell side */
#define NOUT 8    /* output channels per cell (channel 0 is the prediction) */
/* spatial size of the network grid: 64 x 64 for the model; the tests may
 * shrink it (the layers are size-agnostic) */
static int CNN_H = 64, CNN_W = 64;
void cnn_set_size(int h, int w)
{
    CNN_H = h;
    CNN_W = w;
}

static const int CH[CNN_LAYERS + 1] = {40, 64, 64, 128, 128, 128, 64, 64, NOUT};
static const int DIL[CNN_LAYERS] = {1, 2, 4, 8, 16, 32, 1, 1};

int cnn_layers(void) { return CNN_LAYERS; }
int cnn_channels(int l) { return CH[l]; }
int cnn_dilation(int l) { return DIL[l]; }

/* offsets of the packed parameter vector: W_0, b_0, W_1, b_1, ... */
long cnn_param_offset(int l, int bias)
{
    long off = 0;
    for (int k = 0; k < l; ++k) off += 9L * CH[k] * CH[k + 1] + CH[k + 1];
    return bias ? off + 9L * CH[l] * CH[l + 1] : off;
}
long cnn_num_params(void) { return cnn_param_offset(CNN_LAYERS, 0); }

/* scale of a problem: max |u0| over the grid, 1 when u0 is NULL or zero */
double cnn_scale(int n, const double* u0)
{
    double m = 0.0;
    if (u0)
        for (size_t k = 0; k < (size_t)n * n; ++k)
            if (fabs(u0[k]) > m) m = fabs(u0[k]);
    return m > 0.0 ? m : 1.0;
}

/* features of one problem on the (4 CNN_H) x (4 CNN_W) node grid; u0
 * nullable (zeros), s its scale */
void cnn_features(int n, const double* f, const double* b1, const double* b2,
                  const unsigned char* mask, double mu, double sigma, const double* u0,
                  double s, double* x)
{
    for (int r = 0; r < CNN_H; ++r)
        for (int c = 0; c < CNN_W; ++c) {
            double* o = x + ((size_t)r * CNN_W + c) * CH[0];
            double s1 = 0, s2 = 0, sm = 0;
            for (int a = 0; a < SUB; ++a)
                for (int b = 0; b < SUB; ++b) {
                    size_t k = (size_t)(r * SUB + a) * n + (c * SUB + b);
                    o[a * SUB + b] = f[k];
                    o[16 + a * SUB + b] = u0 ? u0[k] / s : 0.0;
                    s1 += b1[k];
                    s2 += b2[k];
                    sm += mask[k];
                }
            o[32] = s1 / (SUB * SUB);
            o[33] = s2 / (SUB * SUB);
            o[34] = (log10(mu) + 2.5) / 1.5;
            o[35] = sigma - 1.0;
            o[36] = sm / (SUB * SUB);
            o[37] = o[38] = o[39] = 0.0;
        }
}

/* target of one problem [H][W]: the cell means of (u - u0), divided by s;
 * u0 nullable */
void cnn_target(int n, const double* u, const double* u0, double s, double* t)
{
    for (int r = 0; r < CNN_H; ++r)
        for (int c = 0; c < CNN_W; ++c) {
            double sum = 0.0;
            for (int a = 0; a < SUB; ++a)
                for (int b = 0; b < SUB; ++b) {
                    size_t k = (size_t)(r * SUB + a) * n + (c * SUB + b);
                    sum += u[k] - (u0 ? u0[k] : 0.0);
                }
            t[(size_t)r * CNN_W + c] = sum / (SUB * SUB) / s;
        }
}

/* one convolution layer (pre-activation output) */
static void conv(const double* x, int cin, const double* W, const double* bias, int cout, int d,
                 double* y)
{
    for (int r = 0; r < CNN_H; ++r)
        for (int c = 0; c < CNN_W; ++c)
            for (int co = 0; co < cout; ++co) {
                double s = bias[co];
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx) {
                        int rr = r + (ky - 1) * d, cc = c + (kx - 1) * d;
                        if (rr < 0 || rr >= CNN_H || cc < 0 || cc >= CNN_W) continue;
                        const double* xp = x + ((size_t)rr * CNN_W + cc) * cin;
                        const double* wp = W + (size_t)((ky * 3 + kx) * cin) * cout + co;
                        for (int ci = 0; ci < cin; ++ci) s += xp[ci] * wp[(size_t)ci * cout];
                    }
                y[((size_t)r * CNN_W + c) * cout + co] = s;
            }
}

/* forward pass of one sample; acts (nullable) receives the post-activation
 * output of every layer, layer l at acts + cnn_act_offset(l); out (nullable):
 * the last layer's output [H][W][8] */
long cnn_act_offset(int l)
{
    long off = 0;
    for (int k = 0; k < l; ++k) off += (long)CNN_H * CNN_W * CH[k + 1];
    return off;
}

void cnn_forward(const double* params, const double* x, double* acts, double* out)
{
    long total = cnn_act_offset(CNN_LAYERS);
    double* A = acts ? acts : malloc(sizeof(double) * total);
    const double* in = x;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        double* y = A + cnn_act_offset(l);
        conv(in, CH[l], params + cnn_param_offset(l, 0), params + cnn_param_offset(l, 1),
             CH[l + 1], DIL[l], y);
        if (l < CNN_LAYERS - 1)
            for (long k = 0; k < (long)CNN_H * CNN_W * CH[l + 1]; ++k)
                if (y[k] < 0.0) y[k] = 0.0;
        in = y;
    }
    if (out) memcpy(out, A + cnn_act_offset(CNN_LAYERS - 1),
                    sizeof(double) * CNN_H * CNN_W * CH[CNN_LAYERS]);
    if (!acts) free(A);
}

/* loss and gradient over a batch: xs[b] features [H][W][40], ts[b] targets
 * [H][W] (channel 0).  grad (nullable, cnn_num_params) receives d loss /
 * d params.  Returns the loss. */
double cnn_loss_grad(const double* params, int batch, const double* xs, const double* ts,
                     double* grad)
{
    long total = cnn_act_offset(CNN_LAYERS), HW = (long)CNN_H * CNN_W;
    double* acts = malloc(sizeof(double) * total);
    double* dy = malloc(sizeof(double) * HW * 128);
    double* dx = malloc(sizeof(double) * HW * 128);
    const int cl = CH[CNN_LAYERS];
    double loss = 0.0, scale = 1.0 / ((double)batch * HW);
    if (grad) memset(grad, 0, sizeof(double) * cnn_num_params());
    for (int b = 0; b < batch; ++b) {
        const double* x = xs + (size_t)b * HW * CH[0];
        const double* t = ts + (size_t)b * HW;
        cnn_forward(params, x, acts, NULL);
        const double* yl = acts + cnn_act_offset(CNN_LAYERS - 1);
        memset(dy, 0, sizeof(double) * HW * cl);
        for (long k = 0; k < HW; ++k) {
            double e = yl[k * cl] - t[k];
            loss += 0.5 * e * e * scale;
            dy[k * cl] = e * scale;
        }
        if (!grad) continue;
        for (int l = CNN_LAYERS - 1; l >= 0; --l) {
            int cin = CH[l], cout = CH[l + 1], d = DIL[l];
            const double* xin = l == 0 ? x : acts + cnn_act_offset(l - 1);
            const double* y = acts + cnn_act_offset(l);
            /* through the ReLU of this layer (post-activation y > 0) */
            if (l < CNN_LAYERS - 1)
                for (long k = 0; k < HW * cout; ++k)
                    if (!(y[k] > 0.0)) dy[k] = 0.0;
            double* gW = grad + cnn_param_offset(l, 0);
            double* gb = grad + cnn_param_offset(l, 1);
            const double* W = params + cnn_param_offset(l, 0);
            memset(dx, 0, sizeof(double) * HW * cin);
            for (int r = 0; r < CNN_H; ++r)
                for (int c = 0; c < CNN_W; ++c)
                    for (int co = 0; co < cout; ++co) {
                        double g = dy[((size_t)r * CNN_W + c) * cout + co];
                        if (g == 0.0) continue;
                        gb[co] += g;
                        for (int ky = 0; ky < 3; ++ky)
                            for (int kx = 0; kx < 3; ++kx) {
                                int rr = r + (ky - 1) * d, cc = c + (kx - 1) * d;
                                if (rr < 0 || rr >= CNN_H || cc < 0 || cc >= CNN_W) continue;
                                size_t pin = ((size_t)rr * CNN_W + cc) * cin;
                                size_t wb = (size_t)((ky * 3 + kx) * cin) * cout + co;
                                for (int ci = 0; ci < cin; ++ci) {
                                    gW[wb + (size_t)ci * cout] += xin[pin + ci] * g;
                                    dx[pin + ci] += W[wb + (size_t)ci * cout] * g;
                                }
                            }
                    }
            memcpy(dy, dx, sizeof(double) * HW * cin);
        }
    }
    free(acts);
    free(dy);
    free(dx);
    return loss;
}

/* initial state from one output [H][W][8]: u = u0 + s * bilinear(y[..][0])
 * at the interior nodes, 0 elsewhere; cell centres at node 4 k + 1.5, the
 * interpolation clamped at the outer half cells; u0 nullable */
void cnn_upsample(int n, const double* y, const double* u0, double s,
                  const unsigned char* interior, double* u)
{
    for (int r = 0; r < CNN_H * SUB; ++r)
        for (int c = 0; c < CNN_W * SUB; ++c) {
            double fy = (r - (SUB - 1) * 0.5) / SUB, fx = (c - (SUB - 1) * 0.5) / SUB;
            if (fy < 0) fy = 0;
            if (fx < 0) fx = 0;
            if (fy > CNN_H - 1) fy = CNN_H - 1;
            if (fx > CNN_W - 1) fx = CNN_W - 1;
            int y0 = (int)fy, x0 = (int)fx;
            if (y0 > CNN_H - 2) y0 = CNN_H - 2;
            if (x0 > CNN_W - 2) x0 = CNN_W - 2;
            double ly = fy - y0, lx = fx - x0;
#define Y(rr, cc) y[((size_t)(rr) * CNN_W + (cc)) * NOUT]
            double v = (1 - ly) * ((1 - lx) * Y(y0, x0) + lx * Y(y0, x0 + 1)) +
                       ly * ((1 - lx) * Y(y0 + 1, x0) + lx * Y(y0 + 1, x0 + 1));
#undef Y
            size_t k = (size_t)r * n + c;
            u[k] = interior[k] ? (u0 ? u0[k] : 0.0) + s * v : 0.0;
        }
}
