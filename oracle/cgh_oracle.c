/*
 * cgh_oracle.c -- FP64 CPU oracle for complex-valued 2D Gaussian hologram optimisation
 * (arXiv 2511.15022).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * CPU-baseline leg of the benchmark call this file; the product path never does.
 *
 * Plain, slow, obviously-correct restatement of the paper's definitions:
 *   - activations                       (Suppl. "Parameter Activation Functions")
 *   - 2D covariance and its inverse     (Suppl. "2D Covariance Matrix Computation/Inversion")
 *   - Gaussian evaluation, power clamp  (Suppl. "Gaussian Evaluation")
 *   - complex accumulation, 0.99 clamp and 1/255 skip   (Algorithm 2; Sec. 3.1 Eqs. for g_n, H_n)
 *   - analytic backward                 (Suppl. "Detailed Gradient Derivation")
 *   - textbook mixed-radix FFT + direct DFT
 *   - band-limited angular spectrum     (Algorithm 3; Suppl. "Transfer Function Evaluation")
 *   - adjoint propagation with conj(H)  (Suppl. "Backward Pass", BLASM)
 *   - multi-plane intensity MSE          (Sec. 3.2, L_MSE)
 *   - Adam (PyTorch semantics)
 * No tiling, no culling, no fusion: every pixel meets every Gaussian.
 *
 * Readings of the paper where it is silent, ambiguous or inconsistent:
 *   - pixel centres are the 0-based integers 0..W-1, 0..H-1 (Sec. 3.1 counts pixels from 1
 *     while the means live in [0, W]; the difference is a reparametrisation);
 *   - the zero-pad of Algorithm 1 is 2x and centred, the image at offset (N-n)/2 per axis,
 *     and the crop takes the same window back;
 *   - the frequency of FFT bin k is s(k)/(N*pitch) with s(k)=k for k<N/2 else k-N, which is
 *     the centred index i-N/2 of Algorithm 3 after an fftshift;
 *   - the band limit is the rectangular one of Algorithm 3 (not the circular cut of the
 *     Sec. 2 equation), with the extent L taken on the PADDED grid (the propagation step
 *     of Algorithm 1 receives the padded field);
 *   - pairs with alpha*G above 0.99 are clamped and pass no gradient to alpha, mean and
 *     covariance (amplitude and phase still get 0.99 * ...); pairs below the 1/255 skip
 *     threshold pass none at all (the forward of Algorithm 2 differentiated as written);
 *   - the inverse-covariance to covariance step, absent from the paper's gradients, is the
 *     exact derivative of the adjugate formula inv = (S11, -S01, S00) / det;
 *   - the loss is the mean over the C*H*W values of each plane, times 1/L (Sec. 3.2 prints
 *     an unnormalised squared norm).
 *
 * Layouts: params are structure-of-arrays: xy_raw[N][2], s_raw[N][2], theta[N], amp[N][C],
 * phase[N][C], alpha_raw[N].  Complex fields are interleaved (re, im) doubles, [C][H][W].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

#define EPS_S 0.1    /* scale regularisation epsilon_s */
#define EPS_C 0.1    /* covariance regularisation epsilon_c */
#define EPS_D 1e-10  /* determinant clamp epsilon_d */
#define POWER_FLOOR (-50.0)
#define ALPHA_CAP 0.99

typedef struct {
    double mx, my;          /* activated mean (pixels) */
    double sx, sy, th;      /* activated scales, rotation */
    double S00, S01, S11;   /* covariance */
    double det;             /* unclamped determinant */
    double i00, i01, i11;   /* inverse covariance */
    double alpha;           /* activated opacity */
    double tx, ty;          /* tanh of raw means (for the backward) */
} orc_gauss;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Activations, covariance and inverse for Gaussian n (Suppl. activation, 2D covariance,
 * inversion). */
static void orc_activate_one(int n, int W, int H, const double* xy_raw, const double* s_raw,
                             const double* theta, const double* alpha_raw, orc_gauss* g) {
    g->tx = tanh(xy_raw[2 * n + 0]);
    g->ty = tanh(xy_raw[2 * n + 1]);
    g->mx = (g->tx + 1.0) / 2.0 * (double)W;
    g->my = (g->ty + 1.0) / 2.0 * (double)H;
    g->sx = exp(s_raw[2 * n + 0]) + EPS_S;
    g->sy = exp(s_raw[2 * n + 1]) + EPS_S;
    g->th = theta[n];
    g->alpha = 1.0 / (1.0 + exp(-alpha_raw[n]));
    double c = cos(g->th), s = sin(g->th);
    double sx2 = g->sx * g->sx, sy2 = g->sy * g->sy;
    g->S00 = sx2 * c * c + sy2 * s * s + EPS_C;
    g->S01 = (sx2 - sy2) * c * s;
    g->S11 = sx2 * s * s + sy2 * c * c + EPS_C;
    g->det = g->S00 * g->S11 - g->S01 * g->S01;
    double ds = g->det > EPS_D ? g->det : EPS_D;
    g->i00 = g->S11 / ds;
    g->i01 = -g->S01 / ds;
    g->i11 = g->S00 / ds;
}

/* Activated quantities for all Gaussians (exposed for tests).
 * out[N][12] = mx, my, sx, sy, theta, S00, S01, S11, i00, i01, i11, alpha. */
void orc_activate(int N, int W, int H, const double* xy_raw, const double* s_raw,
                  const double* theta, const double* alpha_raw, double* out) {
    for (int n = 0; n < N; ++n) {
        orc_gauss g;
        orc_activate_one(n, W, H, xy_raw, s_raw, theta, alpha_raw, &g);
        double* o = out + 12 * n;
        o[0] = g.mx; o[1] = g.my; o[2] = g.sx; o[3] = g.sy; o[4] = g.th;
        o[5] = g.S00; o[6] = g.S01; o[7] = g.S11;
        o[8] = g.i00; o[9] = g.i01; o[10] = g.i11; o[11] = g.alpha;
    }
}

/* Effective opacity of Gaussian g at pixel (px, py) (Algorithm 2 inner loop):
 * power = max(-mahal/2, -50), G = exp(power), a = min(0.99, alpha*G). */
static inline void orc_eval(const orc_gauss* g, double px, double py, double* dx, double* dy,
                            double* power_raw, double* G, double* a) {
    *dx = px - g->mx;
    *dy = py - g->my;
    double mahal = (*dx) * (*dx) * g->i00 + 2.0 * (*dx) * (*dy) * g->i01 + (*dy) * (*dy) * g->i11;
    *power_raw = -0.5 * mahal;
    double power = *power_raw > POWER_FLOOR ? *power_raw : POWER_FLOOR;
    *G = exp(power);
    double ag = g->alpha * (*G);
    *a = ag < ALPHA_CAP ? ag : ALPHA_CAP;
}

/*
 * Forward rasterisation (Algorithm 2; Sec. 3.1 sum over n of alpha_n c_n g_n exp(j phi_n)).
 * Brute force: every listed pixel against every Gaussian.  If pix_idx is NULL all H*W
 * pixels are computed and U is [C][H][W][2]; otherwise only npix pixels (linear indices
 * y*W+x) are computed and U is [C][npix][2].
 * cutoff: pairs with a < cutoff are skipped (1/255 in the paper, 0 = "smooth mode").
 */
void orc_raster_fwd(int H, int W, int C, int N, const double* xy_raw, const double* s_raw,
                    const double* theta, const double* amp, const double* phase,
                    const double* alpha_raw, double cutoff, int npix, const int64_t* pix_idx,
                    double* U) {
    orc_gauss* gs = (orc_gauss*)malloc(sizeof(orc_gauss) * (size_t)(N > 0 ? N : 1));
    for (int n = 0; n < N; ++n) orc_activate_one(n, W, H, xy_raw, s_raw, theta, alpha_raw, &gs[n]);
    int64_t P = pix_idx ? (int64_t)npix : (int64_t)H * W;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < P; ++q) {
        int64_t lin = pix_idx ? pix_idx[q] : q;
        double px = (double)(lin % W), py = (double)(lin / W);
        double acc_re[16], acc_im[16];
        for (int c = 0; c < C; ++c) { acc_re[c] = 0.0; acc_im[c] = 0.0; }
        for (int n = 0; n < N; ++n) {
            double dx, dy, pr, G, a;
            orc_eval(&gs[n], px, py, &dx, &dy, &pr, &G, &a);
            if (a < cutoff) continue;
            for (int c = 0; c < C; ++c) {
                double scale = amp[(size_t)n * C + c] * a;
                double ph = phase[(size_t)n * C + c];
                acc_re[c] += scale * cos(ph);
                acc_im[c] += scale * sin(ph);
            }
        }
        for (int c = 0; c < C; ++c) {
            U[2 * ((size_t)c * P + q) + 0] = acc_re[c];
            U[2 * ((size_t)c * P + q) + 1] = acc_im[c];
        }
    }
    free(gs);
}

/*
 * Backward rasterisation (Suppl. "Detailed Gradient Derivation", items 1-6).
 * dU is the gradient of the loss w.r.t. the field, [C][H][W][2] holding
 * (dL/dRe, dL/dIm) -- the convention of the Suppl. gradients, which treat real and
 * imaginary parts as separate real outputs.
 * Gradients are written for the pre-activation parameters; if g_idx is NULL all N
 * Gaussians are processed, otherwise only the ng listed ones, and each gradient array is
 * indexed by position in the list (g_xy[ng][2], ...).
 */
void orc_raster_bwd(int H, int W, int C, int N, const double* xy_raw, const double* s_raw,
                    const double* theta, const double* amp, const double* phase,
                    const double* alpha_raw, double cutoff, const double* dU, int ng,
                    const int64_t* g_idx, double* g_xy, double* g_s, double* g_theta,
                    double* g_amp, double* g_phase, double* g_alpha) {
    int64_t G_count = g_idx ? (int64_t)ng : (int64_t)N;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < G_count; ++q) {
        int n = (int)(g_idx ? g_idx[q] : q);
        orc_gauss g;
        orc_activate_one(n, W, H, xy_raw, s_raw, theta, alpha_raw, &g);
        double d_amp[16], d_phase[16], cph[16], sph[16];
        for (int c = 0; c < C; ++c) {
            d_amp[c] = 0.0; d_phase[c] = 0.0;
            cph[c] = cos(phase[(size_t)n * C + c]);
            sph[c] = sin(phase[(size_t)n * C + c]);
        }
        double d_alpha = 0.0, d_mx = 0.0, d_my = 0.0, d_i00 = 0.0, d_i01 = 0.0, d_i11 = 0.0;
        for (int py = 0; py < H; ++py) {
            for (int px = 0; px < W; ++px) {
                double dx, dy, pr, G, a;
                orc_eval(&g, (double)px, (double)py, &dx, &dy, &pr, &G, &a);
                if (a < cutoff) continue;               /* skipped: no gradient (O-6) */
                double dL_da = 0.0;                     /* dL/d alpha_eff */
                for (int c = 0; c < C; ++c) {
                    size_t o = 2 * (((size_t)c * H + py) * W + px);
                    double gR = dU[o], gI = dU[o + 1];
                    double ampc = amp[(size_t)n * C + c];
                    /* item 1: dL/dc = alpha G (cos phi dL/dRe + sin phi dL/dIm) */
                    d_amp[c] += a * (cph[c] * gR + sph[c] * gI);
                    /* item 2: dL/dphi = c alpha G (-sin phi dL/dRe + cos phi dL/dIm) */
                    d_phase[c] += ampc * a * (-sph[c] * gR + cph[c] * gI);
                    dL_da += ampc * (cph[c] * gR + sph[c] * gI);
                }
                if (g.alpha * G >= ALPHA_CAP) continue; /* clamped at 0.99 (O-6) */
                /* item 3: dL/dalpha = sum c G (cos dRe + sin dIm) */
                d_alpha += dL_da * G;
                double dL_dG = dL_da * g.alpha;
                if (pr <= POWER_FLOOR) continue;        /* power clamp: dpower/dmahal = 0 */
                double dL_dpower = dL_dG * G;           /* dG/dpower = G */
                double dL_dmahal = -0.5 * dL_dpower;
                /* item 4: dmahal/dmean = -2 (dx inv00 + dy inv01), -2 (dx inv01 + dy inv11) */
                d_mx += dL_dmahal * (-2.0) * (dx * g.i00 + dy * g.i01);
                d_my += dL_dmahal * (-2.0) * (dx * g.i01 + dy * g.i11);
                /* item 5: mahal = dx^2 inv00 + 2 dx dy inv01 + dy^2 inv11 */
                d_i00 += dL_dmahal * dx * dx;
                d_i01 += dL_dmahal * 2.0 * dx * dy;
                d_i11 += dL_dmahal * dy * dy;
            }
        }
        /* sigmoid backward (item 3) */
        double ga = d_alpha * g.alpha * (1.0 - g.alpha);
        /* tanh backward (item 4): dx/dxraw = W/2 (1 - tanh^2) */
        double gx = d_mx * (double)W / 2.0 * (1.0 - g.tx * g.tx);
        double gy = d_my * (double)H / 2.0 * (1.0 - g.ty * g.ty);
        /* inverse -> covariance (O-13): inv = (S11, -S01, S00) / D, D = S00 S11 - S01^2 */
        double a_ = g.S00, b_ = g.S01, c_ = g.S11;
        double dS00, dS01, dS11;
        if (g.det > EPS_D) {
            double D = g.det, D2 = D * D;
            dS00 = d_i00 * (-c_ * c_ / D2) + d_i01 * (b_ * c_ / D2) + d_i11 * (-b_ * b_ / D2);
            dS01 = d_i00 * (2.0 * b_ * c_ / D2) + d_i01 * (-(a_ * c_ + b_ * b_) / D2)
                 + d_i11 * (2.0 * a_ * b_ / D2);
            dS11 = d_i00 * (-b_ * b_ / D2) + d_i01 * (a_ * b_ / D2) + d_i11 * (-a_ * a_ / D2);
        } else {
            dS00 = d_i11 / EPS_D;
            dS01 = -d_i01 / EPS_D;
            dS11 = d_i00 / EPS_D;
        }
        /* item 6 (scales) and item 7 (rotation) */
        double cth = cos(g.th), sth = sin(g.th);
        double sx2 = g.sx * g.sx, sy2 = g.sy * g.sy;
        double d_sx = 2.0 * g.sx * (cth * cth * dS00 + cth * sth * dS01 + sth * sth * dS11);
        double d_sy = 2.0 * g.sy * (sth * sth * dS00 - cth * sth * dS01 + cth * cth * dS11);
        double d_th = 2.0 * (sy2 - sx2) * cth * sth * dS00
                    + (sx2 - sy2) * (cth * cth - sth * sth) * dS01
                    + 2.0 * (sx2 - sy2) * cth * sth * dS11;
        /* exponential backward: ds/ds_raw = exp(s_raw) */
        g_xy[2 * q + 0] = gx;
        g_xy[2 * q + 1] = gy;
        g_s[2 * q + 0] = d_sx * exp(s_raw[2 * n + 0]);
        g_s[2 * q + 1] = d_sy * exp(s_raw[2 * n + 1]);
        g_theta[q] = d_th;
        for (int c = 0; c < C; ++c) {
            g_amp[(size_t)q * C + c] = d_amp[c];
            g_phase[(size_t)q * C + c] = d_phase[c];
        }
        g_alpha[q] = ga;
    }
}

/* ------------------------------------------------------------------------------------- */
/* Discrete Fourier transforms.  Forward: X[k] = sum_n x[n] exp(-2 pi i k n / N),        */
/* inverse: x[n] = sum_k X[k] exp(+2 pi i k n / N) (unnormalised; callers divide by N).  */

/* Direct O(N^2) DFT of a strided complex sequence (interleaved doubles). */
void orc_dft1d(int n, double* data, int64_t stride, int inverse) {
    double* tmp = (double*)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    double sgn = inverse ? 1.0 : -1.0;
    for (int k = 0; k < n; ++k) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < n; ++j) {
            /* reduce k*j mod n exactly before forming the angle */
            int64_t kj = ((int64_t)k * j) % n;
            double ang = sgn * 2.0 * ORC_PI * (double)kj / (double)n;
            double xr = data[2 * j * stride], xi = data[2 * j * stride + 1];
            re += xr * cos(ang) - xi * sin(ang);
            im += xr * sin(ang) + xi * cos(ang);
        }
        tmp[2 * k] = re; tmp[2 * k + 1] = im;
    }
    for (int k = 0; k < n; ++k) {
        data[2 * k * stride] = tmp[2 * k];
        data[2 * k * stride + 1] = tmp[2 * k + 1];
    }
    free(tmp);
}

static int orc_smallest_factor(int n) {
    if (n % 4 == 0) return 4;
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* Recursive mixed-radix decimation-in-time FFT (Cooley-Tukey): for n = p*m, split the
 * input into p interleaved subsequences x[r + p*j], transform each (length m), then
 * X[k + m*q] = sum_r W_n^{r (k + m q)} Y_r[k].  Contiguous in/out, out != in. */
static void orc_fft_rec(int n, const double* in, int64_t istride, double* out, double sgn,
                        double* scratch) {
    if (n == 1) { out[0] = in[0]; out[1] = in[1]; return; }
    int p = orc_smallest_factor(n);
    int m = n / p;
    if (m == 1) {  /* prime (or 4) length: direct DFT */
        for (int k = 0; k < n; ++k) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < n; ++j) {
                int64_t kj = ((int64_t)k * j) % n;
                double ang = sgn * 2.0 * ORC_PI * (double)kj / (double)n;
                double xr = in[2 * j * istride], xi = in[2 * j * istride + 1];
                re += xr * cos(ang) - xi * sin(ang);
                im += xr * sin(ang) + xi * cos(ang);
            }
            out[2 * k] = re; out[2 * k + 1] = im;
        }
        return;
    }
    /* sub-transforms Y_r = FFT_m(x[r], x[r+p], ...) stored in scratch[r*m + k] */
    double* Y = scratch;
    double* sub_scratch = scratch + 2 * (size_t)n;
    for (int r = 0; r < p; ++r)
        orc_fft_rec(m, in + 2 * r * istride, istride * p, Y + 2 * (size_t)r * m, sgn, sub_scratch);
    for (int q = 0; q < p; ++q) {
        for (int k = 0; k < m; ++k) {
            int kk = k + m * q;
            double re = 0.0, im = 0.0;
            for (int r = 0; r < p; ++r) {
                int64_t rk = ((int64_t)r * kk) % n;
                double ang = sgn * 2.0 * ORC_PI * (double)rk / (double)n;
                double yr = Y[2 * ((size_t)r * m + k)], yi = Y[2 * ((size_t)r * m + k) + 1];
                re += yr * cos(ang) - yi * sin(ang);
                im += yr * sin(ang) + yi * cos(ang);
            }
            out[2 * kk] = re; out[2 * kk + 1] = im;
        }
    }
}

/* In-place FFT of a strided sequence of length n. */
void orc_fft1d(int n, double* data, int64_t stride, int inverse) {
    if (n <= 1) return;
    double* in = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    double* out = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    /* scratch: each recursion level needs 2n doubles, depth <= log2 n + 1 */
    size_t depth = 2;
    for (int t = n; t > 1; t /= 2) ++depth;
    double* scratch = (double*)malloc(sizeof(double) * 4 * (size_t)n * depth);
    for (int j = 0; j < n; ++j) {
        in[2 * j] = data[2 * j * stride];
        in[2 * j + 1] = data[2 * j * stride + 1];
    }
    orc_fft_rec(n, in, 1, out, inverse ? 1.0 : -1.0, scratch);
    for (int j = 0; j < n; ++j) {
        data[2 * j * stride] = out[2 * j];
        data[2 * j * stride + 1] = out[2 * j + 1];
    }
    free(scratch); free(out); free(in);
}

/* 2D FFT of a [ny][nx] interleaved complex array: every row, then every column. */
void orc_fft2d(int ny, int nx, double* data, int inverse) {
    #pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < ny; ++y) orc_fft1d(nx, data + 2 * (size_t)y * nx, 1, inverse);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int x = 0; x < nx; ++x) orc_fft1d(ny, data + 2 * (size_t)x, nx, inverse);
}

/* ------------------------------------------------------------------------------------- */
/* Band-limited angular spectrum method (Algorithm 3, Suppl. "Spatial Frequency          */
/* Computation", "Bandlimit Computation", "Transfer Function Evaluation").               */

/* signed frequency index of FFT bin k: the centred index i - N/2 after an fftshift */
static inline int orc_signed_index(int k, int n) { return k < (n + 1) / 2 ? k : k - n; }

/* Transfer function H(f_x, f_y; lambda, d) on an ny x nx grid in FFT bin order.
 * aperture > 0 additionally zeroes bins outside the circle of Algorithm 3 (index space,
 * centre N/2 - 0.5 in the centred layout).  out[ny][nx][2]. */
void orc_blasm_transfer(int ny, int nx, double lambda, double pitch, double d, double aperture,
                        double* out) {
    double k = 2.0 * ORC_PI / lambda;
    double Lx = nx * pitch, Ly = ny * pitch;
    double fxmax = 1.0 / (lambda * sqrt((2.0 * d / Lx) * (2.0 * d / Lx) + 1.0));
    double fymax = 1.0 / (lambda * sqrt((2.0 * d / Ly) * (2.0 * d / Ly) + 1.0));
    for (int ky = 0; ky < ny; ++ky) {
        for (int kx = 0; kx < nx; ++kx) {
            int sx = orc_signed_index(kx, nx), sy = orc_signed_index(ky, ny);
            double fx = (double)sx / Lx, fy = (double)sy / Ly;
            double re = 0.0, im = 0.0;
            if (fabs(fx) < fxmax && fabs(fy) < fymax) {
                double kz2 = k * k - 4.0 * ORC_PI * ORC_PI * (fx * fx + fy * fy);
                double kz = kz2 > 0.0 ? sqrt(kz2) : 0.0;
                re = cos(kz * d);
                im = sin(kz * d);
            }
            if (aperture > 0.0) {
                /* centred index i = s + N/2; distance from (N/2 - 0.5) is s + 0.5 */
                double ax = (double)sx + 0.5, ay = (double)sy + 0.5;
                if (ax * ax + ay * ay >= aperture * aperture) { re = 0.0; im = 0.0; }
            }
            out[2 * ((size_t)ky * nx + kx)] = re;
            out[2 * ((size_t)ky * nx + kx) + 1] = im;
        }
    }
}

/* Propagate one H x W complex field by distance d with pad factor `pad`:
 * centred zero-pad -> FFT2 -> x H (or conj H) -> IFFT2 / N -> crop the same window.
 * conj_h selects the adjoint (backward) transfer function.  Accumulates into out
 * (out += result) so that the backward sum over planes is a plain loop. */
static void orc_propagate_accumulate(int H, int W, int pad, double lambda, double pitch,
                                     double d, double aperture, int conj_h, const double* in,
                                     double* out) {
    int ny = pad * H, nx = pad * W;
    int oy = (ny - H) / 2, ox = (nx - W) / 2;
    size_t tot = (size_t)ny * nx;
    double* P = (double*)calloc(2 * tot, sizeof(double));
    double* T = (double*)malloc(sizeof(double) * 2 * tot);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t s = 2 * ((size_t)y * W + x), t = 2 * ((size_t)(y + oy) * nx + (x + ox));
            P[t] = in[s]; P[t + 1] = in[s + 1];
        }
    orc_fft2d(ny, nx, P, 0);
    orc_blasm_transfer(ny, nx, lambda, pitch, d, aperture, T);
    for (size_t i = 0; i < tot; ++i) {
        double hr = T[2 * i], hi = conj_h ? -T[2 * i + 1] : T[2 * i + 1];
        double ur = P[2 * i], ui = P[2 * i + 1];
        P[2 * i] = ur * hr - ui * hi;
        P[2 * i + 1] = ur * hi + ui * hr;
    }
    orc_fft2d(ny, nx, P, 1);
    double inv_n = 1.0 / (double)tot;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t s = 2 * ((size_t)(y + oy) * nx + (x + ox)), t = 2 * ((size_t)y * W + x);
            out[t] += P[s] * inv_n;
            out[t + 1] += P[s + 1] * inv_n;
        }
    free(T); free(P);
}

/* Forward BLASM for C channels and L planes: Ud[l][c] = crop(IFFT(H_{c,l} FFT(pad(U0[c])))).
 * U0 [C][H][W][2], Ud [L][C][H][W][2]. */
void orc_blasm_fwd(int H, int W, int C, int L, int pad, const double* lambda, double pitch,
                   const double* z, double aperture, const double* U0, double* Ud) {
    size_t S = 2 * (size_t)H * W;
    memset(Ud, 0, sizeof(double) * S * (size_t)C * L);
    for (int l = 0; l < L; ++l)
        for (int c = 0; c < C; ++c)
            orc_propagate_accumulate(H, W, pad, lambda[c], pitch, z[l], aperture, 0,
                                     U0 + S * c, Ud + S * ((size_t)l * C + c));
}

/* Adjoint BLASM (Suppl. BLASM "Backward Pass"): dU0[c] = sum_l crop(IFFT(conj(H_{c,l})
 * FFT(pad(dUd[l][c])))).  The gradient convention (dL/dRe, dL/dIm) makes this the exact
 * adjoint of the forward map. */
void orc_blasm_bwd(int H, int W, int C, int L, int pad, const double* lambda, double pitch,
                   const double* z, double aperture, const double* dUd, double* dU0) {
    size_t S = 2 * (size_t)H * W;
    memset(dU0, 0, sizeof(double) * S * (size_t)C);
    for (int c = 0; c < C; ++c)
        for (int l = 0; l < L; ++l)
            orc_propagate_accumulate(H, W, pad, lambda[c], pitch, z[l], aperture, 1,
                                     dUd + S * ((size_t)l * C + c), dU0 + S * c);
}

/* ------------------------------------------------------------------------------------- */
/* Multi-plane intensity MSE (Sec. 3.2): I_l = |U(d_l)|^2,                                */
/* L = (1/L) sum_l mean_{c,p} (I_l - I^_l)^2.  Returns L; writes dL/dUd as (dRe, dIm):    */
/* dL/dRe = dL/dI * 2 Re, dL/dIm = dL/dI * 2 Im.                                          */
double orc_mse_loss(int L, int C, int H, int W, const double* Ud, const double* target,
                    double* dUd) {
    size_t tot = (size_t)L * C * H * W;
    double norm = 1.0 / ((double)L * (double)C * (double)H * (double)W);
    double acc = 0.0;
    for (size_t i = 0; i < tot; ++i) {
        double re = Ud[2 * i], im = Ud[2 * i + 1];
        double I = re * re + im * im;
        double diff = I - target[i];
        acc += diff * diff;
        if (dUd) {
            double dI = 2.0 * diff * norm;
            dUd[2 * i] = dI * 2.0 * re;
            dUd[2 * i + 1] = dI * 2.0 * im;
        }
    }
    return acc * norm;
}

/* Reconstruction loss of Sec. 3.2 (the three-term L_recon):                             */
/*   L = (1/L) sum_l mean_{c,p} [ (I - I^)^2 + (I M - I^ M)^2 + (I I^ - I^ I^)^2 ]         */
/* with I = |Ud|^2, I^ the target and M_l the binary depth mask of plane l (one byte per    */
/* pixel, shared by the colour channels; mask == NULL means M = 0).  The mean over c and p  */
/* follows the same reading as orc_mse_loss.  Returns L; writes dL/dUd as (dRe, dIm).       */
double orc_recon_loss(int L, int C, int H, int W, const double* Ud, const double* target,
                      const unsigned char* mask, double* dUd) {
    double norm = 1.0 / ((double)L * (double)C * (double)H * (double)W);
    double acc = 0.0;
    for (int l = 0; l < L; ++l)
        for (int c = 0; c < C; ++c)
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    size_t i = (((size_t)l * C + c) * H + y) * W + x;
                    double M = mask ? (double)(mask[((size_t)l * H + y) * W + x] != 0) : 0.0;
                    double re = Ud[2 * i], im = Ud[2 * i + 1];
                    double I = re * re + im * im, T = target[i];
                    double t1 = I - T;
                    double t2 = I * M - T * M;
                    double t3 = I * T - T * T;
                    acc += t1 * t1 + t2 * t2 + t3 * t3;
                    if (dUd) {
                        /* dL/dI of the three squares */
                        double dI = 2.0 * norm * (t1 + M * t2 + T * t3);
                        dUd[2 * i] = dI * 2.0 * re;
                        dUd[2 * i + 1] = dI * 2.0 * im;
                    }
                }
    return acc * norm;
}

/* Plane-averaged PSNR of the reconstructed intensities against the targets (Sec. 5
 * reports PSNR averaged over planes); intensities are clipped to [0, 1]. */
double orc_psnr(int L, int C, int H, int W, const double* Ud, const double* target) {
    size_t per = (size_t)C * H * W;
    double sum = 0.0;
    for (int l = 0; l < L; ++l) {
        double se = 0.0;
        for (size_t i = 0; i < per; ++i) {
            size_t j = (size_t)l * per + i;
            double I = Ud[2 * j] * Ud[2 * j] + Ud[2 * j + 1] * Ud[2 * j + 1];
            if (I > 1.0) I = 1.0;
            if (I < 0.0) I = 0.0;
            double d = I - target[j];
            se += d * d;
        }
        double mse = se / (double)per;
        sum += 10.0 * log10(1.0 / (mse > 1e-300 ? mse : 1e-300));
    }
    return sum / (double)L;
}

/* Adan step (adaptive Nesterov momentum; the optimiser the paper trains with, Sec. 4),
 * restated from its published algorithm with the bias corrections of the authors' release,
 * betas in the "running average" convention (defaults 0.98, 0.92, 0.99):
 *   d = g - g_prev (d = 0 at t = 1)
 *   m = b1 m + (1 - b1) g;   v = b2 v + (1 - b2) d;   n = b3 n + (1 - b3) (g + b2 d)^2
 *   p = (p - lr (m / (1 - b1^t) + b2 v / (1 - b2^t)) / (sqrt(n / (1 - b3^t)) + eps))
 *       / (1 + lr wd);   g_prev = g.  Step t >= 1. */
void orc_adan(int64_t n, double* p, const double* g, double* m, double* v, double* nn,
              double* gprev, double lr, double b1, double b2, double b3, double eps,
              double wd, int t) {
    double bc1 = 1.0 - pow(b1, (double)t);
    double bc2 = 1.0 - pow(b2, (double)t);
    double bc3 = 1.0 - pow(b3, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        double d = (t == 1) ? 0.0 : g[i] - gprev[i];
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * d;
        double u = g[i] + b2 * d;
        nn[i] = b3 * nn[i] + (1.0 - b3) * u * u;
        double step = (m[i] / bc1 + b2 * v[i] / bc2) / (sqrt(nn[i] / bc3) + eps);
        p[i] = (p[i] - lr * step) / (1.0 + lr * wd);
        gprev[i] = g[i];
    }
}

/* Adam step with PyTorch semantics (no weight decay, no amsgrad), step t >= 1. */
void orc_adam(int64_t n, double* p, const double* g, double* m, double* v, double lr,
              double beta1, double beta2, double eps, int t) {
    double bc1 = 1.0 - pow(beta1, (double)t);
    double bc2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double denom = sqrt(v[i]) / sqrt(bc2) + eps;
        p[i] -= lr / bc1 * m[i] / denom;
    }
}
