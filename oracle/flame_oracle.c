/*
 * flame_oracle.c -- plain, slow, FP64 CPU oracle for one explicit time step of
 * the Sivashinsky-type model of an expanding spherical flame (Karlin,
 * "Global communications in multiprocessor simulations of flames",
 * Sec. 2 eq. (SivCurv1c) and Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Everything is double precision.  Complex numbers are C99 double _Complex,
 * which has the same memory layout as numpy complex128.
 *
 * Conventions (where the paper is silent or its text garbled, these are the
 * readings taken):
 *   grid         x_i = 2*pi*j_i/N_i, j_i = 0..N_i-1, i = 1 (theta), 2 (phi)
 *   coefficients Phi(x) = sum_k Phi_k exp(i (k1 x1 + k2 x2))
 *   wavenumbers  kappa = (s1 k1, s2 k2)      (s1 = s2 = theta_pi as printed)
 *   truncation   |k1| <= K1, |k2| <= K2, N_i >= 4 K_i + 1   (Sec. 3)
 *   state        compact half spectrum: rows k1 = -K1..K1, columns
 *                k2 = 0..K2, k2 fastest; the k = 0 slot is ignored, the mean
 *                mode Phi_0 is a separate double.
 *   r0(t) = t (Sec. 2), omega_k = -|kappa|^2/r0^2 + gamma |kappa|/(2 r0),
 *   nonlinear coefficient c = 1/(2 r0^2) acting on |grad Phi|^2.
 *
 * Parity pins: every exported function is pinned by tests/test_oracle_*.py
 * against brute force, closed forms or invariants; see the header comment of
 * each function for what pins it.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

#define ORC_LINEAR_ONLY 1u
#define ORC_NONLINEAR_ONLY 2u

typedef struct {
    int n1, n2;     /* grid N1 x N2 (theta, phi), powers of two            */
    int K1, K2;     /* retained harmonics, 4 K_i + 1 <= N_i                */
    double gamma;   /* density contrast, eq. (SivCurv1c)                   */
    double s1, s2;  /* wavenumber scales (theta_pi in eq. (SivCurv1c))    */
    double t0, dt;  /* initial time and explicit Euler step               */
    unsigned flags; /* ORC_LINEAR_ONLY / ORC_NONLINEAR_ONLY (test modes)   */
} orc_params;

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------------ */
/* 1-D transforms                                                           */
/* ------------------------------------------------------------------------ */

/* Brute-force DFT, the definition: y[k] = sum_j x[j] exp(sign 2 pi i j k / n).
 * Any n >= 1, O(n^2).  The angle is reduced modulo n in integers so that it
 * stays exact.  Pinned by closed forms (impulse, single exponential). */
void orc_dft(int n, const cplx *x, cplx *y, int sign)
{
    for (int k = 0; k < n; k++) {
        cplx acc = 0;
        for (int j = 0; j < n; j++) {
            long m = ((long)j * (long)k) % n;
            double a = sign * TWO_PI * (double)m / (double)n;
            acc += x[j] * (cos(a) + I * sin(a));
        }
        y[k] = acc;
    }
}

/* Recursive radix-2 decimation-in-time step: y[0..n) = DFT of the n samples
 * x[0], x[stride], ..., using the root table tw[m] = exp(sign 2 pi i m / N)
 * of the top-level length N, so that exp(sign 2 pi i k / n) = tw[k*twstride]
 * with twstride = N / n. */
static void fft_rec(int n, const cplx *x, int stride, cplx *y,
                    const cplx *tw, int twstride)
{
    if (n == 1) {
        y[0] = x[0];
        return;
    }
    int h = n / 2;
    fft_rec(h, x, 2 * stride, y, tw, 2 * twstride);          /* even samples */
    fft_rec(h, x + stride, 2 * stride, y + h, tw, 2 * twstride); /* odd */
    for (int k = 0; k < h; k++) {
        cplx e = y[k];
        cplx o = tw[k * twstride] * y[k + h];
        y[k] = e + o;
        y[k + h] = e - o;
    }
}

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* Complex FFT of length n (a power of two), in place, unnormalised:
 * x[k] <- sum_j x[j] exp(sign 2 pi i j k / n).  Plain recursive radix-2.
 * Pinned against orc_dft (tests) and Parseval.  Returns 0, or -1 if n is not
 * a power of two. */
int orc_fft(int n, cplx *x, int sign)
{
    if (!is_pow2(n)) return -1;
    cplx *tw = malloc(sizeof(cplx) * (size_t)(n / 2 + 1));
    cplx *y = malloc(sizeof(cplx) * (size_t)n);
    for (int m = 0; m < n / 2 + 1; m++) {
        double a = sign * TWO_PI * (double)m / (double)n;
        tw[m] = cos(a) + I * sin(a);
    }
    fft_rec(n, x, 1, y, tw, 1);
    memcpy(x, y, sizeof(cplx) * (size_t)n);
    free(y);
    free(tw);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 2-D real transforms as tensor products of 1-D ones (Sec. 2, Sec. 3)      */
/* ------------------------------------------------------------------------ */

/* Unnormalised 2-D analysis of a real n1 x n2 array:
 *   out[k1][k2] = sum_{j1,j2} in[j1][j2] exp(-2 pi i (k1 j1/n1 + k2 j2/n2)),
 * kept for k2 = 0..n2/2 (row-major n1 x (n2/2+1)).  Rows first, then columns.
 * Pinned against the 2-D DFT definition on small grids. */
int orc_rfft2(int n1, int n2, const double *in, cplx *out)
{
    if (!is_pow2(n1) || !is_pow2(n2)) return -1;
    int h2 = n2 / 2 + 1;
#pragma omp parallel for schedule(static)
    for (int j1 = 0; j1 < n1; j1++) {
        cplx *row = malloc(sizeof(cplx) * (size_t)n2);
        for (int j2 = 0; j2 < n2; j2++) row[j2] = in[(size_t)j1 * n2 + j2];
        orc_fft(n2, row, -1);
        for (int k2 = 0; k2 < h2; k2++) out[(size_t)j1 * h2 + k2] = row[k2];
        free(row);
    }
#pragma omp parallel for schedule(static)
    for (int k2 = 0; k2 < h2; k2++) {
        cplx *col = malloc(sizeof(cplx) * (size_t)n1);
        for (int j1 = 0; j1 < n1; j1++) col[j1] = out[(size_t)j1 * h2 + k2];
        orc_fft(n1, col, -1);
        for (int k1 = 0; k1 < n1; k1++) out[(size_t)k1 * h2 + k2] = col[k1];
        free(col);
    }
    return 0;
}

/* Unnormalised 2-D synthesis from a half spectrum:
 *   out[j1][j2] = sum over the full (Hermitian-extended) spectrum of
 *                 X[k1][k2] exp(+2 pi i (k1 j1/n1 + k2 j2/n2)),
 * with X[k1][-k2] = conj(X[-k1][k2]).  Columns first (first index), then rows
 * (second index), the order of Sec. 3.  Imaginary parts that a Hermitian
 * spectrum would not have are discarded by taking the real part.
 * orc_irfft2(orc_rfft2(x)) = n1 n2 x (pinned in the tests). */
int orc_irfft2(int n1, int n2, const cplx *in, double *out)
{
    if (!is_pow2(n1) || !is_pow2(n2)) return -1;
    int h2 = n2 / 2 + 1;
    cplx *tmp = malloc(sizeof(cplx) * (size_t)n1 * (size_t)h2);
#pragma omp parallel for schedule(static)
    for (int k2 = 0; k2 < h2; k2++) {
        cplx *col = malloc(sizeof(cplx) * (size_t)n1);
        for (int k1 = 0; k1 < n1; k1++) col[k1] = in[(size_t)k1 * h2 + k2];
        orc_fft(n1, col, +1);
        for (int j1 = 0; j1 < n1; j1++) tmp[(size_t)j1 * h2 + k2] = col[j1];
        free(col);
    }
#pragma omp parallel for schedule(static)
    for (int j1 = 0; j1 < n1; j1++) {
        cplx *row = malloc(sizeof(cplx) * (size_t)n2);
        const cplx *y = tmp + (size_t)j1 * h2;
        for (int k2 = 0; k2 < n2; k2++)
            row[k2] = (k2 <= n2 / 2) ? y[k2] : conj(y[n2 - k2]);
        orc_fft(n2, row, +1);
        for (int j2 = 0; j2 < n2; j2++) out[(size_t)j1 * n2 + j2] = creal(row[j2]);
        free(row);
    }
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Model pieces                                                             */
/* ------------------------------------------------------------------------ */

static size_t box_index(const orc_params *p, int k1, int k2)
{
    return (size_t)(k1 + p->K1) * (size_t)(p->K2 + 1) + (size_t)k2;
}

/* Validates the parameters; 0 if usable. */
int orc_check(const orc_params *p)
{
    if (!is_pow2(p->n1) || !is_pow2(p->n2)) return -1;
    if (p->K1 < 0 || p->K2 < 0) return -1;
    if (4 * p->K1 + 1 > p->n1 || 4 * p->K2 + 1 > p->n2) return -1;
    return 0;
}

/* Retained modes of a real field on the grid, the initial perturbation of
 * Sec. 2 (Phi(theta, phi, t0) = eps eta, |eta| <= 1 at every grid point):
 *   Phi_k = (1/(n1 n2)) sum_{j1,j2} field[j1][j2] exp(-2 pi i (k1 j1/n1 + k2 j2/n2))
 * for |k1| <= K1, 0 <= k2 <= K2 (orc_rfft2, then the box rows k1 mod n1).
 * On k2 = 0 the k1 < 0 entries are replaced by the conjugates of the k1 > 0
 * ones (Sec. 3's symmetrisation), the k = 0 slot is 0 and *mean is the k = 0
 * coefficient, the field's average.  Pinned by fields synthesised from known
 * coefficients by the definition of the series, and by the grid average. */
int orc_state_from_field(const orc_params *p, const double *field, cplx *state, double *mean)
{
    if (orc_check(p)) return -1;
    int h2 = p->n2 / 2 + 1;
    cplx *half = malloc(sizeof(cplx) * (size_t)p->n1 * (size_t)h2);
    if (!half) return -1;
    orc_rfft2(p->n1, p->n2, field, half);
    double inv = 1.0 / ((double)p->n1 * (double)p->n2);
    for (int k1 = -p->K1; k1 <= p->K1; k1++) {
        int row = (k1 + p->n1) % p->n1;
        for (int k2 = 0; k2 <= p->K2; k2++)
            state[box_index(p, k1, k2)] = half[(size_t)row * h2 + k2] * inv;
    }
    for (int k1 = 1; k1 <= p->K1; k1++)
        state[box_index(p, -k1, 0)] = conj(state[box_index(p, k1, 0)]);
    *mean = creal(half[0]) * inv;
    state[box_index(p, 0, 0)] = 0.0;
    free(half);
    return 0;
}

/* Scatters s*i*kappa_i*Phi_k (which = 1: kappa_1 = s1 k1, which = 2:
 * kappa_2 = s2 k2, which = 0: Phi itself with the mean mode) from the compact
 * box into the zero-padded half spectrum n1 x (n2/2+1): the augmented array
 * Psi of Sec. 3, rows indexed by k1 mod n1. */
static void scatter_box(const orc_params *p, const cplx *state, double mean,
                        int which, cplx *half)
{
    int h2 = p->n2 / 2 + 1;
    memset(half, 0, sizeof(cplx) * (size_t)p->n1 * (size_t)h2);
    for (int k1 = -p->K1; k1 <= p->K1; k1++) {
        int row = (k1 + p->n1) % p->n1;
        for (int k2 = 0; k2 <= p->K2; k2++) {
            cplx v = state[box_index(p, k1, k2)];
            if (k1 == 0 && k2 == 0) v = (which == 0) ? mean : 0.0;
            if (which == 1) v *= I * p->s1 * k1;
            if (which == 2) v *= I * p->s2 * k2;
            half[(size_t)row * h2 + k2] = v;
        }
    }
}

/* Nonlinear term through the FFT, Sec. 3 / eq. (SivCurv1c):
 *   u = d1 Phi, v = d2 Phi on the grid (synthesis of i kappa_i Phi_k),
 *   g = u^2 + v^2 = |grad Phi|^2,
 *   ghat = (1/(n1 n2)) * analysis(g) restricted to the box (incl. k = 0).
 * ghat is written in the compact layout, with ghat_0 (= mean of g) in the
 * k = 0 slot.  Pinned against orc_nonlinear_brute (the literal convolution
 * sum) and the single-cosine closed form. */
void orc_grad2_hat(const orc_params *p, const cplx *state, cplx *ghat)
{
    int n1 = p->n1, n2 = p->n2, h2 = n2 / 2 + 1;
    size_t ng = (size_t)n1 * (size_t)n2;
    cplx *half = malloc(sizeof(cplx) * (size_t)n1 * (size_t)h2);
    double *u = malloc(sizeof(double) * ng);
    double *v = malloc(sizeof(double) * ng);
    scatter_box(p, state, 0.0, 1, half);
    orc_irfft2(n1, n2, half, u);
    scatter_box(p, state, 0.0, 2, half);
    orc_irfft2(n1, n2, half, v);
    for (size_t q = 0; q < ng; q++) u[q] = u[q] * u[q] + v[q] * v[q];
    orc_rfft2(n1, n2, u, half);
    double scale = 1.0 / (double)ng;
    for (int k1 = -p->K1; k1 <= p->K1; k1++) {
        int row = (k1 + n1) % n1;
        for (int k2 = 0; k2 <= p->K2; k2++)
            ghat[box_index(p, k1, k2)] = half[(size_t)row * h2 + k2] * scale;
    }
    free(v);
    free(u);
    free(half);
}

/* Full-box coefficient: the compact half spectrum extended by
 * Phi_{-k} = conj(Phi_k); the k = 0 entry is `mean`. */
static cplx full_coef(const orc_params *p, const cplx *state, double mean,
                      int k1, int k2)
{
    if (k1 == 0 && k2 == 0) return mean;
    if (k2 >= 0) return state[box_index(p, k1, k2)];
    return conj(state[box_index(p, -k1, -k2)]);
}

/* The literal convolution sum of eq. (SivCurv1c), without FFTs:
 *   out_k = - sum_{l, k-l in the box} (kappa(l) . kappa(k-l)) Phi_l Phi_{k-l}
 * for every k of the compact box (k = 0 included), i.e. the coefficient of
 * |grad Phi|^2 (the factor c = 1/(2 r0^2) is applied by the caller).
 * O(K^4): for tiny boxes only. */
void orc_grad2_brute(const orc_params *p, const cplx *state, cplx *out)
{
    for (int k1 = -p->K1; k1 <= p->K1; k1++)
        for (int k2 = 0; k2 <= p->K2; k2++) {
            cplx acc = 0;
            for (int l1 = -p->K1; l1 <= p->K1; l1++)
                for (int l2 = -p->K2; l2 <= p->K2; l2++) {
                    int m1 = k1 - l1, m2 = k2 - l2;
                    if (m1 < -p->K1 || m1 > p->K1 || m2 < -p->K2 || m2 > p->K2)
                        continue;
                    double dot = p->s1 * l1 * p->s1 * m1 + p->s2 * l2 * p->s2 * m2;
                    acc += dot * full_coef(p, state, 0.0, l1, l2) *
                           full_coef(p, state, 0.0, m1, m2);
                }
            out[box_index(p, k1, k2)] = -acc;
        }
}

/* |kappa| and the linear growth rate of eq. (SivCurv1c):
 *   omega_k(t) = -|kappa|^2 / r0^2 + gamma |kappa| / (2 r0),  r0 = t. */
double orc_omega(const orc_params *p, int k1, int k2, double t)
{
    double a = p->s1 * k1, b = p->s2 * k2;
    double kk = sqrt(a * a + b * b);
    return -kk * kk / (t * t) + p->gamma * kk / (2.0 * t);
}

/* Time of step n: t_n = t0 + n dt, with n recovered from t by rounding. */
static long step_index(const orc_params *p, double t)
{
    return lround((t - p->t0) / p->dt);
}

/* Explicit Euler steps of eq. (SivCurv1c) with f = 0 (Sec. 2, Sec. 3):
 *   Phi_k <- Phi_k + dt (omega_k(t_n) Phi_k + c(t_n) ghat_k),  k != 0 in box
 *   Phi_0 <- Phi_0 + dt c(t_n) ghat_0           (omega_0 = 0)
 * then the symmetrization of Sec. 3 on the k2 = 0 column (k1 > 0 is the
 * master, Phi_{-k1,0} = conj(Phi_{k1,0})), the k = 0 slot set to 0, and
 * t <- t0 + (n+1) dt.  Pinned by the brute-force right-hand side, the linear
 * closed forms, translation/reflection invariance and mean-mode properties. */
void orc_step(const orc_params *p, cplx *state, double *mean, double *t,
              int nsteps)
{
    size_t nb = (size_t)(2 * p->K1 + 1) * (size_t)(p->K2 + 1);
    cplx *ghat = malloc(sizeof(cplx) * nb);
    for (int s = 0; s < nsteps; s++) {
        long n = step_index(p, *t);
        double tn = p->t0 + (double)n * p->dt;
        double c = 1.0 / (2.0 * tn * tn);
        int lin = !(p->flags & ORC_NONLINEAR_ONLY);
        int nl = !(p->flags & ORC_LINEAR_ONLY);
        if (nl) orc_grad2_hat(p, state, ghat);
        else memset(ghat, 0, sizeof(cplx) * nb);
        for (int k1 = -p->K1; k1 <= p->K1; k1++)
            for (int k2 = 0; k2 <= p->K2; k2++) {
                if (k1 == 0 && k2 == 0) continue;
                size_t q = box_index(p, k1, k2);
                cplx rhs = c * ghat[q];
                if (lin) rhs += orc_omega(p, k1, k2, tn) * state[q];
                state[q] += p->dt * rhs;
            }
        *mean += p->dt * c * creal(ghat[box_index(p, 0, 0)]);
        for (int k1 = 1; k1 <= p->K1; k1++)
            state[box_index(p, -k1, 0)] = conj(state[box_index(p, k1, 0)]);
        state[box_index(p, 0, 0)] = 0;
        *t = p->t0 + (double)(n + 1) * p->dt;
    }
    free(ghat);
}

/* Physical fields on the grid: phi (with the mean mode), d1 phi, d2 phi. */
static void physical_fields(const orc_params *p, const cplx *state, double mean,
                            double *phi, double *u, double *v)
{
    int h2 = p->n2 / 2 + 1;
    cplx *half = malloc(sizeof(cplx) * (size_t)p->n1 * (size_t)h2);
    if (phi) { scatter_box(p, state, mean, 0, half); orc_irfft2(p->n1, p->n2, half, phi); }
    if (u) { scatter_box(p, state, mean, 1, half); orc_irfft2(p->n1, p->n2, half, u); }
    if (v) { scatter_box(p, state, mean, 2, half); orc_irfft2(p->n1, p->n2, half, v); }
    free(half);
}

/* Unnormalised analysis restricted to the box: out_k = sum_x a(x) e^{-i k.x},
 * scaled by `scale` and multiplied by (-i kappa_which) for which = 1, 2. */
static void gather_box(const orc_params *p, const double *a, int which,
                       double scale, cplx *out, int accumulate)
{
    int n1 = p->n1, h2 = p->n2 / 2 + 1;
    cplx *half = malloc(sizeof(cplx) * (size_t)n1 * (size_t)h2);
    orc_rfft2(n1, p->n2, a, half);
    for (int k1 = -p->K1; k1 <= p->K1; k1++) {
        int row = (k1 + n1) % n1;
        for (int k2 = 0; k2 <= p->K2; k2++) {
            cplx z = half[(size_t)row * h2 + k2] * scale;
            if (which == 1) z *= -I * p->s1 * k1;
            if (which == 2) z *= -I * p->s2 * k2;
            size_t q = box_index(p, k1, k2);
            out[q] = accumulate ? out[q] + z : z;
        }
    }
    free(half);
}

/* Flame surface area in the model's equatorial geometry (project-defined
 * objective; the paper fixes none):
 *   A = sum_grid w R sqrt(R^2 + |grad Phi|^2),  R = r0(t) + Phi(x),
 *   w = (2 pi)^2 / (n1 n2 s1 s2).
 * If grad != NULL it receives dA/dPhi_k for the real inner product
 * <X, Y> = Re sum_{all k} conj(X_k) Y_k over the full spectrum (so a
 * Hermitian direction d has dA = sum_{k2=0} Re(conj(g) d) + 2 sum_{k2>0} ...),
 * with dA/dPhi_0 in *grad_mean and in the k = 0 slot of grad.
 * Pinned by A(Phi = 0) = (2 pi)^2 r0^2/(s1 s2), the small-amplitude cosine
 * expansion, and central finite differences. */
double orc_area(const orc_params *p, const cplx *state, double mean, double t,
                cplx *grad, double *grad_mean)
{
    size_t ng = (size_t)p->n1 * (size_t)p->n2;
    double *phi = malloc(sizeof(double) * ng);
    double *u = malloc(sizeof(double) * ng);
    double *v = malloc(sizeof(double) * ng);
    physical_fields(p, state, mean, phi, u, v);
    double w = TWO_PI * TWO_PI / ((double)ng * p->s1 * p->s2);
    /* Neumaier-compensated sum: the area is ~(2 pi r0)^2 while central
     * differences of it at h = 1e-6 resolve changes ~1e-13 of that. */
    double area = 0.0, comp = 0.0;
    for (size_t q = 0; q < ng; q++) {
        double R = t + phi[q];
        double G = u[q] * u[q] + v[q] * v[q];
        double S = sqrt(R * R + G);
        double term = w * R * S;
        double sum = area + term;
        comp += (fabs(area) >= fabs(term)) ? (area - sum) + term : (term - sum) + area;
        area = sum;
        if (grad) {
            phi[q] = w * (S + R * R / S); /* dA/dphi     */
            u[q] = w * R * u[q] / S;      /* dA/d(d1 phi) */
            v[q] = w * R * v[q] / S;      /* dA/d(d2 phi) */
        }
    }
    if (grad) {
        gather_box(p, phi, 0, 1.0, grad, 0);
        gather_box(p, u, 1, 1.0, grad, 1);
        gather_box(p, v, 2, 1.0, grad, 1);
        if (grad_mean) *grad_mean = creal(grad[box_index(p, 0, 0)]);
    }
    free(v);
    free(u);
    free(phi);
    return area + comp;
}

/* Transposed Jacobian of one Euler step at state (state, t_n), applied to
 * lambda (box incl. k = 0 in the k = 0 slot), in place:
 *   lambda <- lambda + dt (omega_k lambda_k
 *             + c sum_i (-i kappa_i) ghat_i),  ghat_i = analysis of
 *             2 ell(x) d_i phi(x) / (n1 n2),  ell = synthesis of lambda.
 * The adjoint of the step under the full-spectrum inner product: the
 * transpose of orc_step_jvp term by term.  *dgamma accumulates
 * <lambda_in, dt (|kappa|/(2 r0)) Phi> (the gamma-derivative of the step).
 * Pinned by the dot-product test against orc_step_jvp and by finite
 * differences. */
void orc_step_vjp(const orc_params *p, const cplx *state, double t, cplx *lam,
                  double *dgamma)
{
    size_t ng = (size_t)p->n1 * (size_t)p->n2;
    size_t nb = (size_t)(2 * p->K1 + 1) * (size_t)(p->K2 + 1);
    long n = step_index(p, t);
    double tn = p->t0 + (double)n * p->dt;
    double c = 1.0 / (2.0 * tn * tn);
    int lin = !(p->flags & ORC_NONLINEAR_ONLY);
    int nl = !(p->flags & ORC_LINEAR_ONLY);
    cplx *acc = calloc(nb, sizeof(cplx));
    if (nl) {
        double *u = malloc(sizeof(double) * ng);
        double *v = malloc(sizeof(double) * ng);
        double *ell = malloc(sizeof(double) * ng);
        physical_fields(p, state, 0.0, NULL, u, v);
        double lam0 = creal(lam[box_index(p, 0, 0)]);
        physical_fields(p, lam, lam0, ell, NULL, NULL);
        for (size_t q = 0; q < ng; q++) {
            u[q] = 2.0 * ell[q] * u[q];
            v[q] = 2.0 * ell[q] * v[q];
        }
        gather_box(p, u, 1, 1.0 / (double)ng, acc, 0);
        gather_box(p, v, 2, 1.0 / (double)ng, acc, 1);
        free(ell);
        free(v);
        free(u);
    }
    double dg = 0.0;
    for (int k1 = -p->K1; k1 <= p->K1; k1++)
        for (int k2 = 0; k2 <= p->K2; k2++) {
            size_t q = box_index(p, k1, k2);
            double wgt = (k2 == 0) ? 1.0 : 2.0;
            if (k1 == 0 && k2 == 0) continue; /* omega_0 = 0, kappa = 0 */
            double a = p->s1 * k1, b = p->s2 * k2;
            double kk = sqrt(a * a + b * b);
            if (lin)
                dg += wgt * creal(conj(lam[q]) * p->dt * (kk / (2.0 * tn)) * state[q]);
            cplx upd = c * acc[q];
            if (lin) upd += orc_omega(p, k1, k2, tn) * lam[q];
            lam[q] += p->dt * upd;
        }
    if (dgamma) *dgamma += dg;
    free(acc);
}

/* Jacobian of one Euler step applied to a direction d (box incl. k = 0),
 * in place, at (state, t_n):
 *   d <- d + dt (omega_k d_k + c ghat'_k),  ghat' = analysis of
 *   2 grad(phi) . grad(delta phi) / (n1 n2).
 * Used only to pin orc_step_vjp by the dot-product identity. */
void orc_step_jvp(const orc_params *p, const cplx *state, double t, cplx *d)
{
    size_t ng = (size_t)p->n1 * (size_t)p->n2;
    size_t nb = (size_t)(2 * p->K1 + 1) * (size_t)(p->K2 + 1);
    long n = step_index(p, t);
    double tn = p->t0 + (double)n * p->dt;
    double c = 1.0 / (2.0 * tn * tn);
    int lin = !(p->flags & ORC_NONLINEAR_ONLY);
    int nl = !(p->flags & ORC_LINEAR_ONLY);
    cplx *gh = calloc(nb, sizeof(cplx));
    if (nl) {
        double *u = malloc(sizeof(double) * ng), *v = malloc(sizeof(double) * ng);
        double *du = malloc(sizeof(double) * ng), *dv = malloc(sizeof(double) * ng);
        physical_fields(p, state, 0.0, NULL, u, v);
        physical_fields(p, d, 0.0, NULL, du, dv);
        for (size_t q = 0; q < ng; q++) u[q] = 2.0 * (u[q] * du[q] + v[q] * dv[q]);
        gather_box(p, u, 0, 1.0 / (double)ng, gh, 0);
        free(dv); free(du); free(v); free(u);
    }
    for (int k1 = -p->K1; k1 <= p->K1; k1++)
        for (int k2 = 0; k2 <= p->K2; k2++) {
            size_t q = box_index(p, k1, k2);
            cplx upd = c * gh[q];
            if (lin && !(k1 == 0 && k2 == 0)) upd += orc_omega(p, k1, k2, tn) * d[q];
            d[q] += p->dt * upd;
        }
    free(gh);
}

/* Reverse-mode gradient of the final area over nsteps Euler steps:
 *   L = A(Phi(T)),  T = t0 + nsteps dt  (starting at *t_start = t of state0).
 * Stores the whole forward trajectory (plain, memory O(nsteps)), then walks
 * it backwards with orc_step_vjp.  Outputs dL/dPhi(t0) (compact box, k = 0
 * slot = dL/dPhi_0), dL/dgamma and L.  Pinned by central finite
 * differences of orc_step + orc_area. */
double orc_area_grad(const orc_params *p, const cplx *state0, double mean0,
                     double t_start, int nsteps, cplx *grad, double *grad_gamma)
{
    size_t nb = (size_t)(2 * p->K1 + 1) * (size_t)(p->K2 + 1);
    cplx *traj = malloc(sizeof(cplx) * nb * (size_t)(nsteps + 1));
    double *ts = malloc(sizeof(double) * (size_t)(nsteps + 1));
    double mean = mean0, t = t_start;
    memcpy(traj, state0, sizeof(cplx) * nb);
    traj[box_index(p, 0, 0)] = 0;
    ts[0] = t;
    for (int s = 0; s < nsteps; s++) {
        memcpy(traj + nb * (size_t)(s + 1), traj + nb * (size_t)s, sizeof(cplx) * nb);
        orc_step(p, traj + nb * (size_t)(s + 1), &mean, &t, 1);
        ts[s + 1] = t;
    }
    double gm = 0.0;
    double L = orc_area(p, traj + nb * (size_t)nsteps, mean, t, grad, &gm);
    grad[box_index(p, 0, 0)] = gm;
    double dg = 0.0;
    for (int s = nsteps - 1; s >= 0; s--)
        orc_step_vjp(p, traj + nb * (size_t)s, ts[s], grad, &dg);
    if (grad_gamma) *grad_gamma = dg;
    free(ts);
    free(traj);
    return L;
}
