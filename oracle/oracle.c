/*
 * FP64 CPU oracle for the pseudo-spectral Navier-Stokes solver of
 * Mortensen, "Massively parallel implementation in Python of a
 * pseudo-spectral DNS code for turbulent flows" (EuroSciPy 2015).
 *
 * TEST INFRASTRUCTURE ONLY: plain, slow, obviously correct.  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU legs may load it.  It shares
 * no code with the CUDA library.  Every routine follows the paper's
 * definitions in the paper's order:
 *   Eq. realmesh / wavemesh   mesh and wavenumbers (Sec. 2)
 *   Eq. ffteq                 transform pair, forward unnormalised,
 *                             inverse carries 1/N^3; axis order
 *                             F = F_kx(F_ky(F_kz(u))), inverse reversed
 *   Eq. eqNS                  rotational form, omega = curl u
 *   Eq. pressure / NSfinal    pressure elimination -> Leray projection
 *   Sec. 3.4 cross listing    c0 = a1 b2 - a2 b1, c1 = a2 b0 - a0 b2,
 *                             c2 = a0 b1 - a1 b0
 *   Sec. 2 (end)              fourth-order Runge-Kutta integrator
 * Readings where the paper is silent (2/3 rule, k = 0, RK4 variant,
 * diagnostics) are listed in the design notes and restated at each use.
 *
 * OR_MUTANT (compile-time, default 0) plants one deliberate mistake; the
 * test suite builds each mutant and checks that some pin rejects it.
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef OR_MUTANT
#define OR_MUTANT 0
#endif

typedef double complex cplx;

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* 1D FFT: recursive decimation in time on the smallest prime factor.  */
/* ------------------------------------------------------------------ */

static int smallest_factor(int n) {
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* tw[j] = exp(sign * 2 pi i j / n_top), j = 0..n_top-1.  At a recursion
 * level of length n, w_n^j = tw[j * (n_top / n)]. */
static cplx *make_twiddles(int n, int sign) {
    cplx *tw = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!tw) return NULL;
    for (int j = 0; j < n; ++j) {
        double a = 2.0 * M_PI * (double)j / (double)n;
        tw[j] = cos(a) + (double)sign * sin(a) * I;
    }
    return tw;
}

/* out[k] = sum_j in[j*istride] w_n^{jk}, k = 0..n-1, with
 * w_n^m = tw[(m mod n) * twstep].  Textbook Cooley-Tukey: for n = p*m,
 * split x into the p subsequences x[p*j + r]; with Y_r their m-point DFTs,
 *   X[k + q*m] = sum_r w_n^{r*(k + q*m)} Y_r[k],  k < m, q < p. */
static void fft_rec(int n, const cplx *in, long istride, cplx *out,
                    const cplx *tw, long twstep) {
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int p = smallest_factor(n);
    int m = n / p;
    if (p == n) { /* prime length: direct DFT */
        for (int k = 0; k < n; ++k) {
            cplx s = 0.0;
            for (int j = 0; j < n; ++j)
                s += in[(long)j * istride] * tw[(long)(((long)j * k) % n) * twstep];
            out[k] = s;
        }
        return;
    }
    for (int r = 0; r < p; ++r)
        fft_rec(m, in + (long)r * istride, istride * p, out + (long)r * m, tw,
                twstep * p);
    cplx y[64]; /* p <= 3 for the sizes used here; any p < 64 works */
    cplx *yy = (p <= 64) ? y : (cplx *)malloc(sizeof(cplx) * (size_t)p);
    for (int k = 0; k < m; ++k) {
        for (int r = 0; r < p; ++r) yy[r] = out[(long)r * m + k];
        for (int q = 0; q < p; ++q) {
            cplx s = 0.0;
            for (int r = 0; r < p; ++r) {
                long e = ((long)r * (k + (long)q * m)) % n;
#if OR_MUTANT == 1 /* planted: drop the twiddle of the combine step */
                e = ((long)r * q * m) % n;
#endif
                s += yy[r] * tw[e * twstep];
            }
            out[k + (long)q * m] = s;
        }
    }
    if (yy != y) free(yy);
}

/* Transform n values read at stride `stride` from x, in place, with a
 * precomputed table.  work: 2n complex of thread-private scratch. */
static void fft_strided(int n, cplx *x, long stride, const cplx *tw, cplx *work) {
    cplx *a = work, *b = work + n;
    for (int j = 0; j < n; ++j) a[j] = x[(long)j * stride];
    fft_rec(n, a, 1, b, tw, 1);
    for (int j = 0; j < n; ++j) x[(long)j * stride] = b[j];
}

int or_fft1d(int n, double *x, int sign) {
    if (n < 1 || (sign != 1 && sign != -1) || !x) return -1;
    cplx *tw = make_twiddles(n, sign);
    cplx *work = (cplx *)malloc(sizeof(cplx) * 2 * (size_t)n);
    if (!tw || !work) {
        free(tw);
        free(work);
        return -2;
    }
    fft_strided(n, (cplx *)x, 1, tw, work);
    free(tw);
    free(work);
    return 0;
}

int or_dft1d(int n, const double *x, double *y, int sign) {
    if (n < 1 || (sign != 1 && sign != -1) || !x || !y) return -1;
    const cplx *a = (const cplx *)x;
    cplx *b = (cplx *)y;
    for (int k = 0; k < n; ++k) {
        cplx s = 0.0;
        for (int j = 0; j < n; ++j) {
            double ang = 2.0 * M_PI * (double)(((long)j * k) % n) / (double)n;
            s += a[j] * (cos(ang) + (double)sign * sin(ang) * I);
        }
        b[k] = s;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* 3D real transforms, Eq. ffteq and the axis order that follows it.  */
/* ------------------------------------------------------------------ */

/* Pass of 1D transforms along one axis of a complex [n0][n1][n2] array:
 * axis 0 (x), 1 (y) or 2 (z). */
static int fft_axis(cplx *a, int n0, int n1, int n2, int axis, int sign) {
    int n = (axis == 0) ? n0 : (axis == 1) ? n1 : n2;
    long stride = (axis == 0) ? (long)n1 * n2 : (axis == 1) ? n2 : 1;
    long nlines = (long)n0 * n1 * n2 / n;
    cplx *tw = make_twiddles(n, sign);
    if (!tw) return -2;
    int fail = 0;
#pragma omp parallel
    {
        cplx *work = (cplx *)malloc(sizeof(cplx) * 2 * (size_t)n);
        if (!work) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(static)
            for (long l = 0; l < nlines; ++l) {
                long base;
                if (axis == 0) base = l;                     /* l = (y, z) */
                else if (axis == 1) base = (l / n2) * (long)n1 * n2 + (l % n2); /* l = (x, z) */
                else base = l * n2;                          /* l = (x, y) */
                fft_strided(n, a + base, stride, tw, work);
            }
            free(work);
        }
    }
    free(tw);
    return fail ? -2 : 0;
}

int or_rfftn(int N, const double *u, double *uhat) {
    if (N < 1 || !u || !uhat) return -1;
    const int Nh = N / 2 + 1;
    cplx *h = (cplx *)uhat;
    cplx *tw = make_twiddles(N, -1);
    if (!tw) return -2;
    int fail = 0;
    /* F_kz: real lines along z, keep kz = 0..N/2 */
#pragma omp parallel
    {
        cplx *work = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)N);
        if (!work) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(static)
            for (long l = 0; l < (long)N * N; ++l) {
                cplx *line = work + 2 * N;
                for (int z = 0; z < N; ++z) line[z] = u[l * N + z];
                fft_strided(N, line, 1, tw, work);
                for (int k = 0; k < Nh; ++k) h[l * Nh + k] = line[k];
            }
            free(work);
        }
    }
    free(tw);
    if (fail) return -2;
    int rc = fft_axis(h, N, N, Nh, 1, -1); /* F_ky */
    if (rc) return rc;
    return fft_axis(h, N, N, Nh, 0, -1); /* F_kx */
}

int or_irfftn(int N, const double *uhat, double *u) {
    if (N < 1 || !u || !uhat) return -1;
    const int Nh = N / 2 + 1;
    const long nspec = (long)N * N * Nh;
    cplx *h = (cplx *)malloc(sizeof(cplx) * (size_t)nspec);
    cplx *tw = make_twiddles(N, +1);
    if (!h || !tw) {
        free(h);
        free(tw);
        return -2;
    }
    memcpy(h, uhat, sizeof(cplx) * (size_t)nspec);
    int rc = fft_axis(h, N, N, Nh, 0, +1); /* F^-1_x */
    if (!rc) rc = fft_axis(h, N, N, Nh, 1, +1); /* F^-1_y */
    const double scale = 1.0 / ((double)N * N * N);
    int fail = 0;
    /* F^-1_z: real output.  The half line is extended by Hermitian symmetry,
     * X[N-k] = conj(X[k]), transformed as a complex line, and the real part
     * kept (the imaginary parts of X[0] and X[N/2] only feed Im). */
    if (!rc) {
#pragma omp parallel
        {
            cplx *work = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)N);
            if (!work) {
#pragma omp atomic write
                fail = 1;
            } else {
#pragma omp for schedule(static)
                for (long l = 0; l < (long)N * N; ++l) {
                    cplx *line = work + 2 * N;
                    for (int k = 0; k < N; ++k)
                        line[k] = (k < Nh) ? h[l * Nh + k] : conj(h[l * Nh + (N - k)]);
                    fft_strided(N, line, 1, tw, work);
                    for (int z = 0; z < N; ++z) u[l * N + z] = creal(line[z]) * scale;
                }
                free(work);
            }
        }
    }
    free(h);
    free(tw);
    return rc ? rc : (fail ? -2 : 0);
}

int or_dft3_real(int N, const double *u, double *uhat) {
    if (N < 1 || !u || !uhat) return -1;
    const int Nh = N / 2 + 1;
    cplx *h = (cplx *)uhat;
#pragma omp parallel for collapse(2) schedule(static)
    for (int kx = 0; kx < N; ++kx)
        for (int ky = 0; ky < N; ++ky)
            for (int kz = 0; kz < Nh; ++kz) {
                cplx s = 0.0;
                for (int x = 0; x < N; ++x)
                    for (int y = 0; y < N; ++y)
                        for (int z = 0; z < N; ++z) {
                            long e = ((long)kx * x + (long)ky * y + (long)kz * z) % N;
                            double ang = -2.0 * M_PI * (double)e / (double)N;
                            s += u[((long)x * N + y) * N + z] * (cos(ang) + sin(ang) * I);
                        }
                h[((long)kx * N + ky) * Nh + kz] = s;
            }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Right-hand side of Eq. NSfinal.                                     */
/* ------------------------------------------------------------------ */

/* Eq. wavemesh: k in {-N/2+1, ..., N/2}; index i in FFT order. */
static int wavenumber(int i, int N) { return (i <= N / 2) ? i : i - N; }

/* 2/3 rule (the paper only says "the same dealiasing as Tarang"; the
 * reading used is Orszag's cubic truncation): keep k iff 3|k_i| < N. */
static int keep(int kx, int ky, int kz, int N) {
#if OR_MUTANT == 2 /* planted: off-by-one cutoff (3|k| <= N) */
    return 3 * abs(kx) <= N && 3 * abs(ky) <= N && 3 * abs(kz) <= N;
#else
    return 3 * abs(kx) < N && 3 * abs(ky) < N && 3 * abs(kz) < N;
#endif
}

int or_nonlinear(int N, const double *uhat, double *nhat) {
    if (N < 2 || (N & 1) || !uhat || !nhat) return -1;
    const int Nh = N / 2 + 1;
    const long ns = (long)N * N * Nh, np = (long)N * N * N;
    const cplx *U = (const cplx *)uhat;
    cplx *W = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)ns);
    double *u = (double *)malloc(sizeof(double) * 3 * (size_t)np);
    double *w = (double *)malloc(sizeof(double) * 3 * (size_t)np);
    int rc = (!W || !u || !w) ? -2 : 0;
    if (!rc) {
        /* omega^ = i k x uhat (Eq. eqNS: omega = curl u) */
#pragma omp parallel for collapse(2) schedule(static)
        for (int ix = 0; ix < N; ++ix)
            for (int iy = 0; iy < N; ++iy)
                for (int iz = 0; iz < Nh; ++iz) {
                    const double kx = wavenumber(ix, N), ky = wavenumber(iy, N), kz = iz;
                    const long m = ((long)ix * N + iy) * Nh + iz;
                    const cplx ux = U[m], uy = U[ns + m], uz = U[2 * ns + m];
#if OR_MUTANT == 3 /* planted: transposed operands in the curl's x component */
                    W[m] = I * (kz * uy - ky * uz);
#else
                    W[m] = I * (ky * uz - kz * uy);
#endif
                    W[ns + m] = I * (kz * ux - kx * uz);
                    W[2 * ns + m] = I * (kx * uy - ky * ux);
                }
        /* u = F^-1(uhat), omega = F^-1(omega^) */
        for (int c = 0; c < 3 && !rc; ++c) {
            rc = or_irfftn(N, (const double *)(U + c * ns), u + c * np);
            if (!rc) rc = or_irfftn(N, (const double *)(W + c * ns), w + c * np);
        }
    }
    if (!rc) {
        /* u x omega pointwise, component order of the Sec. 3.4 cross listing;
         * the result overwrites omega. */
#pragma omp parallel for schedule(static)
        for (long p = 0; p < np; ++p) {
            const double a0 = u[p], a1 = u[np + p], a2 = u[2 * np + p];
            const double b0 = w[p], b1 = w[np + p], b2 = w[2 * np + p];
#if OR_MUTANT == 4 /* planted: omega x u instead of u x omega */
            w[p] = b1 * a2 - b2 * a1;
            w[np + p] = b2 * a0 - b0 * a2;
            w[2 * np + p] = b0 * a1 - b1 * a0;
#else
            w[p] = a1 * b2 - a2 * b1;
            w[np + p] = a2 * b0 - a0 * b2;
            w[2 * np + p] = a0 * b1 - a1 * b0;
#endif
        }
        for (int c = 0; c < 3 && !rc; ++c)
            rc = or_rfftn(N, w + c * np, nhat + 2 * c * ns);
    }
    free(W);
    free(u);
    free(w);
    return rc;
}

int or_rhs(int N, double nu, const double *uhat, double *duhat) {
    if (N < 2 || (N & 1) || !uhat || !duhat) return -1;
    const int Nh = N / 2 + 1;
    const long ns = (long)N * N * Nh;
    int rc = or_nonlinear(N, uhat, duhat);
    if (rc) return rc;
    const cplx *U = (const cplx *)uhat;
    cplx *D = (cplx *)duhat;
#pragma omp parallel for collapse(2) schedule(static)
    for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy)
            for (int iz = 0; iz < Nh; ++iz) {
                const int kx = wavenumber(ix, N), ky = wavenumber(iy, N), kz = iz;
                const long m = ((long)ix * N + iy) * Nh + iz;
                const double k2 = (double)kx * kx + (double)ky * ky + (double)kz * kz;
                /* dealias the nonlinear term */
                const double msk = keep(kx, ky, kz, N) ? 1.0 : 0.0;
                cplx n0 = msk * D[m], n1 = msk * D[ns + m], n2 = msk * D[2 * ns + m];
                /* Eq. pressure / NSfinal: subtract k (k . N^)/|k|^2; at k = 0
                 * the numerator is 0, so |k|^2 is replaced by 1 there. */
                const cplx kdotn = kx * n0 + ky * n1 + kz * n2;
                const double inv = 1.0 / (k2 > 0.0 ? k2 : 1.0);
#if OR_MUTANT == 5 /* planted: projection with the wrong sign */
                n0 += kx * kdotn * inv;
                n1 += ky * kdotn * inv;
                n2 += kz * kdotn * inv;
#else
                n0 -= kx * kdotn * inv;
                n1 -= ky * kdotn * inv;
                n2 -= kz * kdotn * inv;
#endif
                /* viscous term -nu |k|^2 uhat */
#if OR_MUTANT == 6 /* planted: viscous term dropped from the z component */
                D[m] = n0 - nu * k2 * U[m];
                D[ns + m] = n1 - nu * k2 * U[ns + m];
                D[2 * ns + m] = n2;
#else
                D[m] = n0 - nu * k2 * U[m];
                D[ns + m] = n1 - nu * k2 * U[ns + m];
                D[2 * ns + m] = n2 - nu * k2 * U[2 * ns + m];
#endif
            }
    return 0;
}

/* Classical fourth-order Runge-Kutta (the paper names a fourth-order RK
 * method; the classical tableau is the reading):
 *   U1 = U0;  for s = 0..3:  dU = rhs(U);  U1 += a_s dt dU;
 *                            U = U0 + b_s dt dU (s < 3);
 *   U = U1;   a = (1/6, 1/3, 1/3, 1/6), b = (1/2, 1/2, 1). */
int or_rk4(int N, double nu, double dt, int nsteps, double *uhat) {
    if (N < 2 || (N & 1) || !uhat || nsteps < 0) return -1;
    const long n = 3L * N * N * (N / 2 + 1);
    const double a[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
#if OR_MUTANT == 7 /* planted: explicit-midpoint-like stage weights */
    const double b[3] = {0.5, 0.5, 0.5};
#else
    const double b[3] = {0.5, 0.5, 1.0};
#endif
    cplx *U = (cplx *)uhat;
    cplx *U0 = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *U1 = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *dU = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    int rc = (!U0 || !U1 || !dU) ? -2 : 0;
    for (int step = 0; step < nsteps && !rc; ++step) {
        memcpy(U0, U, sizeof(cplx) * (size_t)n);
        memcpy(U1, U, sizeof(cplx) * (size_t)n);
        for (int s = 0; s < 4 && !rc; ++s) {
            rc = or_rhs(N, nu, (const double *)U, (double *)dU);
            if (rc) break;
#pragma omp parallel for schedule(static)
            for (long m = 0; m < n; ++m) {
                U1[m] += a[s] * dt * dU[m];
                if (s < 3) U[m] = U0[m] + b[s] * dt * dU[m];
            }
        }
        if (!rc) memcpy(U, U1, sizeof(cplx) * (size_t)n);
    }
    free(U0);
    free(U1);
    free(dU);
    return rc;
}

/* Integrating-factor RK4 (Lawson).  The paper allows any integrator
 * (end of Sec. 2); with L = nu |k|^2 and v = exp(L t) uhat, Eq. NSfinal
 * becomes dv/dt = exp(L t) NL(exp(-L t) v), NL(u) = P(m (u x omega)^), and
 * classical RK4 on v over one step, written back in uhat with
 * E1 = exp(-L dt/2), E2 = exp(-L dt), reads
 *   k1 = NL(u_n)
 *   k2 = NL(E1 (u_n + dt/2 k1))
 *   k3 = NL(E1 u_n + dt/2 k2)
 *   k4 = NL(E2 u_n + dt E1 k3)
 *   u_{n+1} = E2 u_n + dt/6 (E2 k1 + 2 E1 k2 + 2 E1 k3 + k4).
 * The viscous decay is exact; NL is or_rhs with nu = 0. */
int or_rk4_if(int N, double nu, double dt, int nsteps, double *uhat) {
    if (N < 2 || (N & 1) || !uhat || nsteps < 0) return -1;
    const int Nh = N / 2 + 1;
    const long ns = (long)N * N * Nh, n = 3 * ns;
    cplx *U = (cplx *)uhat;
    cplx *U0 = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *U1 = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *K = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    double *E1 = (double *)malloc(sizeof(double) * (size_t)ns);
    double *E2 = (double *)malloc(sizeof(double) * (size_t)ns);
    int rc = (!U0 || !U1 || !K || !E1 || !E2) ? -2 : 0;
    if (!rc) {
        for (long m = 0; m < ns; ++m) {
            const int iz = (int)(m % Nh), iy = (int)((m / Nh) % N), ix = (int)(m / ((long)Nh * N));
            const double kx = wavenumber(ix, N), ky = wavenumber(iy, N), kz = iz;
            const double L = nu * (kx * kx + ky * ky + kz * kz);
            E1[m] = exp(-L * dt / 2.0);
            E2[m] = exp(-L * dt);
        }
    }
    for (int step = 0; step < nsteps && !rc; ++step) {
        memcpy(U0, U, sizeof(cplx) * (size_t)n);
        for (int s = 0; s < 4 && !rc; ++s) {
            rc = or_rhs(N, 0.0, (const double *)U, (double *)K);
            if (rc) break;
#pragma omp parallel for schedule(static)
            for (long e = 0; e < n; ++e) {
                const long m = e % ns;
                const double e1 = E1[m], e2 = E2[m];
                if (s == 0) {
                    U1[e] = e2 * U0[e] + (dt / 6.0) * e2 * K[e];
                    U[e] = e1 * (U0[e] + (dt / 2.0) * K[e]);
                } else if (s == 1) {
                    U1[e] += (dt / 3.0) * e1 * K[e];
                    U[e] = e1 * U0[e] + (dt / 2.0) * K[e];
                } else if (s == 2) {
                    U1[e] += (dt / 3.0) * e1 * K[e];
                    U[e] = e2 * U0[e] + dt * e1 * K[e];
                } else {
                    U1[e] += (dt / 6.0) * K[e];
                }
            }
        }
        if (!rc) memcpy(U, U1, sizeof(cplx) * (size_t)n);
    }
    free(U0);
    free(U1);
    free(K);
    free(E1);
    free(E2);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Diagnostics.  The paper defines none; the readings are:             */
/*   E   = <|u|^2>/2        = sum_k w |uhat|^2 / (2 N^6)               */
/*   eps = nu <|grad u|^2>  = nu sum_k w |k|^2 |uhat|^2 / N^6          */
/*   E(s) = sum over |k| in [s-1/2, s+1/2) of w |uhat|^2 / (2 N^6)     */
/* with w = 1 on the kz = 0 and kz = N/2 planes and 2 elsewhere (the    */
/* half spectrum stands for the full one by Hermitian symmetry).       */
/* ------------------------------------------------------------------ */

static double mode_weight(int iz, int N) { return (iz == 0 || 2 * iz == N) ? 1.0 : 2.0; }

int or_energy(int N, const double *uhat, double *E) {
    if (N < 2 || !uhat || !E) return -1;
    const int Nh = N / 2 + 1;
    const long ns = (long)N * N * Nh;
    const cplx *U = (const cplx *)uhat;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (long m = 0; m < ns; ++m) {
        const double w = mode_weight((int)(m % Nh), N);
        for (int c = 0; c < 3; ++c) {
            const cplx v = U[c * ns + m];
            s += w * (creal(v) * creal(v) + cimag(v) * cimag(v));
        }
    }
    const double N3 = (double)N * N * N;
    *E = s / (2.0 * N3 * N3);
    return 0;
}

int or_dissipation(int N, double nu, const double *uhat, double *eps) {
    if (N < 2 || !uhat || !eps) return -1;
    const int Nh = N / 2 + 1;
    const long ns = (long)N * N * Nh;
    const cplx *U = (const cplx *)uhat;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (long m = 0; m < ns; ++m) {
        const int iz = (int)(m % Nh), iy = (int)((m / Nh) % N), ix = (int)(m / ((long)Nh * N));
        const double kx = wavenumber(ix, N), ky = wavenumber(iy, N), kz = iz;
        const double k2 = kx * kx + ky * ky + kz * kz;
        const double w = mode_weight(iz, N);
        for (int c = 0; c < 3; ++c) {
            const cplx v = U[c * ns + m];
            s += w * k2 * (creal(v) * creal(v) + cimag(v) * cimag(v));
        }
    }
    const double N3 = (double)N * N * N;
    *eps = nu * s / (N3 * N3);
    return 0;
}

int or_spectrum(int N, const double *uhat, double *Ek, int nshells) {
    if (N < 2 || !uhat || !Ek || nshells < 1) return -1;
    const int Nh = N / 2 + 1;
    const long ns = (long)N * N * Nh;
    const cplx *U = (const cplx *)uhat;
    const double N3 = (double)N * N * N;
    for (int s = 0; s < nshells; ++s) Ek[s] = 0.0;
    for (long m = 0; m < ns; ++m) { /* serial: fixed summation order */
        const int iz = (int)(m % Nh), iy = (int)((m / Nh) % N), ix = (int)(m / ((long)Nh * N));
        const double kx = wavenumber(ix, N), ky = wavenumber(iy, N), kz = iz;
        const int shell = (int)floor(sqrt(kx * kx + ky * ky + kz * kz) + 0.5);
        if (shell >= nshells) continue;
        double e = 0.0;
        for (int c = 0; c < 3; ++c) {
            const cplx v = U[c * ns + m];
            e += creal(v) * creal(v) + cimag(v) * cimag(v);
        }
        Ek[shell] += mode_weight(iz, N) * e / (2.0 * N3 * N3);
    }
    return 0;
}
