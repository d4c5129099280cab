/*
 * FP64 CPU oracle for the learned subgrid closure of a coarse LES built on
 * the pseudo-spectral solver (not in the paper; the configuration is a
 * 64^3 LES fed by box-filtered DNS).  TEST INFRASTRUCTURE ONLY, like
 * oracle.c, whose transforms and right-hand side it calls.
 *
 * Filtered equations: with the sharp spectral filter (keep |k_i| <= kc of
 * the DNS field, kc = floor((n-1)/3) for an n^3 LES mesh) and
 * tau_ij = filt(u_i u_j) - ubar_i ubar_j, the filtered field obeys Eq.
 * NSfinal plus the term -i k_j tau_ij^, projected and dealiased like the
 * nonlinear term.
 *
 * Network: three periodic 3x3x3 convolutions (cross-correlation, tap
 * t = 9 tx + 3 ty + tz at offset (tx-1, ty-1, tz-1)) with GELU between them,
 * 9 gradient channels g[3i+j] = d_j ubar_i in, 6 stress channels
 * (xx, yy, zz, xy, xz, yz) out; loss = mean of squared errors.
 *
 * Layouts: channel-major [C][n][n][n] (z fastest); weights [Cout][Cin][27].
 *
 * OR_MUTANT 8..13 plant one deliberate mistake each in this file (see
 * oracle.c); the LES pins must reject every one.
 */
#include "oracle.h"

#ifndef OR_MUTANT
#define OR_MUTANT 0
#endif

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static int wn(int i, int N) { return (i <= N / 2) ? i : i - N; }

static long vox(int n, int x, int y, int z) {
    x = (x % n + n) % n;
    y = (y % n + n) % n;
    z = (z % n + n) % n;
    return ((long)x * n + y) * n + z;
}

int or_conv3d_fwd(int n, int cin, int cout, const double *x, const double *w, const double *b, double *y) {
    if (n < 1 || cin < 1 || cout < 1 || !x || !w || !y) return -1;
    const long V = (long)n * n * n;
#pragma omp parallel for collapse(2) schedule(static)
    for (int o = 0; o < cout; ++o)
        for (int px = 0; px < n; ++px)
            for (int py = 0; py < n; ++py)
                for (int pz = 0; pz < n; ++pz) {
                    double s = b ? b[o] : 0.0;
                    for (int c = 0; c < cin; ++c)
                        for (int t = 0; t < 27; ++t) {
#if OR_MUTANT == 8 /* planted: convolution (flipped taps) instead of cross-correlation */
                            const int tx = 1 - t / 9, ty = 1 - (t / 3) % 3, tz = 1 - t % 3;
#else
                            const int tx = t / 9 - 1, ty = (t / 3) % 3 - 1, tz = t % 3 - 1;
#endif
                            s += w[((long)o * cin + c) * 27 + t] * x[c * V + vox(n, px + tx, py + ty, pz + tz)];
                        }
                    y[o * V + vox(n, px, py, pz)] = s;
                }
    return 0;
}

/* Given dL/dy: dL/dx (if dx), dL/dw, dL/db (accumulated: the caller zeroes). */
int or_conv3d_bwd(int n, int cin, int cout, const double *x, const double *w, const double *dy, double *dx,
                  double *dw, double *db) {
    if (n < 1 || cin < 1 || cout < 1 || !x || !w || !dy || !dw || !db) return -1;
    const long V = (long)n * n * n;
    if (dx) {
#pragma omp parallel for collapse(2) schedule(static)
        for (int c = 0; c < cin; ++c)
            for (int px = 0; px < n; ++px)
                for (int py = 0; py < n; ++py)
                    for (int pz = 0; pz < n; ++pz) {
                        /* y[o][q] uses x[c][q + off]: x at p feeds q = p - off */
                        double s = 0.0;
                        for (int o = 0; o < cout; ++o)
                            for (int t = 0; t < 27; ++t) {
                                const int tx = t / 9 - 1, ty = (t / 3) % 3 - 1, tz = t % 3 - 1;
                                s += w[((long)o * cin + c) * 27 + t] * dy[o * V + vox(n, px - tx, py - ty, pz - tz)];
                            }
                        dx[c * V + vox(n, px, py, pz)] = s;
                    }
    }
#pragma omp parallel for collapse(2) schedule(static)
    for (int o = 0; o < cout; ++o)
        for (int c = 0; c < cin; ++c)
            for (int t = 0; t < 27; ++t) {
                const int tx = t / 9 - 1, ty = (t / 3) % 3 - 1, tz = t % 3 - 1;
                double s = 0.0;
                for (int px = 0; px < n; ++px)
                    for (int py = 0; py < n; ++py)
                        for (int pz = 0; pz < n; ++pz)
                            s += dy[o * V + vox(n, px, py, pz)] * x[c * V + vox(n, px + tx, py + ty, pz + tz)];
                dw[((long)o * cin + c) * 27 + t] += s;
            }
    for (int o = 0; o < cout; ++o) {
        double s = 0.0;
        for (long p = 0; p < V; ++p) s += dy[o * V + p];
        db[o] += s;
    }
    return 0;
}

/* GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2 and its derivative
 * Phi(x) + x phi(x), phi(x) = exp(-x^2/2) / sqrt(2 pi). */
static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
static double gelu_d(double x) {
#if OR_MUTANT == 9 /* planted: the x phi(x) term of the derivative dropped */
    return 0.5 * (1.0 + erf(x / sqrt(2.0)));
#else
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
#endif
}

int or_gelu(long count, const double *x, double *y, double *dydx) {
    if (count < 0 || !x) return -1;
    for (long i = 0; i < count; ++i) {
        if (y) y[i] = gelu(x[i]);
        if (dydx) dydx[i] = gelu_d(x[i]);
    }
    return 0;
}

/* Forward and backward of the closure network on one sample.
 * w1 [32][9][27], w2 [32][32][27], w3 [6][32][27]; b1 [32], b2 [32], b3 [6].
 * out (optional) [6][V]; loss = mean over 6 V of (out - target)^2; the
 * gradients (optional, accumulated) have the shapes of the weights. */
int or_net(int n, const double *g, const double *target, const double *w1, const double *b1, const double *w2,
           const double *b2, const double *w3, const double *b3, double *out, double *loss, double *gw1,
           double *gb1, double *gw2, double *gb2, double *gw3, double *gb3) {
    if (n < 1 || !g || !w1 || !b1 || !w2 || !b2 || !w3 || !b3) return -1;
    const long V = (long)n * n * n;
    double *z1 = malloc(sizeof(double) * 32 * V), *a1 = malloc(sizeof(double) * 32 * V);
    double *z2 = malloc(sizeof(double) * 32 * V), *a2 = malloc(sizeof(double) * 32 * V);
    double *y = malloc(sizeof(double) * 6 * V);
    int rc = (!z1 || !a1 || !z2 || !a2 || !y) ? -2 : 0;
    if (!rc) rc = or_conv3d_fwd(n, 9, 32, g, w1, b1, z1);
    if (!rc) rc = or_gelu(32 * V, z1, a1, NULL);
    if (!rc) rc = or_conv3d_fwd(n, 32, 32, a1, w2, b2, z2);
    if (!rc) rc = or_gelu(32 * V, z2, a2, NULL);
    if (!rc) rc = or_conv3d_fwd(n, 32, 6, a2, w3, b3, y);
    if (!rc && out) memcpy(out, y, sizeof(double) * 6 * V);
    if (!rc && target && loss) {
        double s = 0.0;
        for (long i = 0; i < 6 * V; ++i) s += (y[i] - target[i]) * (y[i] - target[i]);
        *loss = s / (6.0 * V);
    }
    if (!rc && target && gw1 && gb1 && gw2 && gb2 && gw3 && gb3) {
        double *dy = malloc(sizeof(double) * 6 * V), *d2 = malloc(sizeof(double) * 32 * V);
        double *d1 = malloc(sizeof(double) * 32 * V);
        rc = (!dy || !d2 || !d1) ? -2 : 0;
        if (!rc) {
            for (long i = 0; i < 6 * V; ++i) dy[i] = 2.0 * (y[i] - target[i]) / (6.0 * V);
            rc = or_conv3d_bwd(n, 32, 6, a2, w3, dy, d2, gw3, gb3);           /* d2 = dL/da2 */
            for (long i = 0; !rc && i < 32 * V; ++i) d2[i] *= gelu_d(z2[i]);  /* dL/dz2 */
            if (!rc) rc = or_conv3d_bwd(n, 32, 32, a1, w2, d2, d1, gw2, gb2);
            for (long i = 0; !rc && i < 32 * V; ++i) d1[i] *= gelu_d(z1[i]);  /* dL/dz1 */
            if (!rc) rc = or_conv3d_bwd(n, 9, 32, g, w1, d1, NULL, gw1, gb1);
        }
        free(dy);
        free(d2);
        free(d1);
    }
    free(z1);
    free(a1);
    free(z2);
    free(a2);
    free(y);
    return rc;
}

/* Filtered inputs and subgrid stresses of an N^3 DNS field (full layout) on
 * an n^3 LES mesh: ubar_hat (full layout, n), g[9][n^3] = d_j ubar_i and
 * tau[6][n^3] = filt(u_i u_j) - ubar_i ubar_j at the LES grid points. */
int or_les_inputs(int N, const double *uhat, int n, double *ubar_hat, double *g, double *tau) {
    if (N < 2 || n < 2 || n > N || (N & 1) || (n & 1) || !uhat || !ubar_hat || !g || !tau) return -1;
    const int Nh = N / 2 + 1, nh = n / 2 + 1, kc = (n - 1) / 3;
    const long NS = (long)N * N * Nh, ns = (long)n * n * nh, NP = (long)N * N * N, np = (long)n * n * n;
    const double scale = ((double)n * n * n) / ((double)N * N * N);
    const cplx *U = (const cplx *)uhat;
    cplx *Ub = (cplx *)ubar_hat;
    int rc = 0;
    /* sharp cutoff |k_i| <= kc, moved to the n^3 mesh */
    memset(Ub, 0, sizeof(cplx) * 3 * (size_t)ns);
    for (int c = 0; c < 3; ++c)
        for (int ix = 0; ix < n; ++ix)
            for (int iy = 0; iy < n; ++iy)
                for (int iz = 0; iz < nh; ++iz) {
                    const int kx = wn(ix, n), ky = wn(iy, n), kz = iz;
                    if (abs(kx) > kc || abs(ky) > kc || kz > kc) continue;
                    const long src = ((long)((kx + N) % N) * N + (ky + N) % N) * Nh + kz;
                    Ub[c * ns + ((long)ix * n + iy) * nh + iz] = scale * U[c * NS + src];
                }
    /* gradients d_j ubar_i = F^-1(i k_j ubar_i^) */
    cplx *tmp = malloc(sizeof(cplx) * (size_t)ns);
    double *ub = malloc(sizeof(double) * 3 * (size_t)np);
    double *u = malloc(sizeof(double) * 3 * (size_t)NP);
    double *prod = malloc(sizeof(double) * (size_t)NP);
    cplx *ph = malloc(sizeof(cplx) * (size_t)NS);
    cplx *pb = malloc(sizeof(cplx) * (size_t)ns);
    double *pf = malloc(sizeof(double) * (size_t)np);
    if (!tmp || !ub || !u || !prod || !ph || !pb || !pf) rc = -2;
    for (int i = 0; i < 3 && !rc; ++i) {
        rc = or_irfftn(n, (const double *)(Ub + i * ns), ub + i * np);
        for (int j = 0; j < 3 && !rc; ++j) {
            for (int ix = 0; ix < n; ++ix)
                for (int iy = 0; iy < n; ++iy)
                    for (int iz = 0; iz < nh; ++iz) {
                        const int k[3] = {wn(ix, n), wn(iy, n), iz};
                        const long m = ((long)ix * n + iy) * nh + iz;
#if OR_MUTANT == 13 /* planted: transposed gradient, g[3i+j] = d_i u_j */
                        tmp[m] = I * (double)k[i] * Ub[j * ns + m];
#else
                        tmp[m] = I * (double)k[j] * Ub[i * ns + m];
#endif
                    }
            rc = or_irfftn(n, (const double *)tmp, g + (3 * i + j) * np);
        }
    }
    /* tau_ij = filt(u_i u_j) - ubar_i ubar_j */
    for (int c = 0; c < 3 && !rc; ++c) rc = or_irfftn(N, (const double *)(U + c * NS), u + c * NP);
    const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < 6 && !rc; ++q) {
        for (long p = 0; p < NP; ++p) prod[p] = u[pi[q] * NP + p] * u[pj[q] * NP + p];
        rc = or_rfftn(N, prod, (double *)ph);
        if (rc) break;
        memset(pb, 0, sizeof(cplx) * (size_t)ns);
        for (int ix = 0; ix < n; ++ix)
            for (int iy = 0; iy < n; ++iy)
                for (int iz = 0; iz < nh; ++iz) {
                    const int kx = wn(ix, n), ky = wn(iy, n), kz = iz;
                    if (abs(kx) > kc || abs(ky) > kc || kz > kc) continue;
                    pb[((long)ix * n + iy) * nh + iz] = scale * ph[((long)((kx + N) % N) * N + (ky + N) % N) * Nh + kz];
                }
        rc = or_irfftn(n, (const double *)pb, pf);
#if OR_MUTANT == 10 /* planted: tau = filt(u_i u_j) + ubar_i ubar_j */
        for (long p = 0; !rc && p < np; ++p) tau[q * np + p] = pf[p] + ub[pi[q] * np + p] * ub[pj[q] * np + p];
#else
        for (long p = 0; !rc && p < np; ++p) tau[q * np + p] = pf[p] - ub[pi[q] * np + p] * ub[pj[q] * np + p];
#endif
    }
    free(tmp);
    free(ub);
    free(u);
    free(prod);
    free(ph);
    free(pb);
    free(pf);
    return rc;
}

/* LES right-hand side: Eq. NSfinal on ubar plus P(m (-i k_j tau_ij^)),
 * tau given at the n^3 grid points (6 channels, order xx yy zz xy xz yz). */
int or_rhs_les(int n, double nu, const double *ubar_hat, const double *tau, double *duhat) {
    if (n < 2 || (n & 1) || !ubar_hat || !tau || !duhat) return -1;
    const int nh = n / 2 + 1;
    const long ns = (long)n * n * nh, np = (long)n * n * n;
    int rc = or_rhs(n, nu, ubar_hat, duhat);
    cplx *th = malloc(sizeof(cplx) * 6 * (size_t)ns);
    if (!th) rc = -2;
    for (int q = 0; q < 6 && !rc; ++q) rc = or_rfftn(n, tau + q * np, (double *)(th + q * ns));
    if (!rc) {
        cplx *D = (cplx *)duhat;
        /* component (i, j) of the symmetric tensor */
        const int idx[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
        for (int ix = 0; ix < n; ++ix)
            for (int iy = 0; iy < n; ++iy)
                for (int iz = 0; iz < nh; ++iz) {
                    const int k[3] = {wn(ix, n), wn(iy, n), iz};
                    if (!(3 * abs(k[0]) < n && 3 * abs(k[1]) < n && 3 * abs(k[2]) < n)) continue;
                    const long m = ((long)ix * n + iy) * nh + iz;
                    cplx f[3];
                    for (int i = 0; i < 3; ++i) {
                        f[i] = 0.0;
#if OR_MUTANT == 11 /* planted: closure term +i k_j tau_ij instead of -i k_j tau_ij */
                        for (int j = 0; j < 3; ++j) f[i] += I * (double)k[j] * th[idx[i][j] * ns + m];
#else
                        for (int j = 0; j < 3; ++j) f[i] += -I * (double)k[j] * th[idx[i][j] * ns + m];
#endif
                    }
                    const double k2 = (double)k[0] * k[0] + (double)k[1] * k[1] + (double)k[2] * k[2];
                    const cplx kf = k[0] * f[0] + k[1] * f[1] + k[2] * f[2];
                    for (int i = 0; i < 3; ++i) D[i * ns + m] += f[i] - (k2 > 0 ? k[i] * kf / k2 : 0.0);
                }
    }
    free(th);
    return rc;
}

/* Smagorinsky eddy-viscosity closure (the classic non-learned comparator;
 * not in the paper): with S_ij = (d_j u_i + d_i u_j)/2 and
 * |S| = sqrt(2 S_ij S_ij), tau_ij = -2 (C_s Delta)^2 |S| S_ij, computed
 * pointwise from the gradients g[3i+j] = d_j u_i of the LES field. */
int or_smagorinsky(long np, const double *g, double cs_delta2, double *tau) {
    if (np < 1 || !g || !tau) return -1;
    const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
    for (long p = 0; p < np; ++p) {
        double S[3][3], ss = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) S[i][j] = 0.5 * (g[(3 * i + j) * np + p] + g[(3 * j + i) * np + p]);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) ss += S[i][j] * S[i][j];
        const double mag = sqrt(2.0 * ss);
#if OR_MUTANT == 12 /* planted: the factor 2 of the eddy-viscosity stress dropped */
        for (int q = 0; q < 6; ++q) tau[q * np + p] = -cs_delta2 * mag * S[pi[q]][pj[q]];
#else
        for (int q = 0; q < 6; ++q) tau[q * np + p] = -2.0 * cs_delta2 * mag * S[pi[q]][pj[q]];
#endif
    }
    return 0;
}
