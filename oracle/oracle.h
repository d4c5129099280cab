/*
 * FP64 CPU oracle for the pseudo-spectral Navier-Stokes right-hand side
 * (Mortensen, "Massively parallel implementation in Python of a
 * pseudo-spectral DNS code for turbulent flows", Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It
 * shares no source, header, table or helper with the CUDA library.
 *
 * Layouts (C order, complex = interleaved re, im doubles):
 *   physical  u[3][N][N][N]      index (c, x, y, z), z fastest, x_i = 2*pi*i/N
 *   spectral  uhat[3][N][N][Nh]  index (c, kx, ky, kz), Nh = N/2+1,
 *             kx, ky in FFT order 0..N/2, -N/2+1..-1 (Eq. wavemesh keeps the
 *             Nyquist index N/2 as +N/2), kz = 0..N/2.
 * All functions return 0 on success and a negative value on bad arguments
 * or allocation failure.
 */
#ifndef ORACLE_NS_ORACLE_H
#define ORACLE_NS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Threads OpenMP will use (1 when built without OpenMP). */
int or_num_threads(void);
void or_set_num_threads(int n);

/* 1D complex FFT, unnormalised, in place: X[k] = sum_n x[n] exp(sign*2*pi*i*k*n/n).
 * sign = -1 is the forward transform of Eq. ffteq, +1 the (unscaled) inverse.
 * Any n >= 1 (recursive mixed radix on the smallest prime factor). */
int or_fft1d(int n, double *x, int sign);
/* Brute-force O(n^2) DFT with the same convention (pin for or_fft1d). */
int or_dft1d(int n, const double *x, double *y, int sign);

/* Forward 3D real transform of Eq. ffteq: uhat = F_kx(F_ky(F_kz(u))), unnormalised.
 * u[N][N][N] real -> uhat[N][N][N/2+1] complex. */
int or_rfftn(int N, const double *u, double *uhat);
/* Inverse 3D real transform of Eq. ffteq: u = F^-1_z(F^-1_y(F^-1_x(uhat))) / N^3. */
int or_irfftn(int N, const double *uhat, double *u);
/* Brute-force O(N^6) forward 3D DFT of a real field, half spectrum out (pin). */
int or_dft3_real(int N, const double *u, double *uhat);

/* Nonlinear term (u x omega)^ of Eq. NSfinal before dealiasing and projection:
 * omega^ = i k x uhat; u, omega by the inverse transform; pointwise u x omega;
 * forward transform.  uhat, nhat: [3][N][N][Nh]. */
int or_nonlinear(int N, const double *uhat, double *nhat);
/* Full right-hand side of Eq. NSfinal with 2/3-rule dealiasing of the
 * nonlinear term: du = P(m * (u x omega)^) - nu |k|^2 uhat. */
int or_rhs(int N, double nu, const double *uhat, double *duhat);
/* nsteps classical RK4 steps of Eq. NSfinal, in place on uhat. */
int or_rk4(int N, double nu, double dt, int nsteps, double *uhat);
/* nsteps integrating-factor (Lawson) RK4 steps: exact viscous decay,
 * classical RK4 on the nonlinear term; in place on uhat. */
int or_rk4_if(int N, double nu, double dt, int nsteps, double *uhat);

/* Diagnostics of a spectral field (half-spectrum Parseval weights). */
int or_energy(int N, const double *uhat, double *E);
int or_dissipation(int N, double nu, const double *uhat, double *eps);
int or_spectrum(int N, const double *uhat, double *Ek, int nshells);

/* ---- learned subgrid closure of a coarse LES (oracle_les.c) ---------- */
/* Periodic 3x3x3 cross-correlation y[o] = b[o] + sum_{c,t} w[o][c][t] x[c](p + off(t)),
 * tap t = 9 tx + 3 ty + tz at offset (tx-1, ty-1, tz-1); [C][n][n][n] layouts. */
int or_conv3d_fwd(int n, int cin, int cout, const double *x, const double *w, const double *b, double *y);
/* Gradients of a convolution: dx (optional, overwritten), dw and db (accumulated). */
int or_conv3d_bwd(int n, int cin, int cout, const double *x, const double *w, const double *dy, double *dx,
                  double *dw, double *db);
/* GELU(x) = x (1 + erf(x/sqrt 2))/2 and its derivative (either output optional). */
int or_gelu(long count, const double *x, double *y, double *dydx);
/* 3-layer closure network (9 -> 32 -> 32 -> 6, GELU): output, mean-squared
 * loss against target, and accumulated weight/bias gradients (optional). */
int or_net(int n, const double *g, const double *target, const double *w1, const double *b1, const double *w2,
           const double *b2, const double *w3, const double *b3, double *out, double *loss, double *gw1,
           double *gb1, double *gw2, double *gb2, double *gw3, double *gb3);
/* Sharp-cutoff filter of an N^3 DNS field to an n^3 LES mesh: ubar_hat,
 * gradients g[9][n^3] (g[3i+j] = d_j ubar_i), stresses tau[6][n^3]. */
int or_les_inputs(int N, const double *uhat, int n, double *ubar_hat, double *g, double *tau);
/* LES right-hand side: Eq. NSfinal on ubar plus P(m (-i k_j tau_ij^)). */
int or_rhs_les(int n, double nu, const double *ubar_hat, const double *tau, double *duhat);
/* Smagorinsky stresses tau_ij = -2 (C_s Delta)^2 |S| S_ij from gradients g[9][np]. */
int or_smagorinsky(long np, const double *g, double cs_delta2, double *tau);

#ifdef __cplusplus
}
#endif
#endif
