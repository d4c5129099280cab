/*
 * libdns: single-GPU pseudo-spectral Navier-Stokes solver (GB300, sm_103a).
 *
 * Method: Mortensen, "Massively parallel implementation in Python of a
 * pseudo-spectral DNS code for turbulent flows" (EuroSciPy 2015), Sec. 2:
 * triply periodic box [0, 2 pi]^3 on an N^3 mesh (Eq. realmesh), wavenumbers
 * k in {-N/2+1, ..., N/2}^3 (Eq. wavemesh), transform pair of Eq. ffteq
 * (forward unnormalised, inverse 1/N^3), right-hand side of Eq. NSfinal in
 * rotational form
 *     d uhat/dt = P[ m(k) (u x omega)^ ] - nu |k|^2 uhat,
 *     P = I - k k^T / |k|^2   (pressure eliminated, Eq. pressure),
 * with the 2/3-rule mask m(k) = [3|kx| < N and 3|ky| < N and 3|kz| < N]
 * and the classical fourth-order Runge-Kutta integrator (end of Sec. 2).
 *
 * Conventions shared by every entry point:
 *  - Every function returns an int status (dns_status); nothing throws.
 *  - One handle is used by one host thread at a time.
 *  - The handle owns all device memory it needs; it is allocated by
 *    dns_init and released by dns_free.  Caller buffers are not retained:
 *    the library copies in or out before returning (or, for device buffers,
 *    in stream order on the handle's stream); the one exception is the
 *    asynchronous host I/O, which uses the caller's host buffer until
 *    dns_synchronize returns.
 *  - `on_device` = 1: the pointer is device memory (e.g. a torch CUDA
 *    tensor's data_ptr()); 0: host memory (pinned or pageable).
 *  - Spectral layout ("full"): uhat[3][N][N][N/2+1] complex, C order,
 *    interleaved (re, im); kx and ky in FFT order 0..N/2, -N/2+1..-1, kz =
 *    0..N/2.  Physical layout: u[3][N][N][N] real, z fastest, x_i = 2 pi i/N.
 *  - I/O element type: DNS_F32 -> complex64 / float32;
 *    DNS_F64 and DNS_F32_ACC64 -> complex128 / float64.
 *  - The state lives in the dealiased set: modes with 3|k_i| >= N are not
 *    stored.  Inputs are projected onto that set on entry (such modes are
 *    ignored); outputs carry exact zeros there.  For inputs that are already
 *    dealiased (every field this library produces) this is Eq. NSfinal
 *    exactly, because its right-hand side never leaves the set.
 *  - Inputs must be Hermitian on the kz = 0 plane (real fields); the kz = 0
 *    modes enter the inverse transform through their real part only, as in
 *    the usual inverse real FFT.
 */
#ifndef DNS_H
#define DNS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dns_ctx *dns_handle;

/* Arithmetic of the path.
 * DNS_F32:       every field and transform in float.
 * DNS_F64:       every field and transform in double.
 * DNS_F32_ACC64: transforms and right-hand side in float; the RK4 start and
 *                accumulator states (u0, u1) in double.
 * Diagnostics always accumulate in double. */
enum dns_dtype { DNS_F32 = 0, DNS_F64 = 1, DNS_F32_ACC64 = 2 };

enum dns_status {
    DNS_OK = 0,
    DNS_ERR_ARG = 1,         /* bad pointer, size or value */
    DNS_ERR_OOM = 2,         /* device or host allocation failed */
    DNS_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    DNS_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
    DNS_ERR_NONFINITE = 5,   /* NaN or Inf found in the state */
    DNS_ERR_UNSUPPORTED = 6, /* N, dtype or option not supported */
    DNS_ERR_GUARD = 7,       /* a guard region around a device buffer was overwritten */
    DNS_ERR_INDEX = 8        /* index-checked build: a kernel met an address outside every buffer */
};

/* Create a solver for an N^3 box.  N: one of the compiled mesh sizes 6, 8,
 * 12, 16, 18, 24, 32, 36, 48, 54, 64, 72, 96, 108, 128, 144, 162, 192, 216,
 * 256, 288, 324, 384, 432, 486, 512, 576, 648, 768, 864, 972, 1024, i.e.
 * every even N = 2^a 3^b from 6 to 1024 (transform stages of radix 3 and
 * powers of two); any other N is
 * DNS_ERR_UNSUPPORTED.  nu > 0 viscosity, dt > 0 time step.
 * cuda_stream: a cudaStream_t to run on, or NULL for a stream the handle
 * creates.  The velocity starts at zero, t = 0, step = 0.
 * Errors: DNS_ERR_ARG, DNS_ERR_UNSUPPORTED, DNS_ERR_OOM, DNS_ERR_CUDA. */
int dns_init(int N, double nu, double dt, int dtype, void *cuda_stream, dns_handle *out);

/* Release the handle and its device memory.  NULL is accepted. */
int dns_free(dns_handle h);

/* Set the state from a full spectral field (layout and type above).
 * Synchronous with respect to the host buffer.  Does not change t or step. */
int dns_set_velocity(dns_handle h, const void *uhat, int on_device);

/* Set the state from a physical field u[3][N][N][N] (I/O real type), by the
 * forward transform of Eq. ffteq followed by the dealiasing mask. */
int dns_set_velocity_physical(dns_handle h, const void *u, int on_device);

/* Copy the state out as a full spectral field (zeros outside the dealiased
 * set).  Synchronises the handle's stream. */
int dns_get_velocity(dns_handle h, void *uhat, int on_device);

/* Asynchronous host I/O, for streaming many fields through one handle
 * (set, step, get, set, ...) with the host copies overlapping the steps of
 * the neighbouring fields.  uhat is HOST memory in the full spectral layout
 * above (page-locked memory lets the copies overlap; pageable memory is
 * still correct).  Both calls only queue work and return at once.
 *
 * dns_set_velocity_async: the copy of uhat into an internal staging buffer
 * runs on an internal copy stream as soon as the previous asynchronous set
 * has been converted; the state is replaced (and its curl computed) on the
 * handle's stream, after everything queued there before.  uhat must stay
 * valid and unchanged until dns_synchronize returns.
 *
 * dns_get_velocity_async: the state as it is when the handle's stream
 * reaches this call is converted into one of two staging buffers (taking
 * turns) and copied to uhat on a second copy stream; uhat holds it once
 * dns_synchronize has returned.
 *
 * The first call allocates three staging buffers of the full layout's size
 * (counted by dns_device_bytes); DNS_ERR_OOM if they do not fit, the handle
 * is then unchanged.  dns_synchronize waits for the copy streams too. */
int dns_set_velocity_async(dns_handle h, const void *uhat);
int dns_get_velocity_async(dns_handle h, void *uhat);

/* One evaluation of the right-hand side of Eq. NSfinal on uhat_in (full
 * layout), written to duhat_out (full layout).  Leaves the state unchanged.
 * Synchronises the handle's stream. */
int dns_rhs(dns_handle h, const void *uhat_in, void *duhat_out, int on_device);

/* Advance n >= 0 classical RK4 steps.  Asynchronous: work is queued on the
 * handle's stream (as replays of a CUDA graph of one step, captured on the
 * first call); errors from the device surface at the next synchronising
 * call.  Not to be called while the handle's stream is being captured. */
int dns_step(dns_handle h, int n);

/* Advance n steps with plain kernel launches and CUDA events around every
 * launch, and add the device time of each pass to pass_ms[0..5]:
 * [0] inverse x transform + curl, [1] inverse y transform,
 * [2] z transforms + cross product, [3] forward y transform,
 * [4] forward x transform (dealiased), [5] projection + viscous term + RK4.
 * total_ms receives the device time from the first launch to the last.
 * Synchronises the handle's stream. */
int dns_step_profiled(dns_handle h, int n, double *pass_ms, double *total_ms);

/* Time integrator of dns_step / dns_step_profiled.  The paper allows any
 * integrator and uses a fourth-order Runge-Kutta method (end of Sec. 2).
 * DNS_RK4 (default): classical RK4 on Eq. NSfinal, viscous term explicit.
 * DNS_IFRK4: integrating-factor (Lawson) RK4: classical RK4 applied to
 * exp(nu |k|^2 t) uhat, so the viscous decay exp(-nu |k|^2 dt) is exact
 * and does not limit dt; stages use E1 = exp(-nu|k|^2 dt/2), E2 =
 * exp(-nu|k|^2 dt) and the projected nonlinear term k_s:
 *   u_{n+1} = E2 u_n + dt/6 (E2 k1 + 2 E1 k2 + 2 E1 k3 + k4).
 * DNS_ERR_ARG for other values.  dns_rhs is not affected. */
enum dns_integrator { DNS_RK4 = 0, DNS_IFRK4 = 1 };
int dns_set_integrator(dns_handle h, int kind);

/* Wait for the handle's queued work (its stream and the copy streams of the
 * asynchronous host I/O); reports device errors, and
 * DNS_ERR_TIMEOUT when a kernel gave up one of its bounded waits (a bulk
 * copy into shared memory that did not complete within one second; the
 * state is then not trustworthy and the status stays set). */
int dns_synchronize(dns_handle h);

/* Stray-write check (the paper has no counterpart; a memory checker is not
 * available on every system): every device buffer a handle allocates sits
 * between two 256-byte guard regions filled with a fixed byte pattern.  This
 * call drains the handle's streams, reads every guard region back and
 * returns DNS_ERR_GUARD if any byte changed, i.e. if some kernel wrote past
 * either end of a buffer; DNS_OK otherwise (DNS_ERR_CUDA on a copy error).
 * Synchronising; the buffers themselves are untouched. */
int dns_check_guards(dns_handle h);

/* Check of the failure detection above: queue on the handle's stream a
 * one-block kernel whose bounded wait (on an mbarrier nothing completes)
 * gives up after `seconds` (0 < seconds <= 2, else DNS_ERR_ARG), so that the
 * next dns_synchronize returns DNS_ERR_TIMEOUT.  Leaves the handle's status
 * set, as a real timeout does; the CUDA context stays usable.  For tests of
 * the error path; faults nothing. */
int dns_check_wait_timeout(dns_handle h, double seconds);

/* Index-checked build (no counterpart in the paper; a bounds checker for
 * systems without a memory checker).  The library can also be compiled as
 * libdns_checked.so (-DDNS_CHECKED; the mesh sizes 16, 24, 36, 64, 96, 128,
 * 256, 512 and 1024 only, others return DNS_ERR_UNSUPPORTED), whose solver
 * kernels -- every pass of the right-hand side and of the RK4 update, the
 * layout conversions, curl and diagnostics, and the source of every bulk
 * copy -- compare each global address they are about to use with the
 * handle's buffers (guard regions excluded) and, for the duration of a call
 * given device buffers, the caller's.  An address outside all of them is
 * not accessed (a load reads zero, a store or copy is skipped); the first
 * one is recorded, and dns_synchronize / dns_ensemble_synchronize return
 * DNS_ERR_INDEX from then on.  The learned-closure kernels are not checked.
 *
 * dns_checked_build: 1 in the checked library, 0 otherwise.
 * dns_first_bad_access: after draining the handle's stream, the source
 * line of the check that rejected the first address and that address
 * (0, 0 if none was rejected).
 * dns_check_index_selftest: queues a one-thread kernel that hands the
 * check the address one byte past the end of the handle's largest buffer
 * (compared, never accessed), so that the next dns_synchronize returns
 * DNS_ERR_INDEX; DNS_ERR_UNSUPPORTED in the unchecked library. */
int dns_checked_build(void);
int dns_first_bad_access(dns_handle h, int *line, unsigned long long *address);
int dns_check_index_selftest(dns_handle h);

/* Diagnostics of the current state, accumulated in double (synchronising):
 * E = <|u|^2>/2, eps = nu <|grad u|^2>, and the shell spectrum
 * Ek[s] = sum over modes with floor(|k| + 1/2) = s of |uhat|^2 / (2 N^6)
 * (half-spectrum modes with kz > 0 counted twice).  nshells >= 1; shells
 * beyond nshells-1 are dropped.  A non-finite E or eps returns
 * DNS_ERR_NONFINITE (the value is still written). */
int dns_energy(dns_handle h, double *E);
int dns_dissipation(dns_handle h, double *eps);
int dns_spectrum(dns_handle h, double *Ek, int nshells);

/* Simulated time and step count; dns_set_time restores them on resume. */
int dns_time(dns_handle h, double *t, long *step);
int dns_set_time(dns_handle h, double t, long step);

/* Handle parameters: N, dtype, and the largest kept wavenumber
 * kmax = floor((N-1)/3).  Any output pointer may be NULL. */
int dns_query(dns_handle h, int *N, int *dtype, int *kmax, double *nu, double *dt);

/* Bytes of device memory the handle holds. */
int dns_device_bytes(dns_handle h, long long *bytes);

/* ------------------------------------------------------------------------
 * Autotuner.  Each of the five tuned passes (0: inverse x, 1: inverse y,
 * 2: z transforms + cross product, 3: forward y, 4: forward x) is compiled
 * in a few launch shapes: lines per block, largest radix of the FFT plan
 * and thread count, and with its input either loaded by the threads or
 * landed in shared memory by bulk asynchronous copies.  Pass 4 also has
 * fused variants (numbers from 10 up) that transform along x and apply the
 * projection, viscous term and RK4 stage in the same launch.  A "plan"
 * picks one variant per pass; variant 0 is the default.  Every variant
 * computes the same right-hand side (up to rounding order).
 * ------------------------------------------------------------------------ */

/* Time every compiled variant of every pass on the handle's scratch buffers
 * (the state is not changed), keep the fastest per pass, and write the plan
 * to plan_out[5] (may be NULL).  cache_path (may be NULL): a JSON-lines file
 * keyed by GPU name, N, dtype and box count; a matching entry is applied
 * without timing, and a new result is appended.  Synchronising.  The next
 * dns_step recaptures its graph. */
int dns_autotune(dns_handle h, const char *cache_path, int *plan_out);
int dns_get_plan(dns_handle h, int *plan);
/* DNS_ERR_UNSUPPORTED if a variant is not compiled for this N and dtype. */
int dns_set_plan(dns_handle h, const int *plan);
/* Shape of one variant: lines per block, radix cap, threads per block. */
int dns_variant_info(dns_handle h, int pass, int variant, int *lines, int *max_radix, int *threads);

/* ------------------------------------------------------------------------
 * Batched ensemble: many independent boxes (each its own N, nu and initial
 * field; one dt and dtype) advanced together.  Boxes of one N share every
 * kernel launch (the grid covers all of them), and one RK4 step of every box
 * is a single CUDA graph.  Same layouts, types and conventions as above, per
 * box.  N as in dns_init; nbox >= 1; nu[b] > 0.
 * ------------------------------------------------------------------------ */
typedef struct dns_ens_ctx *dns_ensemble;

int dns_ensemble_init(int nbox, const int *N, const double *nu, double dt, int dtype, void *cuda_stream,
                      dns_ensemble *out);
int dns_ensemble_free(dns_ensemble e);
/* dns_check_guards for every context of an ensemble. */
int dns_ensemble_check_guards(dns_ensemble e);
/* Set / read box b (0 <= b < nbox); synchronising like the single-box calls. */
int dns_ensemble_set_velocity(dns_ensemble e, int box, const void *uhat, int on_device);
int dns_ensemble_get_velocity(dns_ensemble e, int box, void *uhat, int on_device);
/* Advance every box n RK4 steps (asynchronous graph replays). */
int dns_ensemble_step(dns_ensemble e, int n);
/* As dns_synchronize, for every box. */
int dns_ensemble_synchronize(dns_ensemble e);
/* Kinetic energy of every box, E[0..nbox-1] (double accumulation).  Returns
 * DNS_ERR_NONFINITE if any is not finite. */
int dns_ensemble_energy(dns_ensemble e, double *E);
int dns_ensemble_time(dns_ensemble e, double *t, long *step);
/* Autotune every size class of the ensemble (as dns_autotune). */
int dns_ensemble_autotune(dns_ensemble e, const char *cache_path);

/* ------------------------------------------------------------------------
 * Learned subgrid closure for a coarse LES (not in the paper).  The LES
 * solves the filtered equations: Eq. NSfinal on the sharp-cutoff filtered
 * field ubar (|k_i| <= kc = floor((n-1)/3) on an n^3 mesh) plus the term
 * P[ m (-i k_j tau_ij^) ] with tau_ij = filt(u_i u_j) - ubar_i ubar_j.  A
 * network maps the 9 filtered velocity gradients g[3i+j] = d_j ubar_i to the
 * 6 stresses (order xx, yy, zz, xy, xz, yz): three periodic 3x3x3
 * convolutions (cross-correlation; tap t = 9 tx + 3 ty + tz at offset
 * (tx-1, ty-1, tz-1)), 9 -> 32 -> 32 -> 6 channels, GELU between them, BF16
 * weights and activations on the tensor cores with FP32 accumulation, FP32
 * master weights trained by Adam on the mean squared error.
 * Physical fields are channel-major float arrays [C][n][n][n] in device
 * memory.  n: 16, 32, 64, 128 or 256 for the closure and the data builder.
 * One host thread and one stream per object; a network attached to an LES
 * handle must not be trained or evaluated concurrently with its steps.
 * ------------------------------------------------------------------------ */
typedef struct dns_net_ctx *dns_net;
typedef struct dns_les_builder_ctx *dns_les_builder;

/* Network for an n^3 mesh, weights drawn from `seed` (scaled normal, zero
 * biases).  cuda_stream as in dns_init. */
int dns_net_create(int n, unsigned long long seed, void *cuda_stream, dns_net *out);
int dns_net_free(dns_net net);
/* Number of FP32 parameters, in the order w1[32][9][27], b1[32],
 * w2[32][32][27], b2[32], w3[6][32][27], b3[6]. */
long dns_net_param_count(void);
/* Convolution engine of the network's layers (forward and input
 * gradients): DNS_CONV_MMA_SYNC runs warp-level BF16 MMAs with the weights
 * staged in shared memory; DNS_CONV_TCGEN05 runs the
 * fifth-generation tensor cores (accumulators in tensor memory, operands
 * in shared memory, one thread issuing the MMAs of a 128-voxel tile, the
 * shifted activations of each of the 27 taps gathered in turn);
 * DNS_CONV_TCGEN05_SLAB runs them from a shared-memory halo slab of a few
 * z lines, every tap's operand a shifted view of the slab, so all 27 taps'
 * MMAs of a tile issue back to back (persistent blocks, next slab copied
 * while the current one's MMAs run; the default, the fastest of the three
 * at the 64^3 LES mesh).  All compute the same layers (BF16 operands, FP32
 * accumulation).  DNS_ERR_ARG for any other value. */
enum dns_conv_engine { DNS_CONV_MMA_SYNC = 0, DNS_CONV_TCGEN05 = 1, DNS_CONV_TCGEN05_SLAB = 2 };
int dns_net_set_engine(dns_net net, int engine);
int dns_net_get_engine(dns_net net, int *engine);
int dns_net_get_params(dns_net net, float *host, long count);
int dns_net_set_params(dns_net net, const float *host, long count);
/* Scales used only when the network serves as an LES closure: the network
 * sees g * in_scale and the closure uses tau = output * out_scale (the
 * normalisation the training data had).  Defaults 1, 1. */
int dns_net_set_closure_scaling(dns_net net, double in_scale, double out_scale);
/* tau[6][n^3] = network(g[9][n^3]) (device buffers; synchronising). */
int dns_net_forward(dns_net net, const float *g, float *tau);
/* reps forwards of dns_net_forward queued back to back on the network's
 * stream, with CUDA events around each convolution layer and around each
 * forward (no synchronisation between them): layer_ms[0..2] receives the
 * mean device time of layers 1, 2 and 3, total_ms the mean time per forward
 * from the first launch of the first to the last of the last (input
 * conversion and output unpacking included).  Same arguments as
 * dns_net_forward otherwise; 1 <= reps <= 10000, else DNS_ERR_ARG.
 * Synchronising.  No counterpart in the paper (measurement). */
int dns_net_forward_profiled(dns_net net, const float *g, float *tau, int reps, double *layer_ms, double *total_ms);
/* Mean squared error loss of one sample and (optional) its gradient with
 * respect to every parameter, in the parameter order above (host buffer). */
int dns_net_gradients(dns_net net, const float *g, const float *tau, double *loss, float *grad_host, long count);
/* One Adam step (beta 0.9, 0.999, eps 1e-8) on the mean gradient of
 * nsamples consecutive samples g[s][9][n^3], tau[s][6][n^3]; loss = their
 * mean loss before the step. */
int dns_net_train_step(dns_net net, int nsamples, const float *g, const float *tau, double lr, double *loss);

/* Training data from a DNS handle (DNS_F32, mesh N) for an n^3 LES:
 * g[9][n^3] and tau[6][n^3] at the LES grid points, and (optional) the
 * filtered field on the n mesh in the full spectral layout (complex64). */
int dns_les_builder_create(int N, int n, dns_les_builder *out);
int dns_les_builder_free(dns_les_builder b);
int dns_les_builder_run(dns_les_builder b, dns_handle dns, float *g, float *tau, void *ubar_hat);

/* Attach a network as the subgrid closure of an LES handle (DNS_F32, N =
 * the network's n), or detach it with net = NULL.  With a closure attached,
 * dns_step and dns_rhs add the closure term, evaluated from each stage's
 * input.  The handle does not own the network. */
int dns_les_set_closure(dns_handle h, dns_net net);
/* Attach the Smagorinsky eddy-viscosity closure instead (the classic
 * non-learned comparator; not in the paper): tau_ij = -2 (cs delta)^2 |S| S_ij
 * from the stage input's resolved strain S_ij, |S| = sqrt(2 S_ij S_ij);
 * delta <= 0 selects the mesh spacing 2 pi / N.  Detach with
 * dns_les_set_closure(h, NULL).  Same handle restrictions as above;
 * DNS_ERR_ARG for cs < 0 or non-finite arguments. */
int dns_les_set_smagorinsky(dns_handle h, double cs, double delta);
/* When the closure term of an attached closure is evaluated: every_stage = 1
 * (default) from each RK4 stage's input; 0 from the first stage's input (the
 * state at the start of the step) only, the same term then held through the
 * step's four stages (one network evaluation per step instead of four; the
 * closure term becomes first-order accurate in time, the resolved dynamics
 * stay RK4).  Takes effect at the next dns_step (the step graph is
 * re-captured); dns_rhs always evaluates it from its input.  DNS_ERR_ARG for
 * other values. */
int dns_les_set_closure_stages(dns_handle h, int every_stage);

/* ------------------------------------------------------------------------
 * Diagnostics without allocation.  The paper has no counterpart: this is a
 * service for callers that cannot call cudaMalloc where they need the
 * numbers, such as callbacks and real-time loops that must stay out of the
 * allocator (a device allocation can synchronise the device or block), or
 * processes whose device memory belongs to another framework's pool or
 * budget, so that memory obtained behind that framework's back could push it
 * out of memory.
 *
 * Kinetic energy out[0] = <|u|^2>/2 and dissipation out[1] = nu <|grad u|^2>
 * of a full-layout spectral field uhat on the device (mesh N, I/O type of
 * `dtype`), with the weights of dns_energy; no handle is needed.  Scratch
 * lives in a file-scope device array of 2*1024+2 doubles (16 KB on every
 * device that loads the library, held until the process exits), so N must be
 * even and at most 1024 (else DNS_ERR_UNSUPPORTED; odd N is DNS_ERR_ARG).
 * The first call on a device looks up that array's device address and should
 * come before any stream capture; later calls only launch two kernels (plus
 * a 16-byte copy for a host output).  All calls on a device share the array:
 * calls that overlap on the GPU race and must be serialised by the caller.
 * out_on_device = 1: out is device memory and the call is asynchronous on
 * cuda_stream; 0: out is host memory and the call synchronises cuda_stream
 * (DNS_ERR_NONFINITE if a result is not finite).  cuda_stream may be NULL.
 * ------------------------------------------------------------------------ */
int dns_energy_noalloc(int N, int dtype, const void *uhat, double nu, double *out, int out_on_device,
                       void *cuda_stream);

/* ------------------------------------------------------------------------
 * Measurement utility (the paper has no counterpart): the FP64 arithmetic
 * peak of the current device, as the denominator of the FP64 path's
 * roofline.  Runs a kernel of independent FP64 fused multiply-adds over
 * every SM for about `seconds` (0 < seconds <= 10, else DNS_ERR_ARG) on the
 * default stream, synchronises, and writes the achieved rate in TFLOP/s (two
 * flops per FMA) to *tflops (host memory).  Allocates nothing; DNS_ERR_CUDA
 * on a launch or event error.
 * ------------------------------------------------------------------------ */
int dns_fp64_fma_rate(double seconds, double *tflops);

/* Human-readable name of a status code (static storage). */
const char *dns_strerror(int status);

/* Text of the last CUDA runtime error this thread saw inside the library
 * (static storage; "no error" if none). */
const char *dns_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif
