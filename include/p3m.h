/*
 * p3m.h -- C ABI of the GB300 (sm_103a) P3M gravity step.
 *
 * The library evaluates the P3M force of the CONCEPT code (arXiv:1510.07621, the CONCEPT
 * user's guide): particle-mesh long-range force plus a short-range particle-particle sum
 * inside a cutoff, split at a Gaussian scale (Ch. Parameters, "Numerical parameters":
 * PM_gridsize, PM_scale, P3M_cutoff, softeningfactors; "Simulation options": kick_algorithms
 * 'PM' / 'P3M'), and advances comoving particles with a kick-drift-kick leapfrog over the
 * scale factor (Ch. Parameters, "Cosmological parameters"; Ch. Snapshot Formats: comoving
 * positions posx..posz and momenta momx..momz).  The guide prints no formulas; the
 * arithmetic below is the textbook P3M method:
 *
 *   mesh:   CIC counts n(node), nodes at i*h, h = box/mesh
 *           G(k) = -4 pi G m / h^3 * exp(-k^2 r_s^2) / k^2 / W(k)^2,  W = prod sinc^2(k_d h/2)
 *           a_mesh,d = IFFT(-i k_d G(k) FFT(n - N/mesh^3)),  k_d = 0 on the Nyquist plane of d
 *           a_LR(particle) = CIC interpolation of a_mesh
 *   pairs:  a_SR,i = sum_{0 < |d_ij| < r_c} G m g(r/r_s) d_ij / (r^2 + eps^2)^(3/2),
 *           g(x) = erfc(x/2) + x/sqrt(pi) exp(-x^2/4), d_ij the minimum-image separation
 *   units:  time 1/H0 (H0 = 1), lengths as given (Mpc/h), G m = 3 Omega_m box^3 / (8 pi N)
 *   motion: p = m a^2 dx/dt;  kick p += m a_grav int dt/a;  drift x += p/m int dt/a^2;
 *           positions wrapped into [0, box)
 *
 * Conventions shared by every entry point
 *   - Every function returns P3M_OK (0) or a negative P3M_E* code; nothing throws across the
 *     ABI.  After a failure p3m_last_error(ctx) holds a one-line message (for p3m_init, the
 *     message is available through p3m_last_error(NULL)).
 *   - Particle arrays are structure of arrays [3][n] of doubles: all x, then all y, then all
 *     z.  Caller arrays are borrowed for the duration of the call only.
 *   - on_device != 0: the pointers are CUDA device pointers on the current device; the call
 *     returns with the work queued on the context's stream (host arrays: the call returns
 *     after the copies completed).  Page-locked (pinned) host arrays are read and written in
 *     place by the kernels over the CPU-GPU link; other host arrays are staged through copies.
 *   - The context owns all device memory, cuFFT plans and events; p3m_free releases them.
 *   - Particle order: the library keeps particles sorted by chaining cell internally; every
 *     array a caller reads back is in the caller's original order (the order of
 *     p3m_set_particles), except the sorted views of p3m_get_cells.
 *   - Not thread-safe: one host thread at a time per context.
 */
#ifndef P3M_H
#define P3M_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define P3M_OK 0
#define P3M_EINVAL (-1)     /* an argument is out of range; nothing was launched        */
#define P3M_ENOMEM (-2)     /* a device allocation failed                               */
#define P3M_ECUDA (-3)      /* a CUDA runtime call failed                               */
#define P3M_ECUFFT (-4)     /* a cuFFT call failed                                      */
#define P3M_ESTATE (-5)     /* call out of order (e.g. a step before any particles)     */
#define P3M_ETIMEOUT (-6)   /* a bounded device-side wait gave up (error flag was set)  */
#define P3M_ENONFINITE (-7) /* NaN or Inf in the particle input                         */
#define P3M_EBOUNDS (-8)    /* debug builds: a kernel's bounds check failed, or the guard
                               bytes after an allocation were overwritten                  */

/* precision modes */
#define P3M_PREC_MIXED 0 /* FP32 mesh, FFTs and pair forces; FP64 positions, momenta and
                            per-particle accumulators                                      */
#define P3M_PREC_FP64 1  /* every step in FP64 (the all-FP64 comparison mode)              */

typedef struct p3m_ctx p3m_ctx;

/* Cosmological parameters (Ch. Parameters, "Cosmological parameters": H0, Omega_m,
 * Omega_Lambda).  Curvature is 1 - omega_m - omega_lambda.  h0 only records the Hubble
 * constant the caller's units refer to: internally time is measured in 1/H0. */
typedef struct {
    double omega_m;
    double omega_lambda;
    double h0;
} p3m_cosmology;

typedef struct {
    int precision;      /* P3M_PREC_MIXED (default) or P3M_PREC_FP64                          */
    double softening;   /* Plummer radius in units of the mean spacing box/N^(1/3)
                           (Ch. Parameters, "softeningfactors"); default 0.02              */
    int deconvolve_cic; /* 1 (default): divide G(k) by W(k)^2                              */
    int short_range;    /* 1 (default): P3M; 0: pure PM ('PM' kick algorithm: no Gaussian
                           filter, no pair sum)                                             */
    int sub_bits;       /* b in 0..5: each chaining cell is split 2^b per side in the sort key
                           (Hilbert-curve order inside the cell); -1 = default (3).  The key
                           (n_c^3 << 3b) must fit in 32 bits                               */
    void *stream;       /* cudaStream_t for all work of the context; NULL = legacy stream  */
} p3m_options;

/* Diagnostics of the current state (p3m_diagnostics). */
typedef struct {
    double momentum[3];   /* sum_i p_i (FP64, fixed reduction order)                       */
    double kinetic;       /* sum_i |p_i|^2 / (2 m a^2)                                      */
    double potential;     /* W = (1/(2a)) sum_i m Phi_i while energy tracking is on
                             (p3m_track_energy), else NaN                                   */
    double layzer_irvine; /* while tracking: a(K + W) + int_{a0}^{a} K da - a0 (K0 + W0),
                             the Layzer-Irvine residual (0 for exact dynamics), else NaN   */
    double a;             /* scale factor of the state                                      */
    uint64_t pairs;       /* ordered pairs inside r_c in the last force evaluation          */
    uint64_t pairs_total; /* the same, summed over every force evaluation of the context   */
    uint64_t launches;    /* kernels this library launched on the stream since p3m_init
                             (cuFFT's own kernels not included)                             */
    uint64_t pair_warp_j[3]; /* pair kernel work since p3m_init, in warp-iterations over one
                             j particle (32 pair slots each): [0] in chunks entirely inside
                             r_c of every i of the warp, [1] in chunks tested pair by pair,
                             [2] tested ones that some i accepted                          */
    uint64_t pair_blocks_culled; /* 32-particle j blocks skipped by the bounding-box test     */
    uint64_t pair_tiles[2];  /* j tiles streamed through shared memory; [1] of them entirely
                                culled                                                       */
    int64_t n;            /* number of particles                                            */
    int32_t n_cells_side; /* chaining cells per side n_c                                    */
    int32_t max_cell_count; /* most particles in one chaining cell (last sort)              */
} p3m_diag;

/* Fills *opt with the defaults listed above.  Returns P3M_EINVAL for NULL. */
int p3m_default_options(p3m_options *opt);

/*
 * Creates a context for n particles in a periodic box.
 *   box            side of the comoving box (Ch. Parameters, "boxsize"), > 0
 *   n              number of particles, 1 <= n < 2^31
 *   mesh           PM_gridsize M: even, 8 <= M <= 2048
 *   r_s_cells      PM_scale: split scale r_s in mesh cells (> 0)
 *   cutoff_in_rs   P3M_cutoff: r_c = cutoff_in_rs * r_s (> 0); with short_range the box must
 *                  hold n_c = floor(box / r_c) >= 3 chaining cells per side
 *   cosmo, opt     may be NULL (Einstein-de Sitter; p3m_default_options)
 * Allocates every device buffer and plan up front (no allocation happens in later calls).
 * Errors: P3M_EINVAL (arguments), P3M_ENOMEM, P3M_ECUFFT, P3M_ECUDA; *ctx is NULL then.
 */
int p3m_init(p3m_ctx **ctx, double box, int64_t n, int mesh, double r_s_cells,
             double cutoff_in_rs, const p3m_cosmology *cosmo, const p3m_options *opt);

/*
 * Loads particles: pos3n and mom3n [3][n] (comoving positions; momenta m a^2 dx/dt), a
 * common particle mass, and the scale factor a of the state.  Positions outside [0, box)
 * are wrapped.  acc3n (nullable) supplies the accelerations at these positions (as returned
 * by p3m_get_particles) so that the next p3m_step needs no extra force evaluation; without
 * it the first p3m_step evaluates the forces at a first.
 * Errors: P3M_EINVAL (NULL pointers, mass <= 0, a <= 0), P3M_ENONFINITE (NaN/Inf anywhere in
 * the input; the state is then unusable until the next successful call), P3M_ECUDA.
 * Synchronises the stream.
 */
int p3m_set_particles(p3m_ctx *ctx, const double *pos3n, const double *mom3n,
                      const double *acc3n, double mass, double a, int on_device);

/*
 * Evaluates the accelerations (long + short range) at the current positions: sort, mesh
 * force, pair force.  acc3n (nullable) receives them [3][n] in the caller's order.
 * Errors: P3M_ESTATE (no particles), P3M_ECUDA, P3M_ECUFFT.
 */
int p3m_forces(p3m_ctx *ctx, double a, double *acc3n, int on_device);

/*
 * The same evaluation with the two parts returned separately (nullable each): acc_lr3n the
 * mesh part, acc_sr3n the pair part.  Leaves the context's forces valid (their sum).
 */
int p3m_forces_split(p3m_ctx *ctx, double *acc_lr3n, double *acc_sr3n, int on_device);

/*
 * One kick-drift-kick step a -> a + da: half kick with the forces at a, drift, force
 * evaluation at the new positions, half kick with them.  Queued on the stream without any
 * host synchronisation (graph-capturable once forces are valid).
 * Errors: P3M_EINVAL (a <= 0, da <= 0), P3M_ESTATE (no particles), P3M_ECUDA, P3M_ECUFFT.
 */
int p3m_step(p3m_ctx *ctx, double a, double da);

/*
 * Copies the state back in the caller's original particle order: pos3n, mom3n, acc3n
 * (each nullable).  Host arrays: synchronises.  Returns P3M_ETIMEOUT if a device-side wait
 * of an earlier call gave up.
 */
int p3m_get_particles(p3m_ctx *ctx, double *pos3n, double *mom3n, double *acc3n,
                      int on_device);

/*
 * Power spectrum of the current particle distribution on the PM mesh (Ch. Parameters:
 * PM_gridsize is also the power-spectrum grid, R_tophat the radius of the top-hat sphere for
 * sigma; Ch. Tests: powerspec).  delta = n/n_bar - 1 on the CIC count mesh, delta_k its DFT
 * divided by M^3; shell b (0 <= b < n_bins <= M/2) holds the modes with round(|k|/k_f) = b+1,
 * k_f = 2 pi / box:
 *   k_mean[b]  mean |k| of the shell's modes     power[b]  box^3 <|delta_k|^2 / W(k)^2>
 *   n_modes[b] number of modes (both halves of the spectrum)
 * W(k)^2 = prod_d sinc^4(k_d h/2) when deconvolve != 0, else 1; shot noise is not subtracted.
 * sigma (nullable): with tophat_radius R > 0, sigma_R = sqrt(sum_{k != 0} |delta_k|^2 / W^2
 * W_TH(k R)^2), W_TH(x) = 3 (sin x - x cos x) / x^3.  Output arrays are host arrays (each
 * nullable); synchronises.  Overwrites the density mesh of p3m_get_mesh(0) with the current
 * positions.  Errors: P3M_EINVAL, P3M_ESTATE, P3M_ECUDA, P3M_ECUFFT.
 */
int p3m_power_spectrum(p3m_ctx *ctx, int n_bins, int deconvolve, double tophat_radius,
                       double *k_mean, double *power, double *n_modes, double *sigma);

/*
 * Graph-captured stepping.  p3m_run_steps advances the context through n_steps kick-drift-kick
 * steps a_list[0] -> a_list[1] -> ... -> a_list[n_steps] (increasing; n_steps <= 4096 per
 * call).  use_graph = 0 issues every kernel from the host (p3m_step in a loop); use_graph = 1
 * captures one step into a CUDA graph per step parity on first use (the buffers the step swaps
 * return to their roles after two steps) and replays it, the step's kick and drift factors
 * read from a device table filled once per call.  Graph mode needs a non-default stream
 * (p3m_options.stream or p3m_set_stream).  The graphs are recaptured when the context's
 * geometry (p3m_autotune) or buffer roles (an intervening p3m_step) no longer match them.
 */
int p3m_run_steps(p3m_ctx *ctx, const double *a_list, int n_steps, int use_graph);

/* Moves the context to another stream (cudaStream_t; NULL = legacy stream); waits for the
 * work already queued on the old one. */
int p3m_set_stream(p3m_ctx *ctx, void *stream);

/*
 * Ensembles of independent simulations of any sizes (many small boxes stepped together): the
 * contexts advance together through the same schedule of scale factors.  With use_graph = 1
 * one step of every context is captured as parallel branches of a single CUDA graph (one per
 * step parity), so each step of the whole ensemble is one graph launch; with use_graph = 0
 * the host issues every kernel of every context, context after context.  own_streams != 0
 * gives each context a stream of its own (p3m_ensemble_free returns them to the legacy
 * stream).  The ensemble borrows the contexts; free it before them.  Errors are reported
 * through p3m_last_error(NULL).
 */
typedef struct p3m_ensemble p3m_ensemble;
int p3m_ensemble_create(p3m_ensemble **ens, p3m_ctx *const *ctxs, int n_ctx, int own_streams);
int p3m_ensemble_run(p3m_ensemble *ens, const double *a_list, int n_steps, int use_graph);
void p3m_ensemble_free(p3m_ensemble *ens);
/*
 * Batched pair launch (off by default; enable != 0 turns it on when at least one context is an
 * FP32 P3M context): each step runs the contexts' phases up to the mesh force as parallel
 * branches, then merges their pair work lists into one list sorted by estimated cost and
 * evaluates every such context's pair sum in one persistent kernel launch (the contexts'
 * arguments read from a device table).  Other contexts step as before.  Results equal the
 * per-context launches bit for bit.  Every step then waits for all contexts' mesh phases
 * before the pair launch; on the 48-simulation ensemble of 48^3..96^3 particles the two are
 * within 1 % of each other with graphs.  enable = 0 returns to per-context pair launches.
 */
int p3m_ensemble_set_batched(p3m_ensemble *ens, int enable);
/*
 * Size-grouped FFTs (on by default when at least two contexts share a mesh size and precision;
 * enable = 0 turns them off, 1 on): the contexts of each such group get their density, spectrum
 * and force meshes as slices of one allocation per buffer, made by the ensemble, and every step
 * runs one batched R2C and one batched C2R per group on the ensemble's own stream instead of
 * one of each per context.  The steps then advance all contexts in lockstep phases (the mesh
 * deposit of all, the batched R2C, the k-space pass of all, the batched C2R, the gather and pair
 * force of all); without groups each context's steps are one independent branch.  Results equal
 * the per-context FFTs bit for bit.  p3m_ensemble_free (or enable = 0) copies the slices' contents
 * back into the contexts' own meshes and releases the group buffers.  A context already grouped
 * by another ensemble keeps its own FFTs in this one.  Batched pair launches
 * (p3m_ensemble_set_batched) take precedence: with them on, each context runs its own FFTs.
 */
int p3m_ensemble_set_fft_groups(p3m_ensemble *ens, int enable);

/*
 * Autotuner of the sort key's Hilbert depth and of the FP32 pair kernel's tile length: times two
 * force evaluations of the current particles for each sub_bits in 0..3 whose key fits in 32 bits
 * (ms_out[b], nullable; NaN when skipped), keeps the fastest (*sub_bits_out), then (FP32 P3M
 * contexts) times tiles of 3 and 5 blocks of 32 j particles at that depth and keeps the faster,
 * and leaves valid forces.  The cells, and hence which pairs interact, do not depend on either
 * choice; the forces agree up to the FP32 rounding of a different summation order.
 * p3m_get_tuning reports the current choices (tile_blocks: 3 or 5; 5 by default).
 */
int p3m_autotune(p3m_ctx *ctx, int *sub_bits_out, double *ms_out);
int p3m_get_tuning(const p3m_ctx *ctx, int *sub_bits, int *tile_blocks);

/*
 * Reverse-mode derivatives, for gradients of a loss through the step:
 *
 * p3m_force_vjp: out3n = (dA/dx)^T v3n, the transposed Jacobian of the accelerations A at the
 *   current positions applied to the vector field v [3][n] (caller order).  The mesh part is
 *   the CIC gather/deposit transposed through the conjugate Green's-function multiply; the
 *   pair part is sum_j J(d_kj)(v_j - v_k) with J the 3x3 Jacobian of the pair force.  Sorts
 *   and evaluates the mesh part at the current positions (cached forces are invalidated with
 *   P3M: the next p3m_step re-evaluates them).  The discontinuities of the
 *   CIC weight derivatives (mesh planes) and of the pair force at r_c are not differentiated.
 * p3m_density_loss: *loss = sum_nodes (delta - target)^2 with delta = n/n_bar - 1 the CIC
 *   density contrast of the current positions on the M^3 mesh, target[M^3] doubles (index
 *   (ix*M + iy)*M + iz); grad3n (nullable) = dL/dx [3][n].  Synchronises (loss is a host
 *   pointer).
 * p3m_axpy: y3n += alpha x3n over 3n doubles (device arrays).
 * p3m_step_factors: the step's kick factors m K(a, a+da/2), m K(a+da/2, a+da) and drift factor
 *   D(a, a+da)/m, as p3m_step uses them.
 * Pointers follow on_device as elsewhere (p3m_axpy: device only).
 */
int p3m_force_vjp(p3m_ctx *ctx, const double *v3n, double *out3n, int on_device);
int p3m_density_loss(p3m_ctx *ctx, const double *target, double *loss, double *grad3n,
                     int on_device);
int p3m_axpy(p3m_ctx *ctx, double alpha, const double *x3n, double *y3n);
int p3m_step_factors(const p3m_ctx *ctx, double a, double da, double *k1, double *dfac,
                     double *k2);

/* Momentum, kinetic energy, pair count and cell statistics of the current state; with energy
 * tracking on, also the potential energy and the Layzer-Irvine residual (which sort and
 * evaluate the mesh at the current positions, so the next step re-evaluates the forces).
 * Synchronises the stream. */
int p3m_diagnostics(p3m_ctx *ctx, p3m_diag *out);

/*
 * Energies of the current state.  The guide defines no energy diagnostic; this is the standard
 * cosmic-energy check of cosmological N-body codes, the Layzer-Irvine equation
 * d[a (K + W)]/da = -K for the comoving potential Phi with nabla^2 Phi = 4 pi G (rho - rho_bar):
 *   *kinetic   = K = sum_i |p_i|^2 / (2 m a^2)
 *   *potential = W = (1/(2a)) sum_i m Phi_i, Phi_i the potential at particle i without its
 *     own r = 0 self-interaction (its periodic images kept):
 *     Phi_i = Phi_mesh(x_i) - S_i + (phi_per - phi_iso) + Phi_SR,i + 4 pi Gm (N/L^3) r_s^2,
 *     Phi_mesh the CIC-interpolated IFFT(G rho_k), S_i the particle's own share of it (its CIC
 *     weights pushed through K = IFFT(G)), phi_per - phi_iso the exact long-range potential of
 *     its own periodic images, Phi_SR,i = -Gm sum_{r_ij < r_c} erfc(r_ij/(2 r_s))/sqrt(r_ij^2 +
 *     eps^2), and the last term the short-range potential of the neutralising background.
 *     Pure PM (short_range = 0): Phi_mesh - S_i only.
 * Sorts and evaluates the mesh at the current positions (with P3M the next p3m_step
 * re-evaluates the forces).  Host pointers; synchronises.
 *
 * p3m_track_energy(ctx, 1) records a0 and a0 (K0 + W0) of the current state and from then on
 * adds the trapezoid rule's share of int K da after every step (p3m_step, p3m_run_steps,
 * graph-replayed or not; one extra reduction per step); p3m_diagnostics then reports the
 * residual.  p3m_track_energy(ctx, 0) stops it.
 */
int p3m_energy(p3m_ctx *ctx, double *kinetic, double *potential);
int p3m_track_energy(p3m_ctx *ctx, int enable);

/*
 * Sorted views of the last sort (after p3m_forces / p3m_step), for checking:
 *   keys      [n]  sort keys in sorted order: (cell << 3b) | Hilbert(sub-cell), where
 *                  cell = (c_z n_c + c_y) n_c + c_x
 *   ids       [n]  original particle index of each sorted slot
 *   cell_start[n_c^3 + 1] first sorted slot of each chaining cell; last entry n
 * Each pointer nullable; all uint32.
 */
int p3m_get_cells(p3m_ctx *ctx, uint32_t *keys, uint32_t *ids, uint32_t *cell_start,
                  int on_device);

/*
 * Copies a mesh of the last force evaluation: which = 0 the CIC count mesh minus its mean
 * N/M^3, 1..3 the x/y/z mesh accelerations.  M^3 values, index (ix*M + iy)*M + iz, as float
 * (P3M_PREC_MIXED) or double (P3M_PREC_FP64).
 */
int p3m_get_mesh(p3m_ctx *ctx, int which, void *out, int on_device);

/* Number of chaining cells per side, mesh size and precision mode of the context. */
int p3m_get_geometry(const p3m_ctx *ctx, int *n_c, int *mesh, int *precision, int *sub_bits);

/*
 * Per-phase device time.  p3m_set_timing(ctx, 1) records CUDA events on the context's stream
 * around each phase of every later force evaluation and step; p3m_timings synchronises, adds
 * the elapsed times per phase into ms[0..n-1] (milliseconds, summed since the last reset)
 * and, with reset != 0, clears them.  Returns the number of phases (P3M_NPHASES).
 */
#define P3M_NPHASES 10
int p3m_set_timing(p3m_ctx *ctx, int enable);
int p3m_timings(p3m_ctx *ctx, double *ms, int n, int reset);
/* Name of phase i ("kick_drift", "sort", "permute", "deposit", "fft_r2c", "kspace",
 * "fft_c2r", "gather", "pairs", "other"), or NULL. */
const char *p3m_phase_name(int i);

/*
 * Measurement helper (no counterpart in the guide): the FMA throughput of the current GPU in
 * TFLOP/s (an FMA counts 2 flops), FP32 (fp64 = 0) or FP64 (fp64 = 1), from independent
 * multiply-add chains over 8 blocks of 256 threads per SM; best of two timed launches after
 * a warm-up.  Allocates and frees a small device buffer and its own stream; synchronises.
 * Used for the roofline of the pair kernels: FP32 bounds the mixed mode, FP64 the all-FP64
 * mode.  Returns P3M_ECUDA on a CUDA error (*tflops = NaN).
 */
int p3m_measure_fma_peak(int fp64, double *tflops);

/*
 * Allocation-free cell binning.  The paper has no counterpart to this entry point: it serves
 * callers that may not allocate GPU memory themselves.  Examples are code embedded in a
 * framework whose own caching allocator owns the device memory (a cudaMalloc behind its back
 * escapes its accounting and fragments its pool), or a time-critical loop that cannot accept
 * cudaMalloc's device synchronisation and unpredictable latency.  p3m_init allocates; this
 * call does not.
 *
 * From caller-owned device arrays it computes what p3m_get_cells reports after a force
 * evaluation of a context with the same box, n_c and sub_bits:
 *   pos3n          [3][n] doubles on the device (not modified; wrapped into [0, box) for
 *                  the keys only)
 *   keys_out[n], ids_out[n], cell_start_out[n_c^3 + 1]   uint32 device arrays, caller-owned
 *   n_c            chaining cells per side (p3m_get_geometry of a context gives it)
 *   stream         cudaStream_t (NULL: legacy stream); the results are ready when the stream
 *                  reaches the end of the call's work
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its temporary storage is one
 * fixed area of about 12.3 MiB that the library reserves in the GPU's global memory when it
 * is loaded.  Every GPU that loads the library holds that area until the process exits, and
 * it bounds n to at most P3M_NOALLOC_MAX_N particles.  Larger n, NULL pointers or an invalid
 * geometry return P3M_EINVAL before any launch, with the reason in p3m_last_error(NULL).
 * The first call on each device performs a set-up (it looks up the device address of that
 * area with the device current); make that first call before any stream capture begins.
 * Calls made while the stream is not capturing look the address up again, so that after a
 * cudaDeviceReset the next call outside capture refreshes it; a call inside a capture uses the
 * address found by the last call outside one (P3M_ECUDA if there was none).
 * All calls share the one area, which keeps the contents of the last call (nothing in it needs
 * to start at zero): calls whose GPU work overlaps, on different streams or from different
 * host threads, race and corrupt each other's results.  Order them on one stream.
 */

#define P3M_NOALLOC_MAX_N 1048576
int p3m_cell_sort_noalloc(const double *pos3n, int64_t n, double box, int n_c, int sub_bits,
                          uint32_t *keys_out, uint32_t *ids_out, uint32_t *cell_start_out,
                          void *stream);

/*
 * Host-side fault injection, for testing how the library reports failures without making the
 * GPU fault (the guide has no counterpart).  what:
 *   P3M_INJECT_ALLOC       the device allocation number arg (0-based, in the order p3m_init
 *                          makes them) of every following p3m_init fails as if cudaMalloc had
 *                          returned cudaErrorMemoryAllocation: p3m_init frees what it had
 *                          allocated and returns P3M_ENOMEM, and p3m_last_error(NULL) names the
 *                          allocation and says "(injected)".  Process-wide; ctx may be NULL.
 *   P3M_INJECT_FFT_PLAN    every following p3m_init fails at its first cuFFT plan as if the
 *                          plan call had returned CUFFT_ALLOC_FAILED (P3M_ECUFFT).  Process-wide.
 *   P3M_INJECT_SORT_TIMEOUT  on ctx: the particle sort's look-back waits on a zeroed status word
 *                          that nothing sets and gives up after arg clock cycles (1..2^31), so
 *                          force evaluations return P3M_ETIMEOUT right after the sort, before
 *                          any kernel reads the (unreliable) order; the particle state is kept.
 *                          Allocates a zeroed buffer the size of the sort's look-back status.
 *   P3M_INJECT_NONE        clears every injection (and, with ctx, frees that buffer and restores
 *                          the default wait limit of 2^31 cycles); the context is usable again.
 * Returns P3M_EINVAL for an unknown fault or argument.
 */
#define P3M_INJECT_NONE 0
#define P3M_INJECT_ALLOC 1
#define P3M_INJECT_FFT_PLAN 2
#define P3M_INJECT_SORT_TIMEOUT 3
int p3m_inject_fault(p3m_ctx *ctx, int what, int64_t arg);

/*
 * Checks of debug builds (the library compiled with -DP3M_DEBUG_CHECKS; the guide has no
 * counterpart; they stand in for a memory checker).  In such a build the kernels test the
 * indices they compute (mesh nodes of the deposit and gather, source slots of the permute, cell
 * ranges, key range, pair tile lengths) and, on a failed test, set a flag and skip the access;
 * and every device allocation of p3m_init is followed by 256 guard bytes of a fixed pattern.
 * p3m_debug_check synchronises, reports a set flag or an overwritten guard byte as P3M_EBOUNDS
 * (with the allocation's index in the message) and clears the flag; in release builds it checks
 * the flags only.  p3m_debug_poke_canary overwrites one guard byte of allocation k (host-side,
 * inside that allocation), so that a test can see the check catch it; P3M_ESTATE in release
 * builds.
 */
int p3m_debug_check(p3m_ctx *ctx);
int p3m_debug_poke_canary(p3m_ctx *ctx, int k);

/* Message of the last failure on ctx (ctx NULL: the last failed p3m_init).  Never NULL. */
const char *p3m_last_error(const p3m_ctx *ctx);

/* Releases everything the context owns.  NULL is ignored. */
void p3m_free(p3m_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* P3M_H */
