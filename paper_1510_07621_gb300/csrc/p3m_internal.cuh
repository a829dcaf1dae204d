// Internal declarations of the P3M library: the context and the launchers of each phase.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include "p3m.h"

// Degree of the fitted FP32 split factor Q (Chebyshev fit on [0, r_c]).  Its largest error in g
// is 5.8e-6 (near r_c, where g = 0.0175).  Against the FP64 oracle the FP32 short-range force
// then differs by 7.50e-6 relative RMS on the 32^3 Zel'dovich state at a = 0.02 (7.31e-6 at
// degree 10, 1.8e-5 at degree 7: the FP32 rounding of nearly cancelling pair sums dominates)
// and by 1.7e-6 on a clustered state.
#define P3M_SPLIT_DEG 8
// Degree of the FP64 split factor of the FP64 pair kernel: its largest error in g is about
// 4e-14 relative (at r_c), far below the FP64 mode's 1e-12 parity bar.
#define P3M_SPLIT_DEG64 18

// Chaining-cell geometry, mesh constants and the per-evaluation scalars every kernel needs.
struct P3MGeom {
    double box;       // L
    int64_t n;        // N
    int mesh;         // M
    double inv_h;     // M / L
    double r_s, r_c;  // split scale and cutoff (length)
    double eps;       // Plummer softening (length)
    double gm;        // G m
    int n_c;          // chaining cells per side
    int sub_bits;     // b
    int n_fine;       // n_c << b
    double inv_fine;  // n_fine / L
    double cs;        // L / n_c
    int n_cells;      // n_c^3
    double mean_count;  // N / M^3
    uint32_t *flags;    // the context's device error flags (debug bounds checks record here)
};

// Bounds checks of debug builds (compiled with -DP3M_DEBUG_CHECKS): p3m_in_bounds(ok, flags)
// records a failed check in the context's flags (P3M_FLAG_BOUNDS) and returns ok, so that the
// caller skips the access; nothing traps.  In release builds it is the constant true and the
// check disappears.
#define P3M_FLAG_BOUNDS 4u
#ifdef P3M_DEBUG_CHECKS
__device__ __forceinline__ bool p3m_in_bounds(bool ok, uint32_t *flags)
{
    if (!ok && flags) atomicOr(flags, P3M_FLAG_BOUNDS);
    return ok;
}
#else
__device__ __forceinline__ bool p3m_in_bounds(bool, uint32_t *) { return true; }
#endif

struct p3m_ctx {
    P3MGeom g;
    int precision;
    int deconvolve;
    int short_range;
    p3m_cosmology cosmo;
    double mass;
    double a;
    cudaStream_t stream;
    int num_sms;
    int l2_bytes;  // L2 cache size of the device

    // particle state in sorted order, SoA [3][n]
    double *pos, *mom, *acc, *acc_lr;
    uint32_t *pid;
    double *pos_alt, *mom_alt;  // permute targets / staging
    uint32_t *pid_alt;
    void *rel;  // float4 (mixed) or double4_16a (fp64): position relative to its cell origin
    float4 *block_box;  // per 32-slot block of the sorted order: lo, hi (FP32, absolute)
    float *relx;        // FP32 mode: rel as block-SoA, per 32-slot block x[32] y[32] z[32]
    int tile_blocks;    // FP32 pair kernel: 32-slot blocks per shared-memory tile (3 or 5)

    // sort
    uint32_t *keys, *keys_alt, *vals, *vals_alt;
    uint32_t *digit_counts;  // 256 * n_tiles
    uint32_t *scan_aux;      // block sums of the scans
    unsigned long long *sort_status;  // particle sort: 256 look-back entries per 4096-key tile
    uint32_t *sort_hist;              // particle sort: 4 x 256 digit counts, 4 tile counters
    int n_tiles;
    int key_bits;
    long long sort_wait_limit;          // clock cycles one look-back wait may take (2^31 ~ 1 s)
    unsigned long long *sort_probe;     // injected sort timeout: a zeroed status that nothing sets
    uint32_t *cell_start;  // n_cells + 1
    uint32_t *work;        // pair work items (cell, first slot)
    uint32_t *work_off;    // n_cells + 1
    uint32_t *work_key, *work_key_alt;      // cost keys of the work items (max_work)
    uint32_t *work_order, *work_order_alt;  // work items, most expensive first (max_work)
    size_t max_work;
    uint32_t *counters;  // [0] work cursor [1] error flags [2] max cell count [3] spare
    unsigned long long *pair_count;  // [0] last evaluation [1] cumulative
    unsigned long long launches;     // kernels launched by the library (host-side count)
    double *red;  // reduction partials

    // mesh (float or double)
    void *rho, *rho_k, *frc_k, *frc;
    void *tab_k, *tab_kg, *tab_g;  // per-axis |k|, gradient k, Green factor (length M)
    double *tab_invw2;             // per-axis 1/sinc^4(k h/2) (FP64, length M)
    double *tab_one;               // M ones (no deconvolution)
    double *tab_origin;            // n_c chaining-cell origins c * cs (FP64, correctly rounded)
    double *ps_acc;                // power spectrum sums (3 * (M/2) + 1)
    double *ps_part;               // power spectrum per-block partial sums (ps_blocks rows)
    int ps_blocks;
    // fixed-point deposit accumulator: 3 M^3 64-bit integers, cleared before each deposit; sums
    // of integers do not depend on the order of the atomic additions, so every run gives the
    // same mesh
    unsigned long long *rho_fix;
    int *fix_exp;  // scale exponent of the vector deposit (set on the device)
    double green_const;
    float gpoly[12];  // FP32 split factor: g = 1 + r^3 Q(tau), Q = sum gpoly[k] tau^k
                      // (k <= P3M_SPLIT_DEG), tau = r^2 gpoly[11] - 1
    double gpoly64[P3M_SPLIT_DEG64 + 2];  // the same in FP64 (degree P3M_SPLIT_DEG64); the
                                          // last entry is tau's scale
    cufftHandle plan_r2c, plan_c2r, plan_c2r_one;  // R2C, batched 3 x C2R, single C2R
    bool plans_made;

    // timing
    bool timing;
    cudaEvent_t *ev;
    int *ev_phase;
    int ev_used, ev_cap;
    double phase_ms[P3M_NPHASES];

    // graph-replayed steps: per-step factors (K1, D, K2) for up to fac_cap steps, the device
    // step counter, and the two captured step graphs (even and odd step parity)
    double *fac_table;
    uint32_t *step_idx;
    double *cur_fac;  // factors of the step being executed: K1, D, K2
    int fac_cap;
    bool capturing;
    int geom_version;              // bumped when the geometry changes (captured graphs go stale)
    struct p3m_ensemble *self_ens;  // private one-context ensemble of p3m_run_steps

    // reverse-mode derivative buffers
    void *adj_u;       // three real meshes (vector deposit; also target-mesh staging)
    float *adj_vfx;    // FP32 mode: v in slot order as block-SoA (per 32 slots vx[32] vy[32] vz[32];
                       // zero past the last particle)
    double *adj_vs;    // v in slot order, FP64 [3][n]
    double *adj_out;   // result in slot order [3][n]

    // energies: K = IFFT(G) at the 27 offsets around the origin (mesh self-energy), the
    // Layzer-Irvine bookkeeping [integral K da, sum p^2 at the last step, a at the last step]
    double *kself;
    bool kself_ready;
    double *li;
    bool track_energy;
    double li_a0, li_e0;

    // debug builds: the guard bytes after every device allocation of p3m_init (canaries)
    int n_canary;
    void *canary_ptr[64];
    size_t canary_off[64];

    bool fft_grouped;  // its meshes are slices of an ensemble's FFT group (p3m_ensemble_set_fft_groups)

    bool have_particles;
    bool forces_valid;
    bool sorted_valid;
    char err[512];
};

enum {
    PH_KICK_DRIFT = 0,
    PH_SORT,
    PH_PERMUTE,
    PH_DEPOSIT,
    PH_FFT_R2C,
    PH_KSPACE,
    PH_FFT_C2R,
    PH_GATHER,
    PH_PAIRS,
    PH_OTHER
};

#define P3M_MAX_GRAPH_STEPS 4096  // steps per p3m_run_steps / p3m_ensemble_run call
#define P3M_SORT_TILE 4096   // keys per radix-sort tile (256 threads x 16)
#define P3M_PAIR_TI 32       // i-particles per pair work item (one per lane of a warp)
#define P3M_PAIR_TJ 128      // j-particles per shared-memory tile (4 blocks of 32)
#define P3M_FLAG_TIMEOUT 1u  // counters[1] bit: a bounded wait gave up

// Everything the FP32 pair kernel needs from one context: its arrays, geometry, fitted split
// factor and culling radii, where the accelerations go and the fused final half-kick (factor
// kfac, or *kfac_dev when that is set).  Passed by value for one context, or as a device array
// indexed by simulation in the batched ensemble launch.
struct PairArgs {
    const float *relx;
    const float4 *rel;
    const double *pos;
    const float4 *block_box;
    const uint32_t *cell_start;
    const uint32_t *work;
    const double *acc_in;
    double *acc_out;
    double *mom;
    const double *kfac_dev;
    uint32_t *counters;
    unsigned long long *pair_count;
    double kfac;
    P3MGeom g;
    float gpoly[12];
    float rcull2, rin2;
};

// A neighbour cell of a pair work item, for the FP32 pair kernels: the shift between the two
// cells' origins (periodic image included) as an FP32 value plus the FP32 residual of the FP64
// shift, the periodic image alone, and the neighbour's range of sorted slots.
struct NeighbourF {
    uint32_t start, end;
    float sx, sy, sz, rx, ry, rz;
    float imx, imy, imz, pad;
};

// Neighbour nb (0..26, offsets (nb%3-1, nb/3%3-1, nb/9-1)) of cell (cx, cy, cz); an empty
// neighbour gets start = end = 0.
__device__ __forceinline__ NeighbourF make_neighbour(const P3MGeom &g, const uint32_t *cell_start,
                                                     int cx, int cy, int cz, int nb)
{
    const int nc = g.n_c;
    const int ux = cx + nb % 3 - 1, uy = cy + (nb / 3) % 3 - 1, uz = cz + nb / 9 - 1;
    const int wx = (ux + nc) % nc, wy = (uy + nc) % nc, wz = (uz + nc) % nc;
    const uint32_t q = ((uint32_t)wz * nc + wy) * nc + wx;
    NeighbourF r;
    r.start = cell_start[q];
    r.end = cell_start[q + 1];
    if (!p3m_in_bounds(r.start <= r.end && r.end <= (uint32_t)g.n, g.flags)) r.end = r.start;
    if (r.start == r.end) r.start = r.end = 0;
    const double L = g.box, cs = g.cs;
    const double imx = ux < 0 ? -L : (ux >= nc ? L : 0.0);
    const double imy = uy < 0 ? -L : (uy >= nc ? L : 0.0);
    const double imz = uz < 0 ? -L : (uz >= nc ? L : 0.0);
    const double sx = ((double)wx * cs + imx) - (double)cx * cs;
    const double sy = ((double)wy * cs + imy) - (double)cy * cs;
    const double sz = ((double)wz * cs + imz) - (double)cz * cs;
    r.sx = (float)sx;
    r.sy = (float)sy;
    r.sz = (float)sz;
    r.rx = (float)(sx - (double)r.sx);
    r.ry = (float)(sy - (double)r.sy);
    r.rz = (float)(sz - (double)r.sz);
    r.imx = (float)imx;
    r.imy = (float)imy;
    r.imz = (float)imz;
    r.pad = 0.0f;
    return r;
}

#define P3M_FLAG_NONFINITE 2u

// ------------------------------------------------------------------ launchers (sort.cu)
// Wraps positions and writes keys (optionally after a kick with kfac = m K and a drift with
// dfac = D / m).  vals are not touched.
cudaError_t launch_kick_drift_keys(p3m_ctx *c, bool kick_drift, double kfac, double dfac,
                                   bool from_table = false);
// Stable LSD radix sort of (keys, identity) -> c->keys (sorted), c->vals (source slots).
cudaError_t launch_radix_sort(p3m_ctx *c);
// Permutes pos/mom/pid by c->vals, writes the relative coordinates, cell_start, work list.
cudaError_t launch_permute_and_cells(p3m_ctx *c);
// Exclusive scan of n uint32 values (in may equal out); aux needs ceil(n/4096)+1 entries.
cudaError_t launch_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *aux,
                            cudaStream_t s);

// ------------------------------------------------------------------ launchers (mesh.cu)
// from_rel: the sorted state is fresh (right after the permute), so the FP32 mode may take the
// stencils from the cell-relative coordinates; otherwise (any particle order) from pos in FP64.
cudaError_t launch_deposit(p3m_ctx *c, bool from_rel = false);
cudaError_t launch_kspace(p3m_ctx *c);
// Right after the permute: the FP32 mode reads the stencils from the sorted rel and keys.
cudaError_t launch_gather(p3m_ctx *c, double *acc_out);
// kernel attributes of the mesh kernels (shared-memory carveout), set once per process
cudaError_t mesh_set_attributes();
// Bins the spectrum in c->rho_k into acc[3 n_bins + 1] (see k_powspec).
cudaError_t launch_powspec(p3m_ctx *c, const double *inv_w2, double radius, int n_bins, double *acc);

// ------------------------------------------------------------------ launchers (pair.cu)
// acc_out = acc_in + SR (acc_in NULL: SR only); kfac != 0: mom += kfac * acc_out.  kfac_dev
// (nullable): read kfac from device memory instead.
// FP32 contexts: the pair kernel's arguments for the current buffers (host-side fill).
PairArgs pair_args(const p3m_ctx *c, const double *acc_in, double *acc_out, double kfac,
                   const double *kfac_dev);
// One pair launch over the work items of several FP32 contexts: order[k] = (sim << 24) | item,
// sorted by cost; *n_total items; descs[sim] the contexts' arguments; cursor zeroed here.
cudaError_t launch_pairs_batched(const PairArgs *descs, const uint32_t *order,
                                 const uint32_t *n_total, uint32_t *cursor, int num_sms,
                                 cudaStream_t s);
// dst (device) = a, as one kernel (so that captured graphs write the current pointers).
cudaError_t launch_store_pair_args(PairArgs *dst, const PairArgs &a, cudaStream_t s);
// Batched launch bookkeeping: copies one context's sorted work list (n entries) into the merged
// arrays, values coded (slot << 24) | item; *total = sum over nb contexts of *nwork[k].
cudaError_t launch_ens_gather(int slot, const uint32_t *key, const uint32_t *order, size_t n,
                              uint32_t *gkey, uint32_t *gval, cudaStream_t s);
cudaError_t launch_ens_total(const uint32_t *const *nwork, int nb, uint32_t *total, cudaStream_t s);
// Stable LSD radix sort of n (key, value) pairs on the low key_bits bits; k[0]/v[0] hold the
// result on return (the arrays are swapped when an odd number of passes ran).
cudaError_t radix_sort_pairs(uint32_t **k, uint32_t **v, bool identity_vals, int64_t n,
                             int key_bits, uint32_t *counts, uint32_t *aux, cudaStream_t s,
                             unsigned long long *launches);
cudaError_t launch_pairs(p3m_ctx *c, const double *acc_in, double *acc_out, double kfac,
                         const double *kfac_dev = nullptr);

// ------------------------------------------------------------------ launchers (integrate.cu)
cudaError_t launch_kick(p3m_ctx *c, double kfac, const double *kfac_dev = nullptr);
// cur_fac = fac_table[3 s .. 3 s + 2], s = *step_idx, then *step_idx = s + 1 (the first launch
// of a graph-replayed step)
cudaError_t launch_step_begin(p3m_ctx *c);
// y += alpha x over 3n values
cudaError_t launch_axpy(p3m_ctx *c, double *y, const double *x, double alpha);
cudaError_t launch_load_particles(p3m_ctx *c, const double *pos, const double *mom,
                                  const double *acc);
cudaError_t launch_scatter_out(p3m_ctx *c, const double *src, double *dst);
// inv[pid[k]] = k, then dst[j] = src[inv[j]] (3 x n): caller order with sequential writes
cudaError_t launch_inverse_pid(p3m_ctx *c, uint32_t *inv);
cudaError_t launch_gather_out(p3m_ctx *c, const double *src, const uint32_t *inv, double *dst);
cudaError_t launch_diag(p3m_ctx *c, double *host_out /* [4]: px py pz 2*kinetic*m*a^2 */);

// ------------------------------------------------------------------ launchers (adjoint.cu)
// vs (and, FP32 mode, adj_vfx) = v permuted from caller order into slot order
cudaError_t launch_to_slots(p3m_ctx *c, const double *v, double *vs);
// out_slots = (dA/dx)^T v_slots at the current (sorted, evaluated) state
cudaError_t launch_force_vjp(p3m_ctx *c, const double *v_slots, double *out_slots);
// loss_dev = sum (rho/n_bar - target)^2 over the deposited mesh; grad_slots (nullable) = dL/dx
cudaError_t launch_density_loss(p3m_ctx *c, const double *target, double *loss_dev, double *grad_slots);
// phi_slots = potential of each particle (cst added), *sum_dev = sum over particles; needs the
// sorted, evaluated state with FFT(rho) in rho_k
cudaError_t launch_potential(p3m_ctx *c, double cst, double *phi_slots, double *sum_dev);
// Layzer-Irvine: sum p^2 now, then li[0] += (K_prev + K_now)/2 (a_now - li[2]), K = sum p^2/(2 m a^2)
cudaError_t launch_li_update(p3m_ctx *c, const double *a_now_dev, double a_now);

// host helpers (api.cu)
// Records a message for p3m_last_error(NULL) and returns code.
int p3m_fail_global(int code, const char *fmt, ...);
double p3m_kick_factor(const p3m_cosmology &cs, double a1, double a2);
double p3m_drift_factor(const p3m_cosmology &cs, double a1, double a2);
