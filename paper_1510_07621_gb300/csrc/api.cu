// C ABI of the P3M library, core part: argument checks, the context (all device memory and cuFFT
// plans allocated in p3m_init), the order of the phases of a force evaluation and of a
// kick-drift-kick step, particle I/O, power spectrum and diagnostics.  Every kernel launch goes
// to the context's stream.  Ensembles and graphs: ensemble.cu; reverse mode and energies:
// derivatives.cu.
#include <cuda_runtime.h>
#include <cufft.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "host_internal.h"

char g_init_err[512] = "no error";

namespace p3m_host {

int fail(p3m_ctx *c, int code, const char *fmt, ...)
{
    char *buf = c ? c->err : g_init_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return code;
}

// ---------------------------------------------------------------- cosmology (host, FP64)

bool is_eds(const p3m_cosmology &cs) { return cs.omega_m == 1.0 && cs.omega_lambda == 0.0; }

double hubble(const p3m_cosmology &cs, double a)
{
    const double ok = 1.0 - cs.omega_m - cs.omega_lambda;
    return sqrt(cs.omega_m / (a * a * a) + ok / (a * a) + cs.omega_lambda);
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n from the
// Chebyshev-point initial guesses).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

double quad(const p3m_cosmology &cs, double a1, double a2, int power)
{
    static std::vector<double> xg, wg;
    if (xg.empty()) gauss_legendre(48, xg, wg);
    double s = 0.0;
    for (size_t i = 0; i < xg.size(); ++i) {
        const double a = 0.5 * (a2 - a1) * xg[i] + 0.5 * (a2 + a1);
        s += wg[i] / (pow(a, power) * hubble(cs, a));
    }
    return 0.5 * (a2 - a1) * s;
}

// ---------------------------------------------------------------- split factor fit
// g(x) = erfc(x/2) + x/sqrt(pi) exp(-x^2/4) = 1 + x^3 Q(x^2).  Q is smooth (entire) in u = x^2;
// it is interpolated at Chebyshev-Gauss nodes of u in [0, u_c], u_c = (r_c/r_s)^2, truncated to
// the wanted degree (a near-minimax polynomial), and rewritten in monomial form in
// tau = 2u/u_c - 1 for Horner evaluation (the monomial coefficients stay below 0.03 in size up to
// degree 22, so the rewriting costs no accuracy).  The kernels evaluate g = 1 + r^3 Q'(tau)
// directly from r^2, so the coefficients are scaled by r_s^-3 and tau = r^2 (2 / (u_c r_s^2)) - 1.

// Q(u): below u = 1 from its Taylor series (the closed form cancels there),
// Q(u) = (1/sqrt(pi)) sum_{n>=1} (-1)^n u^(n-1) 2n / (4^n n! (2n+1)); above, (g - 1)/(u x).
double split_q(double u)
{
    const double inv_sqrt_pi = 0.56418958354775628695;
    if (u < 1.0) {
        double b = -0.25, sum = 0.0;  // b_n = (-1)^n u^(n-1) / (4^n n!), from b_1 = -1/4
        for (int n = 1; n <= 30; ++n) {
            sum += b * (2.0 * n) / (2.0 * n + 1.0);
            b *= -0.25 * u / (n + 1);
        }
        return inv_sqrt_pi * sum;
    }
    const double x = sqrt(u);
    const double gval = erfc(0.5 * x) + x * inv_sqrt_pi * exp(-0.25 * u);
    return (gval - 1.0) / (u * x);
}

// Monomial coefficients mono[0..deg] of Q in tau (unscaled), from `nodes` Chebyshev nodes.
void fit_split_mono(double cutoff_in_rs, int deg, int nodes, double *mono)
{
    const double uc = cutoff_in_rs * cutoff_in_rs;
    std::vector<double> cheb(deg + 1, 0.0), tk_prev(deg + 1, 0.0), tk(deg + 1, 0.0), next(deg + 1);
    for (int j = 0; j < nodes; ++j) {
        const double th = M_PI * (j + 0.5) / nodes, t = cos(th);
        const double q = split_q(0.5 * (t + 1.0) * uc);
        for (int k = 0; k <= deg; ++k) cheb[k] += q * cos(k * th);
    }
    for (int k = 0; k <= deg; ++k) cheb[k] *= (k == 0 ? 1.0 : 2.0) / nodes;
    // Chebyshev series -> monomials: T_0 = 1, T_1 = t, T_{k+1} = 2 t T_k - T_{k-1}
    for (int i = 0; i <= deg; ++i) mono[i] = 0.0;
    tk_prev[0] = 1.0;
    mono[0] += cheb[0];
    if (deg >= 1) {
        tk[1] = 1.0;
        for (int i = 0; i <= deg; ++i) mono[i] += cheb[1] * tk[i];
    }
    for (int k = 2; k <= deg; ++k) {
        for (int i = 0; i <= deg; ++i) next[i] = -tk_prev[i] + (i > 0 ? 2.0 * tk[i - 1] : 0.0);
        for (int i = 0; i <= deg; ++i) {
            mono[i] += cheb[k] * next[i];
            tk_prev[i] = tk[i];
            tk[i] = next[i];
        }
    }
}

// FP32 coefficients (degree P3M_SPLIT_DEG) into out[0..10], tau's scale into out[11].
void fit_split_poly(double cutoff_in_rs, double r_s, float out[12])
{
    double mono[P3M_SPLIT_DEG + 1];
    fit_split_mono(cutoff_in_rs, P3M_SPLIT_DEG, 40, mono);
    const double uc = cutoff_in_rs * cutoff_in_rs, inv_rs3 = 1.0 / (r_s * r_s * r_s);
    for (int i = 0; i <= P3M_SPLIT_DEG; ++i) out[i] = (float)(mono[i] * inv_rs3);
    for (int i = P3M_SPLIT_DEG + 1; i < 11; ++i) out[i] = 0.0f;
    out[11] = (float)(2.0 / (uc * r_s * r_s));
}

// FP64 coefficients (degree P3M_SPLIT_DEG64, largest error in g about 4e-14 relative) into
// out[0..P3M_SPLIT_DEG64], tau's scale into out[P3M_SPLIT_DEG64 + 1].
void fit_split_poly64(double cutoff_in_rs, double r_s, double *out)
{
    double mono[P3M_SPLIT_DEG64 + 1];
    fit_split_mono(cutoff_in_rs, P3M_SPLIT_DEG64, 64, mono);
    const double uc = cutoff_in_rs * cutoff_in_rs, inv_rs3 = 1.0 / (r_s * r_s * r_s);
    for (int i = 0; i <= P3M_SPLIT_DEG64; ++i) out[i] = mono[i] * inv_rs3;
    out[P3M_SPLIT_DEG64 + 1] = 2.0 / (uc * r_s * r_s);
}

// ---------------------------------------------------------------- phase timing

void harvest(p3m_ctx *c)
{
    if (c->ev_used == 0) return;
    cudaEventSynchronize(c->ev[c->ev_used - 1]);
    for (int i = 0; i + 1 < c->ev_used; i += 2) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]) == cudaSuccess)
            c->phase_ms[c->ev_phase[i]] += ms;
    }
    c->ev_used = 0;
}

const char *kPhaseNames[P3M_NPHASES] = {"kick_drift", "sort",   "permute", "deposit", "fft_r2c",
                                        "kspace",     "fft_c2r", "gather", "pairs",   "other"};

// ---------------------------------------------------------------- context lifetime

void release(p3m_ctx *c)
{
    void *bufs[] = {c->pos,       c->mom,      c->acc,          c->acc_lr,   c->pid,
                    c->pos_alt,   c->mom_alt,  c->pid_alt,      c->rel,      c->keys,
                    c->keys_alt,  c->vals,     c->vals_alt,     c->digit_counts, c->scan_aux,
                    c->cell_start, c->work,    c->work_off,     c->counters, c->pair_count,
                    c->red,       c->rho,      c->rho_k,        c->frc_k,    c->frc,
                    c->tab_k,     c->tab_kg,   c->tab_g,        c->work_key, c->work_key_alt,
                    c->work_order, c->work_order_alt, c->block_box, c->tab_invw2,
                    c->tab_one,   c->ps_acc,   c->fac_table,    c->step_idx, c->cur_fac,
                    c->tab_origin,
                    c->adj_u,     c->adj_vfx,  c->adj_vs,       c->adj_out,  c->kself,
                    c->li,        c->relx,     c->sort_status,  c->sort_hist,
                    c->rho_fix,   c->fix_exp,  c->ps_part,     c->sort_probe};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (c->plans_made) {
        cufftDestroy(c->plan_r2c);
        cufftDestroy(c->plan_c2r);
        cufftDestroy(c->plan_c2r_one);
    }
    if (c->ev) {
        for (int i = 0; i < c->ev_cap; ++i) cudaEventDestroy(c->ev[i]);
        free(c->ev);
        free(c->ev_phase);
    }
}

// Host-side fault injection (p3m_inject_fault): the index of the p3m_init device allocation
// that fails (-1: none) and whether p3m_init's cuFFT plans fail.
int g_inject_alloc = -1;
bool g_inject_fft = false;

#ifdef P3M_DEBUG_CHECKS
constexpr size_t kCanaryBytes = 256;  // guard bytes after each allocation of p3m_init
constexpr unsigned char kCanary = 0xA5;
#endif

template <typename T>
cudaError_t dalloc(T **p, size_t bytes, p3m_ctx *c)
{
    *p = nullptr;
    bytes = bytes < 16 ? 16 : bytes;
#ifdef P3M_DEBUG_CHECKS
    const size_t off = (bytes + 255) / 256 * 256;  // the guard starts 256-byte aligned
    cudaError_t e = cudaMalloc((void **)p, off + kCanaryBytes);
    if (e == cudaSuccess) e = cudaMemset((char *)*p + off, kCanary, kCanaryBytes);
    if (e == cudaSuccess && c->n_canary < 64) {
        c->canary_ptr[c->n_canary] = *p;
        c->canary_off[c->n_canary] = off;
        ++c->n_canary;
    }
    return e;
#else
    (void)c;
    return cudaMalloc((void **)p, bytes);
#endif
}

int check_flags(p3m_ctx *c)
{
    uint32_t flags = 0;
    CK(cudaMemcpyAsync(&flags, c->counters + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (flags & P3M_FLAG_BOUNDS) {
        CK(cudaMemsetAsync(c->counters + 1, 0, sizeof(uint32_t), c->stream));
        c->forces_valid = false;
        return fail(c, P3M_EBOUNDS, "a debug bounds check failed in a kernel (the access was skipped)");
    }
    if (flags & P3M_FLAG_TIMEOUT) {
        CK(cudaMemsetAsync(c->counters + 1, 0, sizeof(uint32_t), c->stream));  // reported once
        c->forces_valid = false;
        c->sorted_valid = false;
        return fail(c, P3M_ETIMEOUT, "a bounded device-side wait gave up");
    }
    return P3M_OK;
}

// ---------------------------------------------------------------- force evaluation
// Sort by cell, mesh force, pair force.  Positions must already be wrapped and keyed
// (c->keys).  Result: c->acc (total), c->acc_lr (mesh part).  kfac != 0: the final half kick
// mom += kfac * acc is fused into the last kernel.  The phases are also run one by one by
// ensembles whose contexts share batched FFTs (eval_pre, the R2C, eval_kspace, the C2R,
// eval_post).

// Sort, permute, cell ranges and work list, CIC deposit.
int eval_pre(p3m_ctx *c)
{
    {
        Phase ph(c, PH_SORT);
        CK(launch_radix_sort(c));
    }
    if (c->sort_probe) {  // injected sort timeout: stop before anything reads the order
        const int rc = check_flags(c);
        if (rc) return rc;
    }
    {
        Phase ph(c, PH_PERMUTE);
        CK(launch_permute_and_cells(c));
    }
    c->sorted_valid = true;
    {
        Phase ph(c, PH_DEPOSIT);
        CK(launch_deposit(c, true));
    }
    return P3M_OK;
}

int eval_r2c(p3m_ctx *c)
{
    Phase ph(c, PH_FFT_R2C);
    CKF(c->precision == P3M_PREC_MIXED
            ? cufftExecR2C(c->plan_r2c, (cufftReal *)c->rho, (cufftComplex *)c->rho_k)
            : cufftExecD2Z(c->plan_r2c, (cufftDoubleReal *)c->rho, (cufftDoubleComplex *)c->rho_k));
    return P3M_OK;
}

int eval_kspace(p3m_ctx *c)
{
    Phase ph(c, PH_KSPACE);
    CK(launch_kspace(c));
    return P3M_OK;
}

int eval_c2r(p3m_ctx *c)
{
    Phase ph(c, PH_FFT_C2R);
    CKF(c->precision == P3M_PREC_MIXED
            ? cufftExecC2R(c->plan_c2r, (cufftComplex *)c->frc_k, (cufftReal *)c->frc)
            : cufftExecZ2D(c->plan_c2r, (cufftDoubleComplex *)c->frc_k, (cufftDoubleReal *)c->frc));
    return P3M_OK;
}

// Gather, then the pair force (or, for pure PM, the mesh force alone) with the final kick.
int eval_post(p3m_ctx *c, double kfac, double *sr_only_out, bool from_table, bool pairs)
{
    const double *kfac_dev = from_table ? c->cur_fac + 2 : nullptr;
    if (c->short_range && !pairs) {  // mesh part only (cells, sorted state, mesh fields)
        Phase ph(c, PH_GATHER);
        CK(launch_gather(c, c->acc_lr));
    } else if (c->short_range) {
        {
            Phase ph(c, PH_GATHER);
            CK(launch_gather(c, c->acc_lr));
        }
        Phase ph(c, PH_PAIRS);
        if (sr_only_out) {
            CK(launch_pairs(c, nullptr, sr_only_out, 0.0));
        } else {
            CK(launch_pairs(c, c->acc_lr, c->acc, kfac, kfac_dev));
        }
    } else {
        // pure PM: the mesh part is the whole force
        {
            Phase ph(c, PH_GATHER);
            CK(launch_gather(c, sr_only_out ? c->acc_lr : c->acc));
        }
        if (sr_only_out) CK(cudaMemsetAsync(sr_only_out, 0, 3 * sizeof(double) * c->g.n, c->stream));
        if (kfac != 0.0 || kfac_dev) {
            Phase ph(c, PH_OTHER);
            CK(launch_kick(c, kfac, kfac_dev));
        }
    }
    return P3M_OK;
}

int evaluate(p3m_ctx *c, double kfac, double *sr_only_out, bool from_table, bool pairs)
{
    int rc = eval_pre(c);
    if (!rc) rc = eval_r2c(c);
    if (!rc) rc = eval_kspace(c);
    if (!rc) rc = eval_c2r(c);
    if (!rc) rc = eval_post(c, kfac, sr_only_out, from_table, pairs);
    return rc;
}

int key_current(p3m_ctx *c)
{
    Phase ph(c, PH_KICK_DRIFT);
    CK(launch_kick_drift_keys(c, false, 0.0, 0.0));
    return P3M_OK;
}

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

// First part of a kick-drift-kick step a -> a + da: the step's factors (host arguments, or the
// device table for graph-replayed steps), the first half kick and the drift with the new keys.
// Returns the second half kick's factor in *k2 (0 when it comes from the table).
int step_kd(p3m_ctx *c, double a, double da, bool from_table, double *k2)
{
    double k1 = 0.0, dfac = 0.0;
    *k2 = 0.0;
    if (from_table) {
        CK(launch_step_begin(c));
    } else {
        const double am = a + 0.5 * da, a2 = a + da;
        k1 = c->mass * p3m_kick_factor(c->cosmo, a, am);
        dfac = p3m_drift_factor(c->cosmo, a, a2) / c->mass;
        *k2 = c->mass * p3m_kick_factor(c->cosmo, am, a2);
    }
    Phase ph(c, PH_KICK_DRIFT);
    CK(launch_kick_drift_keys(c, true, k1, dfac, from_table));
    return P3M_OK;
}

// Last part of a step: the Layzer-Irvine bookkeeping of a context that tracks its energy.
int step_tail(p3m_ctx *c, double a, double da, bool from_table)
{
    if (c->track_energy) {
        Phase ph(c, PH_OTHER);
        CK(launch_li_update(c, from_table ? c->cur_fac + 3 : nullptr, a + da));
    }
    return P3M_OK;
}

// One kick-drift-kick step a -> a + da with valid forces at a.  from_table: the step's factors
// come from the device table (graph-replayed steps; a and da unused).
int step_body(p3m_ctx *c, double a, double da, bool from_table)
{
    double k2 = 0.0;
    int rc = step_kd(c, a, da, from_table, &k2);
    if (!rc) rc = evaluate(c, k2, nullptr, from_table);
    if (!rc) rc = step_tail(c, a, da, from_table);
    return rc;
}

// The part of a step that precedes the pair sum, for a context whose pair sum runs in the
// ensemble's batched launch: kick-drift, sort, mesh force, then its pair arguments into
// *desc and its cost-sorted work list into the merged arrays gk/gv (slot `slot`).
int step_pre(p3m_ctx *c, double a, double da, bool from_table, int slot, PairArgs *desc,
             uint32_t *gk, uint32_t *gv)
{
    double k1 = 0.0, dfac = 0.0, k2 = 0.0;
    if (from_table) {
        CK(launch_step_begin(c));
    } else {
        const double am = a + 0.5 * da, a2 = a + da;
        k1 = c->mass * p3m_kick_factor(c->cosmo, a, am);
        dfac = p3m_drift_factor(c->cosmo, a, a2) / c->mass;
        k2 = c->mass * p3m_kick_factor(c->cosmo, am, a2);
    }
    {
        Phase ph(c, PH_KICK_DRIFT);
        CK(launch_kick_drift_keys(c, true, k1, dfac, from_table));
    }
    int rc = evaluate(c, k2, nullptr, from_table, false);
    if (rc) return rc;
    CK(cudaMemsetAsync(c->pair_count, 0, sizeof(unsigned long long), c->stream));
    c->launches += 2;
    CK(launch_store_pair_args(desc, pair_args(c, c->acc_lr, c->acc, k2, from_table ? c->cur_fac + 2 : nullptr),
                              c->stream));
    CK(launch_ens_gather(slot, c->work_key, c->work_order, c->max_work, gk, gv, c->stream));
    return P3M_OK;
}

PtrState save_ptrs(const p3m_ctx *c)
{
    return PtrState{c->pos,      c->mom,      c->pos_alt,  c->mom_alt,      c->pid,
                    c->pid_alt,  c->keys,     c->keys_alt, c->vals,         c->vals_alt,
                    c->work_key, c->work_key_alt, c->work_order, c->work_order_alt};
}

void load_ptrs(p3m_ctx *c, const PtrState &s)
{
    c->pos = s.pos;
    c->mom = s.mom;
    c->pos_alt = s.pos_alt;
    c->mom_alt = s.mom_alt;
    c->pid = s.pid;
    c->pid_alt = s.pid_alt;
    c->keys = s.keys;
    c->keys_alt = s.keys_alt;
    c->vals = s.vals;
    c->vals_alt = s.vals_alt;
    c->work_key = s.work_key;
    c->work_key_alt = s.work_key_alt;
    c->work_order = s.work_order;
    c->work_order_alt = s.work_order_alt;
}

}  // namespace p3m_host

using namespace p3m_host;

int p3m_fail_global(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_init_err, sizeof(g_init_err), fmt, ap);
    va_end(ap);
    return code;
}

// ---------------------------------------------------------------- host cosmology helpers

double p3m_kick_factor(const p3m_cosmology &cs, double a1, double a2)
{
    if (is_eds(cs)) return 2.0 * (sqrt(a2) - sqrt(a1));
    return quad(cs, a1, a2, 2);
}

double p3m_drift_factor(const p3m_cosmology &cs, double a1, double a2)
{
    if (is_eds(cs)) return 2.0 * (1.0 / sqrt(a1) - 1.0 / sqrt(a2));
    return quad(cs, a1, a2, 3);
}

// ---------------------------------------------------------------- ABI

extern "C" int p3m_default_options(p3m_options *opt)
{
    if (!opt) return P3M_EINVAL;
    opt->precision = P3M_PREC_MIXED;
    opt->softening = 0.02;
    opt->deconvolve_cic = 1;
    opt->short_range = 1;
    opt->sub_bits = 3;
    opt->stream = nullptr;
    return P3M_OK;
}

extern "C" int p3m_init(p3m_ctx **out, double box, int64_t n, int mesh, double r_s_cells,
                        double cutoff_in_rs, const p3m_cosmology *cosmo, const p3m_options *opt_in)
{
    p3m_ctx *c = nullptr;
    if (!out) return fail(c, P3M_EINVAL, "p3m_init: ctx pointer is NULL");
    *out = nullptr;
    p3m_options opt;
    p3m_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.sub_bits < 0) opt.sub_bits = 3;
    p3m_cosmology cs = {1.0, 0.0, 100.0};
    if (cosmo) cs = *cosmo;

    if (!finite_pos(box)) return fail(c, P3M_EINVAL, "p3m_init: box must be finite and > 0");
    if (n < 1 || n >= (int64_t)1 << 31) return fail(c, P3M_EINVAL, "p3m_init: n must be in [1, 2^31)");
    if (mesh < 8 || mesh > 2048 || (mesh & 1))
        return fail(c, P3M_EINVAL, "p3m_init: mesh must be even and in [8, 2048]");
    if (!finite_pos(r_s_cells)) return fail(c, P3M_EINVAL, "p3m_init: r_s_cells must be > 0");
    if (!finite_pos(cutoff_in_rs)) return fail(c, P3M_EINVAL, "p3m_init: cutoff_in_rs must be > 0");
    if (opt.precision != P3M_PREC_MIXED && opt.precision != P3M_PREC_FP64)
        return fail(c, P3M_EINVAL, "p3m_init: unknown precision mode");
    if (!(opt.softening >= 0.0) || !isfinite(opt.softening))
        return fail(c, P3M_EINVAL, "p3m_init: softening must be >= 0");
    if (opt.sub_bits > 5) return fail(c, P3M_EINVAL, "p3m_init: sub_bits must be in 0..5");
    if (!finite_pos(cs.omega_m) || !(cs.omega_lambda >= 0.0) || !isfinite(cs.omega_lambda))
        return fail(c, P3M_EINVAL, "p3m_init: need omega_m > 0 and omega_lambda >= 0");

    P3MGeom g;
    memset(&g, 0, sizeof(g));
    g.box = box;
    g.n = n;
    g.mesh = mesh;
    g.inv_h = (double)mesh / box;
    g.r_s = r_s_cells * (box / mesh);
    g.r_c = cutoff_in_rs * (r_s_cells * (box / mesh));
    g.eps = opt.softening * (box / cbrt((double)n));
    g.gm = 3.0 * cs.omega_m * pow(box, 3.0) / (8.0 * M_PI * (double)n);
    if (opt.short_range) {
        const double ncd = floor(box / g.r_c);
        if (ncd < 3.0)
            return fail(c, P3M_EINVAL,
                        "p3m_init: box/r_c = %.4g: need at least 3 chaining cells per side", box / g.r_c);
        if (ncd > 1024.0) return fail(c, P3M_EINVAL, "p3m_init: more than 1024 chaining cells per side");
        g.n_c = (int)ncd;
    } else {
        g.n_c = mesh / 6 < 3 ? 3 : (mesh / 6 > 1024 ? 1024 : mesh / 6);
    }
    g.sub_bits = opt.sub_bits;
    g.n_fine = g.n_c << g.sub_bits;
    g.inv_fine = (double)g.n_fine / box;
    g.cs = box / g.n_c;
    g.n_cells = g.n_c * g.n_c * g.n_c;
    g.mean_count = (double)n / ((double)mesh * mesh * mesh);
    int key_bits = 0;
    {
        const uint64_t max_key = ((uint64_t)g.n_cells << (3 * g.sub_bits)) - 1;
        if (max_key >= (1ull << 32)) return fail(c, P3M_EINVAL, "p3m_init: sort key exceeds 32 bits");
        while (key_bits < 32 && (max_key >> key_bits)) ++key_bits;
        if (key_bits == 0) key_bits = 1;
    }

    c = (p3m_ctx *)calloc(1, sizeof(p3m_ctx));
    if (!c) return fail(nullptr, P3M_ENOMEM, "p3m_init: host allocation failed");
    c->g = g;
    c->precision = opt.precision;
    c->tile_blocks = 5;
    c->deconvolve = opt.deconvolve_cic ? 1 : 0;
    c->short_range = opt.short_range ? 1 : 0;
    c->cosmo = cs;
    c->mass = 1.0;
    c->a = 1.0;
    c->stream = (cudaStream_t)opt.stream;
    c->key_bits = key_bits;
    c->sort_wait_limit = 1ll << 31;
    c->fac_cap = P3M_MAX_GRAPH_STEPS;
    strcpy(c->err, "no error");

    int rc = P3M_OK;
    do {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->l2_bytes, cudaDevAttrL2CacheSize, dev);
        if (e == cudaSuccess) e = mesh_set_attributes();
        if (e != cudaSuccess) {
            rc = fail(nullptr, P3M_ECUDA, "p3m_init: no CUDA device: %s", cudaGetErrorString(e));
            break;
        }
        const size_t N = (size_t)n, M = (size_t)mesh, nk = M * M * (M / 2 + 1), M3 = M * M * M;
        const size_t real = c->precision == P3M_PREC_MIXED ? 4 : 8;
        c->max_work = N / P3M_PAIR_TI + (size_t)g.n_cells + 1;
        const size_t nsort = N > c->max_work ? N : c->max_work;  // longest array the sorts see
        c->n_tiles = (int)((nsort + P3M_SORT_TILE - 1) / P3M_SORT_TILE);
        const size_t scan_n = (size_t)256 * c->n_tiles > (size_t)g.n_cells + 1 ? (size_t)256 * c->n_tiles
                                                                               : (size_t)g.n_cells + 1;
        struct {
            void **p;
            size_t bytes;
        } allocs[] = {
            {(void **)&c->pos, 24 * N},       {(void **)&c->mom, 24 * N},
            {(void **)&c->acc, 24 * N},       {(void **)&c->acc_lr, 24 * N},
            {(void **)&c->pos_alt, 24 * N},   {(void **)&c->mom_alt, 24 * N},
            {(void **)&c->pid, 4 * N},        {(void **)&c->pid_alt, 4 * N},
            {(void **)&c->rel, 4 * real * N}, {(void **)&c->keys, 4 * N},
            {(void **)&c->block_box, 32 * ((N + 31) / 32)},
            {(void **)&c->relx, opt.precision == P3M_PREC_MIXED ? 384 * ((N + 31) / 32) : 16},
            {(void **)&c->keys_alt, 4 * N},   {(void **)&c->vals, 4 * N},
            {(void **)&c->vals_alt, 4 * N},   {(void **)&c->digit_counts, 4 * 256 * (size_t)c->n_tiles},
            {(void **)&c->scan_aux, 4 * (scan_n / P3M_SORT_TILE + 4)},
            {(void **)&c->sort_status, 8 * 256 * (size_t)c->n_tiles},
            {(void **)&c->sort_hist, 4 * (4 * 256 + 4)},
            {(void **)&c->cell_start, 4 * ((size_t)g.n_cells + 1)},
            {(void **)&c->work, 8 * c->max_work}, {(void **)&c->work_off, 4 * ((size_t)g.n_cells + 1)},
            {(void **)&c->work_key, 4 * c->max_work}, {(void **)&c->work_key_alt, 4 * c->max_work},
            {(void **)&c->work_order, 4 * c->max_work}, {(void **)&c->work_order_alt, 4 * c->max_work},
            {(void **)&c->counters, 16},      {(void **)&c->pair_count, 64},
            {(void **)&c->red, 8 * (1024 * 4 + 8)},
            {(void **)&c->rho, real * M3},    {(void **)&c->rho_k, 2 * real * nk},
            {(void **)&c->frc_k, 6 * real * nk}, {(void **)&c->frc, 3 * real * M3},
            {(void **)&c->tab_k, real * M},   {(void **)&c->tab_kg, real * M},
            {(void **)&c->tab_g, real * M},   {(void **)&c->tab_invw2, 8 * M},
            {(void **)&c->tab_one, 8 * M},    {(void **)&c->ps_acc, 8 * (3 * (M / 2) + 1)},
            {(void **)&c->ps_part, 8 * (3 * (M / 2) + 1) * (size_t)(2 * c->num_sms)},
            {(void **)&c->rho_fix, 8 * 3 * M3}, {(void **)&c->fix_exp, 16},
            {(void **)&c->tab_origin, 8 * (size_t)g.n_c},
            {(void **)&c->fac_table, 8 * 4 * (size_t)P3M_MAX_GRAPH_STEPS},
            {(void **)&c->step_idx, 16},      {(void **)&c->cur_fac, 32},
            {(void **)&c->kself, 8 * 27},     {(void **)&c->li, 8 * 4},
            {(void **)&c->adj_u, 3 * real * M3}, {(void **)&c->adj_vfx, opt.precision == P3M_PREC_MIXED ? 384 * ((N + 31) / 32) : 16},
            {(void **)&c->adj_vs, 24 * N},    {(void **)&c->adj_out, 24 * N},
        };
        int idx = 0;
        for (auto &a : allocs) {
            const bool injected = idx++ == g_inject_alloc;
            e = injected ? cudaErrorMemoryAllocation : dalloc(a.p, a.bytes, c);
            if (e != cudaSuccess) {
                rc = fail(nullptr, P3M_ENOMEM, "p3m_init: cudaMalloc of %zu bytes failed: %s%s", a.bytes,
                          cudaGetErrorString(e), injected ? " (injected)" : "");
                break;
            }
        }
        if (rc != P3M_OK) break;
        c->g.flags = c->counters + 1;
        cudaMemsetAsync(c->counters, 0, 16, c->stream);
        cudaMemsetAsync(c->pair_count, 0, 64, c->stream);
        // sort buffers start at zero: every key and slot they ever hold is then in range
        cudaMemsetAsync(c->keys_alt, 0, 4 * N, c->stream);
        cudaMemsetAsync(c->vals, 0, 4 * N, c->stream);
        cudaMemsetAsync(c->vals_alt, 0, 4 * N, c->stream);
        c->ps_blocks = 2 * c->num_sms;
        if (opt.precision == P3M_PREC_MIXED)  // padding past the last particle stays zero
            cudaMemsetAsync(c->adj_vfx, 0, 384 * ((N + 31) / 32), c->stream);

        // per-axis tables (FP64 on the host, stored in the mesh precision)
        const double h = box / mesh, rs2 = c->short_range ? g.r_s * g.r_s : 0.0;
        std::vector<double> tk(M), tkg(M), tg(M);
        for (int i = 0; i < mesh; ++i) {
            const int m = i <= mesh / 2 ? i : i - mesh;
            const double k = 2.0 * M_PI / box * m;
            tk[i] = k;
            tkg[i] = (i == mesh / 2) ? 0.0 : k;
            double t = exp(-k * k * rs2);
            if (c->deconvolve) {
                const double x = 0.5 * k * h;
                const double s = x == 0.0 ? 1.0 : sin(x) / x;
                t /= (s * s) * (s * s);
            }
            tg[i] = t;
        }
        c->green_const = -4.0 * M_PI * (g.gm / (h * h * h)) / ((double)M3);
        fit_split_poly(cutoff_in_rs, g.r_s, c->gpoly);
        fit_split_poly64(cutoff_in_rs, g.r_s, c->gpoly64);
        if (c->precision == P3M_PREC_MIXED) {
            std::vector<float> f(M);
            const std::vector<double> *src[3] = {&tk, &tkg, &tg};
            void *dst[3] = {c->tab_k, c->tab_kg, c->tab_g};
            for (int t = 0; t < 3; ++t) {
                for (size_t i = 0; i < M; ++i) f[i] = (float)(*src[t])[i];
                e = cudaMemcpy(dst[t], f.data(), 4 * M, cudaMemcpyHostToDevice);
                if (e != cudaSuccess) break;
            }
        } else {
            e = cudaMemcpy(c->tab_k, tk.data(), 8 * M, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(c->tab_kg, tkg.data(), 8 * M, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(c->tab_g, tg.data(), 8 * M, cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) {
            std::vector<double> w2(M), one(M, 1.0);
            for (int i = 0; i < mesh; ++i) {
                const double x = 0.5 * tk[i] * h;
                const double s = x == 0.0 ? 1.0 : sin(x) / x;
                w2[i] = 1.0 / ((s * s) * (s * s));
            }
            e = cudaMemcpy(c->tab_invw2, w2.data(), 8 * M, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(c->tab_one, one.data(), 8 * M, cudaMemcpyHostToDevice);
            std::vector<double> org(g.n_c);
            for (int q = 0; q < g.n_c; ++q) org[q] = (double)q * g.cs;
            if (e == cudaSuccess)
                e = cudaMemcpy(c->tab_origin, org.data(), 8 * (size_t)g.n_c, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            rc = fail(nullptr, P3M_ECUDA, "p3m_init: table upload failed: %s", cudaGetErrorString(e));
            break;
        }

        // cuFFT: one R2C, and the three C2R as one batch of 3 (default layouts)
        int dims[3] = {mesh, mesh, mesh};
        cufftResult r = g_inject_fft ? CUFFT_ALLOC_FAILED
                                     : cufftPlan3d(&c->plan_r2c, mesh, mesh, mesh,
                                                   c->precision == P3M_PREC_MIXED ? CUFFT_R2C : CUFFT_D2Z);
        if (r == CUFFT_SUCCESS) {
            r = cufftPlanMany(&c->plan_c2r, 3, dims, nullptr, 1, (int)nk, nullptr, 1, (int)M3,
                              c->precision == P3M_PREC_MIXED ? CUFFT_C2R : CUFFT_Z2D, 3);
            if (r != CUFFT_SUCCESS) cufftDestroy(c->plan_r2c);
        }
        if (r == CUFFT_SUCCESS) {
            r = cufftPlan3d(&c->plan_c2r_one, mesh, mesh, mesh,
                            c->precision == P3M_PREC_MIXED ? CUFFT_C2R : CUFFT_Z2D);
            if (r != CUFFT_SUCCESS) {
                cufftDestroy(c->plan_r2c);
                cufftDestroy(c->plan_c2r);
            }
        }
        if (r != CUFFT_SUCCESS) {
            rc = fail(nullptr, P3M_ECUFFT, "p3m_init: cuFFT plan creation failed (code %d)%s", (int)r,
                      g_inject_fft ? " (injected)" : "");
            break;
        }
        c->plans_made = true;
        cufftSetStream(c->plan_r2c, c->stream);
        cufftSetStream(c->plan_c2r, c->stream);
        cufftSetStream(c->plan_c2r_one, c->stream);
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            rc = fail(nullptr, P3M_ECUDA, "p3m_init: %s", cudaGetErrorString(e));
            break;
        }
    } while (0);
    if (rc != P3M_OK) {
        release(c);
        free(c);
        return rc;
    }
    *out = c;
    return P3M_OK;
}

namespace {

// The device address of page-locked (pinned) host memory, or NULL for any other pointer: the
// kernels then read or write it directly over the CPU-GPU link instead of staging it through
// a separate copy.
const void *pinned_view(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // older runtimes report unregistered memory as an error
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

}  // namespace

extern "C" int p3m_set_particles(p3m_ctx *c, const double *pos, const double *mom,
                                 const double *acc, double mass, double a, int on_device)
{
    Range nvtx_range("p3m_set_particles");
    if (!c) return fail(c, P3M_EINVAL, "ctx is NULL");
    if (!pos || !mom) return fail(c, P3M_EINVAL, "p3m_set_particles: pos and mom are required");
    if (!finite_pos(mass)) return fail(c, P3M_EINVAL, "p3m_set_particles: mass must be > 0");
    if (!finite_pos(a)) return fail(c, P3M_EINVAL, "p3m_set_particles: a must be > 0");
    const size_t bytes = 3 * sizeof(double) * (size_t)c->g.n;
    CK(cudaMemsetAsync(c->counters + 1, 0, sizeof(uint32_t), c->stream));
    const double *sp = pos, *sm = mom, *sa = acc;
    if (!on_device) {  // pinned host arrays are read in place; others are copied first
        const double *src[3] = {pos, mom, acc};
        double *stage[3] = {c->pos_alt, c->mom_alt, c->acc_lr};
        const double *use[3] = {nullptr, nullptr, nullptr};
        for (int t = 0; t < 3; ++t) {
            if (!src[t]) continue;
            use[t] = (const double *)pinned_view(src[t]);
            if (!use[t]) {
                CK(cudaMemcpyAsync(stage[t], src[t], bytes, cudaMemcpyHostToDevice, c->stream));
                use[t] = stage[t];
            }
        }
        sp = use[0];
        sm = use[1];
        sa = use[2];
    }
    CK(launch_load_particles(c, sp, sm, sa));
    uint32_t flags = 0;
    CK(cudaMemcpyAsync(&flags, c->counters + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->have_particles = false;
    c->forces_valid = false;
    c->sorted_valid = false;
    if (flags & P3M_FLAG_NONFINITE) {
        cudaMemsetAsync(c->counters + 1, 0, sizeof(uint32_t), c->stream);
        return fail(c, P3M_ENONFINITE, "p3m_set_particles: NaN or Inf in the input");
    }
    c->mass = mass;
    c->a = a;
    c->have_particles = true;
    c->forces_valid = acc != nullptr;
    return P3M_OK;
}

extern "C" int p3m_forces(p3m_ctx *c, double a, double *acc3n, int on_device)
{
    Range nvtx_range("p3m_forces");
    if (!c) return fail(c, P3M_EINVAL, "ctx is NULL");
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_forces: no particles loaded");
    if (!finite_pos(a)) return fail(c, P3M_EINVAL, "p3m_forces: a must be > 0");
    int rc = key_current(c);
    if (rc) return rc;
    rc = evaluate(c, 0.0, nullptr);
    if (rc) return rc;
    c->forces_valid = true;
    c->a = a;
    if (acc3n) return p3m_get_particles(c, nullptr, nullptr, acc3n, on_device);
    return P3M_OK;
}

extern "C" int p3m_forces_split(p3m_ctx *c, double *acc_lr, double *acc_sr, int on_device)
{
    if (!c) return fail(c, P3M_EINVAL, "ctx is NULL");
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_forces_split: no particles loaded");
    int rc = key_current(c);
    if (rc) return rc;
    rc = evaluate(c, 0.0, c->acc);  // c->acc = short-range part only
    if (rc) return rc;
    const size_t bytes = 3 * sizeof(double) * (size_t)c->g.n;
    double *outs[2] = {acc_lr, acc_sr};
    const double *srcs[2] = {c->acc_lr, c->acc};
    for (int t = 0; t < 2; ++t) {
        if (!outs[t]) continue;
        if (on_device) {
            CK(launch_scatter_out(c, srcs[t], outs[t]));
        } else {
            CK(launch_scatter_out(c, srcs[t], c->pos_alt));
            CK(cudaMemcpyAsync(outs[t], c->pos_alt, bytes, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
    }
    CK(launch_axpy(c, c->acc, c->acc_lr, 1.0));  // total
    c->forces_valid = true;
    return check_flags(c);
}

extern "C" int p3m_step(p3m_ctx *c, double a, double da)
{
    Range nvtx_range("p3m_step");
    if (!c) return fail(c, P3M_EINVAL, "ctx is NULL");
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_step: no particles loaded");
    if (!finite_pos(a) || !finite_pos(da)) return fail(c, P3M_EINVAL, "p3m_step: need a > 0, da > 0");
    int rc;
    if (!c->forces_valid) {
        rc = key_current(c);
        if (rc) return rc;
        rc = evaluate(c, 0.0, nullptr);
        if (rc) return rc;
        c->forces_valid = true;
    }
    rc = step_body(c, a, da, false);
    if (rc) return rc;
    c->a = a + da;
    return P3M_OK;
}

extern "C" int p3m_power_spectrum(p3m_ctx *c, int n_bins, int deconvolve, double tophat_radius,
                                  double *k_mean, double *power, double *n_modes, double *sigma)
{
    Range nvtx_range("p3m_power_spectrum");
    if (!c) return fail(c, P3M_EINVAL, "ctx is NULL");
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_power_spectrum: no particles loaded");
    const int nb_max = c->g.mesh / 2;
    if (n_bins < 1 || n_bins > nb_max)
        return fail(c, P3M_EINVAL, "p3m_power_spectrum: n_bins must be in [1, %d]", nb_max);
    if (!(tophat_radius >= 0.0) || !isfinite(tophat_radius))
        return fail(c, P3M_EINVAL, "p3m_power_spectrum: tophat_radius must be >= 0");
    CK(launch_deposit(c));
    CKF(c->precision == P3M_PREC_MIXED
            ? cufftExecR2C(c->plan_r2c, (cufftReal *)c->rho, (cufftComplex *)c->rho_k)
            : cufftExecD2Z(c->plan_r2c, (cufftDoubleReal *)c->rho, (cufftDoubleComplex *)c->rho_k));
    CK(launch_powspec(c, deconvolve ? c->tab_invw2 : c->tab_one, sigma ? tophat_radius : 0.0, n_bins,
                      c->ps_acc));
    std::vector<double> h(3 * (size_t)n_bins + 1);
    CK(cudaMemcpyAsync(h.data(), c->ps_acc, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double L3 = c->g.box * c->g.box * c->g.box;
    for (int b = 0; b < n_bins; ++b) {
        const double cnt = h[3 * b + 2];
        if (k_mean) k_mean[b] = cnt > 0 ? h[3 * b + 1] / cnt : NAN;
        if (power) power[b] = cnt > 0 ? L3 * h[3 * b] / cnt : NAN;
        if (n_modes) n_modes[b] = cnt;
    }
    if (sigma) *sigma = tophat_radius > 0.0 ? sqrt(h[3 * n_bins]) : NAN;
    return P3M_OK;
}

extern "C" int p3m_get_particles(p3m_ctx *c, double *pos, double *mom, double *acc, int on_device)
{
    Range nvtx_range("p3m_get_particles");
    if (!c) return fail(c, P3M_EINVAL, "ctx is NULL");
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_get_particles: no particles loaded");
    if (acc && !c->forces_valid) return fail(c, P3M_ESTATE, "p3m_get_particles: forces not evaluated");
    const size_t bytes = 3 * sizeof(double) * (size_t)c->g.n;
    double *outs[3] = {pos, mom, acc};
    const double *srcs[3] = {c->pos, c->mom, c->acc};
    bool inv_ready = false;  // pid_alt is free between sorts: the inverse permutation
    for (int t = 0; t < 3; ++t) {
        if (!outs[t]) continue;
        double *direct = on_device ? nullptr : (double *)pinned_view(outs[t]);
        if (on_device) {
            CK(launch_scatter_out(c, srcs[t], outs[t]));
        } else if (direct) {  // pinned host array: written in place, sequentially
            if (!inv_ready) CK(launch_inverse_pid(c, c->pid_alt));
            inv_ready = true;
            CK(launch_gather_out(c, srcs[t], c->pid_alt, direct));
        } else {
            double *stage = t == 0 ? c->pos_alt : (t == 1 ? c->mom_alt : c->acc_lr);
            CK(launch_scatter_out(c, srcs[t], stage));
            CK(cudaMemcpyAsync(outs[t], stage, bytes, cudaMemcpyDeviceToHost, c->stream));
        }
    }
    if (!on_device) return check_flags(c);
    return P3M_OK;
}

extern "C" int p3m_diagnostics(p3m_ctx *c, p3m_diag *out)
{
    if (!c || !out) return fail(c, P3M_EINVAL, "p3m_diagnostics: NULL argument");
    memset(out, 0, sizeof(*out));
    out->potential = NAN;
    out->layzer_irvine = NAN;
    out->a = c->a;
    out->n = c->g.n;
    out->n_cells_side = c->g.n_c;
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_diagnostics: no particles loaded");
    if (c->track_energy) {
        double kin = 0.0, pot = 0.0, li[4];
        int rc = energy_now(c, &kin, &pot);
        if (rc) return rc;
        CK(cudaMemcpy(li, c->li, sizeof(li), cudaMemcpyDeviceToHost));
        out->potential = pot;
        out->layzer_irvine = c->a * (kin + pot) + li[0] - c->li_e0;
    }
    double r[4];
    CK(launch_diag(c, r));
    out->momentum[0] = r[0];
    out->momentum[1] = r[1];
    out->momentum[2] = r[2];
    out->kinetic = r[3] / (2.0 * c->mass * c->a * c->a);
    unsigned long long pc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t mc = 0;
    CK(cudaMemcpy(pc, c->pair_count, sizeof(pc), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&mc, c->counters + 2, sizeof(mc), cudaMemcpyDeviceToHost));
    out->pairs = pc[0];
    out->pairs_total = pc[1];
    out->pair_warp_j[0] = pc[2];
    out->pair_warp_j[1] = pc[3];
    out->pair_warp_j[2] = pc[4];
    out->pair_blocks_culled = pc[5];
    out->pair_tiles[0] = pc[6];
    out->pair_tiles[1] = pc[7];
    out->launches = c->launches;
    out->max_cell_count = (int32_t)mc;
    return check_flags(c);
}

extern "C" int p3m_get_cells(p3m_ctx *c, uint32_t *keys, uint32_t *ids, uint32_t *cell_start,
                             int on_device)
{
    if (!c) return fail(c, P3M_EINVAL, "ctx is NULL");
    if (!c->sorted_valid) return fail(c, P3M_ESTATE, "p3m_get_cells: nothing sorted yet");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t n = (size_t)c->g.n;
    if (keys) CK(cudaMemcpyAsync(keys, c->keys, 4 * n, kind, c->stream));
    if (ids) CK(cudaMemcpyAsync(ids, c->pid, 4 * n, kind, c->stream));
    if (cell_start)
        CK(cudaMemcpyAsync(cell_start, c->cell_start, 4 * ((size_t)c->g.n_cells + 1), kind, c->stream));
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    return P3M_OK;
}

extern "C" int p3m_get_mesh(p3m_ctx *c, int which, void *out, int on_device)
{
    if (!c || !out) return fail(c, P3M_EINVAL, "p3m_get_mesh: NULL argument");
    if (which < 0 || which > 3) return fail(c, P3M_EINVAL, "p3m_get_mesh: which must be 0..3");
    if (!c->sorted_valid) return fail(c, P3M_ESTATE, "p3m_get_mesh: no force evaluation yet");
    const size_t M3 = (size_t)c->g.mesh * c->g.mesh * c->g.mesh;
    const size_t real = c->precision == P3M_PREC_MIXED ? 4 : 8;
    const char *src = which == 0 ? (const char *)c->rho : (const char *)c->frc + (which - 1) * M3 * real;
    CK(cudaMemcpyAsync(out, src, M3 * real, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream));
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    return P3M_OK;
}

extern "C" int p3m_get_geometry(const p3m_ctx *c, int *n_c, int *mesh, int *precision, int *sub_bits)
{
    if (!c) return P3M_EINVAL;
    if (n_c) *n_c = c->g.n_c;
    if (mesh) *mesh = c->g.mesh;
    if (precision) *precision = c->precision;
    if (sub_bits) *sub_bits = c->g.sub_bits;
    return P3M_OK;
}

extern "C" int p3m_set_timing(p3m_ctx *c, int enable)
{
    if (!c) return P3M_EINVAL;
    if (enable && !c->ev) {
        c->ev_cap = 8192;
        c->ev = (cudaEvent_t *)calloc(c->ev_cap, sizeof(cudaEvent_t));
        c->ev_phase = (int *)calloc(c->ev_cap, sizeof(int));
        if (!c->ev || !c->ev_phase) return fail(c, P3M_ENOMEM, "p3m_set_timing: host allocation failed");
        for (int i = 0; i < c->ev_cap; ++i) CK(cudaEventCreate(&c->ev[i]));
    }
    if (!enable && c->ev) harvest(c);
    c->timing = enable != 0;
    return P3M_OK;
}

extern "C" int p3m_timings(p3m_ctx *c, double *ms, int n, int reset)
{
    if (!c) return P3M_EINVAL;
    harvest(c);
    for (int i = 0; i < n && i < P3M_NPHASES; ++i) ms[i] = c->phase_ms[i];
    if (reset)
        for (int i = 0; i < P3M_NPHASES; ++i) c->phase_ms[i] = 0.0;
    return P3M_NPHASES;
}

extern "C" const char *p3m_phase_name(int i)
{
    return (i >= 0 && i < P3M_NPHASES) ? kPhaseNames[i] : nullptr;
}

extern "C" const char *p3m_last_error(const p3m_ctx *c) { return c ? c->err : g_init_err; }

extern "C" void p3m_free(p3m_ctx *c)
{
    if (!c) return;
    if (c->self_ens) p3m_ensemble_free(c->self_ens);
    cudaStreamSynchronize(c->stream);
    release(c);
    free(c);
}


extern "C" int p3m_inject_fault(p3m_ctx *c, int what, int64_t arg)
{
    switch (what) {
    case P3M_INJECT_NONE:
        g_inject_alloc = -1;
        g_inject_fft = false;
        if (c) {
            if (c->sort_probe) {
                CK(cudaStreamSynchronize(c->stream));
                CK(cudaFree(c->sort_probe));
            }
            c->sort_probe = nullptr;
            c->sort_wait_limit = 1ll << 31;
        }
        return P3M_OK;
    case P3M_INJECT_ALLOC:
        if (arg < 0) return fail(c, P3M_EINVAL, "p3m_inject_fault: allocation index must be >= 0");
        g_inject_alloc = (int)arg;
        return P3M_OK;
    case P3M_INJECT_FFT_PLAN:
        g_inject_fft = true;
        return P3M_OK;
    case P3M_INJECT_SORT_TIMEOUT: {
        if (!c) return fail(c, P3M_EINVAL, "p3m_inject_fault: the sort timeout needs a context");
        if (arg < 1 || arg > (1ll << 31)) return fail(c, P3M_EINVAL, "p3m_inject_fault: wait limit out of range");
        if (!c->sort_probe) {
            const size_t bytes = sizeof(unsigned long long) * 256 * (size_t)c->n_tiles;
            CK(cudaMalloc((void **)&c->sort_probe, bytes));
            CK(cudaMemset(c->sort_probe, 0, bytes));
        }
        c->sort_wait_limit = (long long)arg;
        return P3M_OK;
    }
    default:
        return fail(c, P3M_EINVAL, "p3m_inject_fault: unknown fault %d", what);
    }
}

extern "C" int p3m_debug_check(p3m_ctx *c)
{
    if (!c) return fail(c, P3M_EINVAL, "p3m_debug_check: ctx is NULL");
    const int rc = check_flags(c);
    if (rc) return rc;
#ifdef P3M_DEBUG_CHECKS
    unsigned char guard[kCanaryBytes];
    for (int k = 0; k < c->n_canary; ++k) {
        CK(cudaMemcpy(guard, (const char *)c->canary_ptr[k] + c->canary_off[k], kCanaryBytes,
                      cudaMemcpyDeviceToHost));
        for (size_t b = 0; b < kCanaryBytes; ++b)
            if (guard[b] != kCanary)
                return fail(c, P3M_EBOUNDS, "p3m_debug_check: guard bytes after allocation %d were "
                            "overwritten (byte %zu)", k, b);
    }
#endif
    return P3M_OK;
}

extern "C" int p3m_debug_poke_canary(p3m_ctx *c, int k)
{
    if (!c) return fail(c, P3M_EINVAL, "p3m_debug_poke_canary: ctx is NULL");
#ifdef P3M_DEBUG_CHECKS
    if (k < 0 || k >= c->n_canary) return fail(c, P3M_EINVAL, "p3m_debug_poke_canary: no allocation %d", k);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemset((char *)c->canary_ptr[k] + c->canary_off[k] + 17, 0, 1));
    return P3M_OK;
#else
    (void)k;
    return fail(c, P3M_ESTATE, "p3m_debug_poke_canary: not a debug build (P3M_DEBUG_CHECKS)");
#endif
}
