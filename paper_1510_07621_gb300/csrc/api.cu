// C ABI of the P3M library: argument checks, the context (all device memory and cuFFT plans
// allocated in p3m_init), and the order of the phases of a force evaluation and of a
// kick-drift-kick step.  Every kernel launch goes to the context's stream.
#include <cuda_runtime.h>
#include <cufft.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "p3m_internal.cuh"

namespace {

char g_init_err[512] = "no error";

int fail(p3m_ctx *c, int code, const char *fmt, ...)
{
    char *buf = c ? c->err : g_init_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(c, P3M_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
    } while (0)

#define CKF(call)                                                                           \
    do {                                                                                    \
        cufftResult r_ = (call);                                                            \
        if (r_ != CUFFT_SUCCESS) return fail(c, P3M_ECUFFT, "%s failed: cufft code %d", #call, (int)r_); \
    } while (0)

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
// g(x) = erfc(x/2) + x/sqrt(pi) exp(-x^2/4) = 1 + x^3 Q(x^2).  Q is smooth in u = x^2; it is
// interpolated at 40 Chebyshev-Gauss nodes of u in [0, u_c], u_c = (r_c/r_s)^2, truncated to
// degree P3M_SPLIT_DEG (a near-minimax polynomial), and rewritten in monomial form in tau = 2u/u_c - 1
// for Horner evaluation in FP32.  The kernel evaluates g = 1 + r^3 Q'(tau) directly from
// r^2, so the coefficients are scaled by r_s^-3 and tau = r^2 (2 / (u_c r_s^2)) - 1.

double split_q(double u)
{
    const double x = sqrt(u), inv_sqrt_pi = 0.56418958354775628695;
    if (u < 1e-6) return -inv_sqrt_pi / 6.0 * (1.0 - 0.15 * u);  // series: -(1/(6 sqrt pi))(1 - 3u/20)
    const double gval = erfc(0.5 * x) + x * inv_sqrt_pi * exp(-0.25 * u);
    return (gval - 1.0) / (u * x);
}

void fit_split_poly(double cutoff_in_rs, double r_s, float out[12])
{
    const int deg = P3M_SPLIT_DEG, nodes = 40;
    const double uc = cutoff_in_rs * cutoff_in_rs;
    double cheb[deg + 1] = {0};
    for (int j = 0; j < nodes; ++j) {
        const double th = M_PI * (j + 0.5) / nodes, t = cos(th);
        const double q = split_q(0.5 * (t + 1.0) * uc);
        for (int k = 0; k <= deg; ++k) cheb[k] += q * cos(k * th);
    }
    for (int k = 0; k <= deg; ++k) cheb[k] *= (k == 0 ? 1.0 : 2.0) / nodes;
    // Chebyshev series -> monomials: T_0 = 1, T_1 = t, T_{k+1} = 2 t T_k - T_{k-1}
    double tk_prev[deg + 1] = {0}, tk[deg + 1] = {0}, mono[deg + 1] = {0};
    tk_prev[0] = 1.0;
    tk[1] = 1.0;
    mono[0] += cheb[0];
    for (int i = 0; i <= deg; ++i) mono[i] += cheb[1] * tk[i];
    for (int k = 2; k <= deg; ++k) {
        double next[deg + 1] = {0};
        for (int i = 0; i <= deg; ++i) {
            next[i] = -tk_prev[i] + (i > 0 ? 2.0 * tk[i - 1] : 0.0);
        }
        for (int i = 0; i <= deg; ++i) {
            mono[i] += cheb[k] * next[i];
            tk_prev[i] = tk[i];
            tk[i] = next[i];
        }
    }
    const double inv_rs3 = 1.0 / (r_s * r_s * r_s);
    for (int i = 0; i <= deg; ++i) out[i] = (float)(mono[i] * inv_rs3);
    for (int i = deg + 1; i < 11; ++i) out[i] = 0.0f;
    out[11] = (float)(2.0 / (uc * r_s * r_s));
}

// ---------------------------------------------------------------- phase timing

struct Phase {
    p3m_ctx *c;
    int id;
    Phase(p3m_ctx *c_, int id_) : c(c_), id(id_)
    {
        if (c->timing && !c->capturing && c->ev_used + 2 <= c->ev_cap) {
            cudaEventRecord(c->ev[c->ev_used], c->stream);
            c->ev_phase[c->ev_used] = id;
        } else {
            id = -1;
        }
    }
    ~Phase()
    {
        if (id >= 0) {
            cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
            c->ev_phase[c->ev_used + 1] = id;
            c->ev_used += 2;
        }
    }
};

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
                    c->li,        c->relx};
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

template <typename T>
cudaError_t dalloc(T **p, size_t bytes)
{
    *p = nullptr;
    return cudaMalloc((void **)p, bytes < 16 ? 16 : bytes);
}

int check_flags(p3m_ctx *c)
{
    uint32_t flags = 0;
    CK(cudaMemcpyAsync(&flags, c->counters + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (flags & P3M_FLAG_TIMEOUT) return fail(c, P3M_ETIMEOUT, "a bounded device-side wait gave up");
    return P3M_OK;
}

// ---------------------------------------------------------------- force evaluation
// Sort by cell, mesh force, pair force.  Positions must already be wrapped and keyed
// (c->keys).  Result: c->acc (total), c->acc_lr (mesh part).  kfac != 0: the final half kick
// mom += kfac * acc is fused into the last kernel.
int evaluate(p3m_ctx *c, double kfac, double *sr_only_out, bool from_table = false,
             bool pairs = true)
{
    const double *kfac_dev = from_table ? c->cur_fac + 2 : nullptr;
    {
        Phase ph(c, PH_SORT);
        CK(launch_radix_sort(c));
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
    {
        Phase ph(c, PH_FFT_R2C);
        CKF(c->precision == P3M_PREC_MIXED
                ? cufftExecR2C(c->plan_r2c, (cufftReal *)c->rho, (cufftComplex *)c->rho_k)
                : cufftExecD2Z(c->plan_r2c, (cufftDoubleReal *)c->rho, (cufftDoubleComplex *)c->rho_k));
    }
    {
        Phase ph(c, PH_KSPACE);
        CK(launch_kspace(c));
    }
    {
        Phase ph(c, PH_FFT_C2R);
        CKF(c->precision == P3M_PREC_MIXED
                ? cufftExecC2R(c->plan_c2r, (cufftComplex *)c->frc_k, (cufftReal *)c->frc)
                : cufftExecZ2D(c->plan_c2r, (cufftDoubleComplex *)c->frc_k, (cufftDoubleReal *)c->frc));
    }
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

int key_current(p3m_ctx *c)
{
    Phase ph(c, PH_KICK_DRIFT);
    CK(launch_kick_drift_keys(c, false, 0.0, 0.0));
    return P3M_OK;
}

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

// One kick-drift-kick step a -> a + da with valid forces at a.  from_table: the step's factors
// come from the device table (graph-replayed steps; a and da unused).
int step_body(p3m_ctx *c, double a, double da, bool from_table)
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
    int rc = evaluate(c, k2, nullptr, from_table);
    if (rc) return rc;
    if (c->track_energy) {
        Phase ph(c, PH_OTHER);
        CK(launch_li_update(c, from_table ? c->cur_fac + 3 : nullptr, a + da));
    }
    return P3M_OK;
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

// Buffers whose roles swap during a step (all return to their roles after two steps).
struct PtrState {
    double *pos, *mom, *pos_alt, *mom_alt;
    uint32_t *pid, *pid_alt, *keys, *keys_alt, *vals, *vals_alt;
    uint32_t *work_key, *work_key_alt, *work_order, *work_order_alt;
    bool operator==(const PtrState &o) const { return memcmp(this, &o, sizeof(*this)) == 0; }
};

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

}  // namespace

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
    c->deconvolve = opt.deconvolve_cic ? 1 : 0;
    c->short_range = opt.short_range ? 1 : 0;
    c->cosmo = cs;
    c->mass = 1.0;
    c->a = 1.0;
    c->stream = (cudaStream_t)opt.stream;
    c->key_bits = key_bits;
    c->fac_cap = P3M_MAX_GRAPH_STEPS;
    strcpy(c->err, "no error");

    int rc = P3M_OK;
    do {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
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
            {(void **)&c->tab_origin, 8 * (size_t)g.n_c},
            {(void **)&c->fac_table, 8 * 4 * (size_t)P3M_MAX_GRAPH_STEPS},
            {(void **)&c->step_idx, 16},      {(void **)&c->cur_fac, 32},
            {(void **)&c->kself, 8 * 27},     {(void **)&c->li, 8 * 4},
            {(void **)&c->adj_u, 3 * real * M3}, {(void **)&c->adj_vfx, opt.precision == P3M_PREC_MIXED ? 384 * ((N + 31) / 32) : 16},
            {(void **)&c->adj_vs, 24 * N},    {(void **)&c->adj_out, 24 * N},
        };
        for (auto &a : allocs) {
            e = dalloc(a.p, a.bytes);
            if (e != cudaSuccess) {
                rc = fail(nullptr, P3M_ENOMEM, "p3m_init: cudaMalloc of %zu bytes failed: %s", a.bytes,
                          cudaGetErrorString(e));
                break;
            }
        }
        if (rc != P3M_OK) break;
        cudaMemsetAsync(c->counters, 0, 16, c->stream);
        cudaMemsetAsync(c->pair_count, 0, 64, c->stream);
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
        cufftResult r = cufftPlan3d(&c->plan_r2c, mesh, mesh, mesh,
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
            rc = fail(nullptr, P3M_ECUFFT, "p3m_init: cuFFT plan creation failed (code %d)", (int)r);
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

extern "C" int p3m_set_particles(p3m_ctx *c, const double *pos, const double *mom,
                                 const double *acc, double mass, double a, int on_device)
{
    if (!c) return fail(c, P3M_EINVAL, "ctx is NULL");
    if (!pos || !mom) return fail(c, P3M_EINVAL, "p3m_set_particles: pos and mom are required");
    if (!finite_pos(mass)) return fail(c, P3M_EINVAL, "p3m_set_particles: mass must be > 0");
    if (!finite_pos(a)) return fail(c, P3M_EINVAL, "p3m_set_particles: a must be > 0");
    const size_t bytes = 3 * sizeof(double) * (size_t)c->g.n;
    CK(cudaMemsetAsync(c->counters + 1, 0, sizeof(uint32_t), c->stream));
    const double *sp = pos, *sm = mom, *sa = acc;
    if (!on_device) {
        CK(cudaMemcpyAsync(c->pos_alt, pos, bytes, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->mom_alt, mom, bytes, cudaMemcpyHostToDevice, c->stream));
        sp = c->pos_alt;
        sm = c->mom_alt;
        if (acc) {
            CK(cudaMemcpyAsync(c->acc_lr, acc, bytes, cudaMemcpyHostToDevice, c->stream));
            sa = c->acc_lr;
        }
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
    if (!c) return fail(c, P3M_EINVAL, "ctx is NULL");
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_get_particles: no particles loaded");
    if (acc && !c->forces_valid) return fail(c, P3M_ESTATE, "p3m_get_particles: forces not evaluated");
    const size_t bytes = 3 * sizeof(double) * (size_t)c->g.n;
    double *outs[3] = {pos, mom, acc};
    const double *srcs[3] = {c->pos, c->mom, c->acc};
    for (int t = 0; t < 3; ++t) {
        if (!outs[t]) continue;
        if (on_device) {
            CK(launch_scatter_out(c, srcs[t], outs[t]));
        } else {
            double *stage = t == 0 ? c->pos_alt : (t == 1 ? c->mom_alt : c->acc_lr);
            CK(launch_scatter_out(c, srcs[t], stage));
            CK(cudaMemcpyAsync(outs[t], stage, bytes, cudaMemcpyDeviceToHost, c->stream));
        }
    }
    if (!on_device) return check_flags(c);
    return P3M_OK;
}

namespace {
int energy_now(p3m_ctx *c, double *kin, double *pot);
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

// ---------------------------------------------------------------- streams, graphs, ensembles

extern "C" int p3m_set_stream(p3m_ctx *c, void *stream)
{
    if (!c) return P3M_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    c->stream = (cudaStream_t)stream;
    CKF(cufftSetStream(c->plan_r2c, c->stream));
    CKF(cufftSetStream(c->plan_c2r, c->stream));
    CKF(cufftSetStream(c->plan_c2r_one, c->stream));
    return P3M_OK;
}

struct p3m_ensemble {
    int n;
    p3m_ctx **c;
    cudaStream_t parent;      // the graphs are launched here
    cudaStream_t *own;        // streams the ensemble created for its contexts (or NULL)
    cudaEvent_t fork, *join;  // fork/join of the captured branches
    cudaGraphExec_t gexec[2]; // one captured step for each step parity
    cudaGraphExec_t gchunk;   // kChunkSteps steps from parity 0: the contexts do not meet
                              // between these steps, so a short simulation runs ahead
    bool ready;
    int parity;               // parity of the next step to replay
    PtrState *state[2];       // per context: buffer roles before an even / odd step
    int *version;             // per context: geometry version the graphs were captured with

    // Batched pair launch: the FP32 P3M contexts' work items merged into one cost-sorted list
    // and evaluated by one persistent pair kernel per step.
    bool batched;             // on (default when at least two contexts qualify)
    int nb;                   // contexts that qualify (FP32, short range)
    int *slot;                // per context: its index among them, or -1
    size_t *base;             // per qualifying context: offset of its work list in gkey/gval
    size_t cap;               // sum of the qualifying contexts' work-list capacities
    PairArgs *descs;          // device: pair arguments per qualifying context
    const uint32_t **nwork;   // device: per qualifying context, its work-item count pointer
    uint32_t *gkey[2], *gval[2], *gcounts, *gaux, *gtotal, *gcursor;
    cudaEvent_t after_pairs;
    unsigned long long launches;
};

namespace {

constexpr int kChunkSteps = 8;  // steps per chunk graph (even: buffer roles have period 2)

// Captures `steps` consecutive steps of every context as parallel branches of one graph
// (one branch per context, its steps in sequence) into *out.
int ens_step(p3m_ensemble *e, double a, double da, bool from_table);

int capture_steps(p3m_ensemble *e, int steps, cudaGraphExec_t *out)
{
    p3m_ctx *c = nullptr;
    cudaGraph_t graph = nullptr;
    cudaError_t err = cudaStreamBeginCapture(e->parent, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess)
        return p3m_fail_global(P3M_ECUDA, "graph capture: %s", cudaGetErrorString(err));
    int rc = P3M_OK;
    if (e->batched) {  // the steps one after another, each with its batched pair launch
        for (int i = 0; i < e->n; ++i) e->c[i]->capturing = true;
        for (int k = 0; k < steps && rc == P3M_OK; ++k) rc = ens_step(e, 0.0, 0.0, true);
        for (int i = 0; i < e->n; ++i) e->c[i]->capturing = false;
    } else {  // each context's steps as one branch
        err = cudaEventRecord(e->fork, e->parent);
        for (int i = 0; i < e->n && err == cudaSuccess && rc == P3M_OK; ++i) {
            c = e->c[i];
            err = cudaStreamWaitEvent(c->stream, e->fork, 0);
            if (err != cudaSuccess) break;
            c->capturing = true;
            for (int k = 0; k < steps && rc == P3M_OK; ++k) rc = step_body(c, 0.0, 0.0, true);
            c->capturing = false;
            if (rc == P3M_OK) err = cudaEventRecord(e->join[i], c->stream);
            if (err == cudaSuccess && rc == P3M_OK) err = cudaStreamWaitEvent(e->parent, e->join[i], 0);
        }
    }
    cudaError_t end = cudaStreamEndCapture(e->parent, &graph);
    if (rc != P3M_OK) {
        if (graph) cudaGraphDestroy(graph);
        return p3m_fail_global(rc, "graph capture: %s", c ? c->err : g_init_err);
    }
    if (err == cudaSuccess) err = end;
    if (err == cudaSuccess) err = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (err != cudaSuccess)
        return p3m_fail_global(P3M_ECUDA, "graph capture: %s", cudaGetErrorString(err));
    return P3M_OK;
}

// One step of every context with the batched pair launch: the contexts' pre-pair phases as
// parallel branches (fork/join on the parent stream), then on the parent the merged work
// list's total, its 16-bit cost sort and one pair kernel over all of them, then the energy
// bookkeeping of contexts that track it.  from_table: graph-replayed (factors on the device).
int ens_step(p3m_ensemble *e, double a, double da, bool from_table)
{
    cudaError_t err = cudaEventRecord(e->fork, e->parent);
    int rc = P3M_OK;
    for (int i = 0; i < e->n && err == cudaSuccess && rc == P3M_OK; ++i) {
        p3m_ctx *c = e->c[i];
        err = cudaStreamWaitEvent(c->stream, e->fork, 0);
        if (err != cudaSuccess) break;
        const int sl = e->slot[i];
        rc = sl < 0 ? step_body(c, a, da, from_table)
                    : step_pre(c, a, da, from_table, sl, e->descs + sl, e->gkey[0] + e->base[sl],
                               e->gval[0] + e->base[sl]);
        if (rc == P3M_OK) err = cudaEventRecord(e->join[i], c->stream);
        if (err == cudaSuccess && rc == P3M_OK) err = cudaStreamWaitEvent(e->parent, e->join[i], 0);
    }
    if (rc != P3M_OK) {
        for (int i = 0; i < e->n; ++i)
            if (e->c[i]->err[0]) return p3m_fail_global(rc, "ensemble step: %s", e->c[i]->err);
        return p3m_fail_global(rc, "ensemble step failed");
    }
    if (err == cudaSuccess) err = launch_ens_total(e->nwork, e->nb, e->gtotal, e->parent);
    if (err == cudaSuccess) {
        uint32_t *k[2] = {e->gkey[0], e->gkey[1]}, *v[2] = {e->gval[0], e->gval[1]};
        err = radix_sort_pairs(k, v, false, (int64_t)e->cap, 16, e->gcounts, e->gaux, e->parent,
                               &e->launches);
        // two 8-bit passes: the result is back in gkey[0] / gval[0]
        if (err == cudaSuccess && (k[0] != e->gkey[0] || v[0] != e->gval[0])) err = cudaErrorUnknown;
    }
    if (err == cudaSuccess)
        err = launch_pairs_batched(e->descs, e->gval[0], e->gtotal, e->gcursor, e->c[0]->num_sms,
                                   e->parent);
    e->launches += 2;
    bool tracking = false;
    for (int i = 0; i < e->n; ++i) tracking = tracking || (e->slot[i] >= 0 && e->c[i]->track_energy);
    if (err == cudaSuccess && tracking) {
        err = cudaEventRecord(e->after_pairs, e->parent);
        for (int i = 0; i < e->n && err == cudaSuccess; ++i) {
            p3m_ctx *c = e->c[i];
            if (e->slot[i] < 0 || !c->track_energy) continue;
            err = cudaStreamWaitEvent(c->stream, e->after_pairs, 0);
            if (err == cudaSuccess)
                err = launch_li_update(c, from_table ? c->cur_fac + 3 : nullptr, a + da);
            if (err == cudaSuccess) err = cudaEventRecord(e->join[i], c->stream);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(e->parent, e->join[i], 0);
        }
    }
    if (err != cudaSuccess)
        return p3m_fail_global(P3M_ECUDA, "ensemble step: %s", cudaGetErrorString(err));
    return P3M_OK;
}

void drop_graphs(p3m_ensemble *e)
{
    for (int p = 0; p < 2; ++p)
        if (e->gexec[p]) {
            cudaGraphExecDestroy(e->gexec[p]);
            e->gexec[p] = nullptr;
        }
    if (e->gchunk) {
        cudaGraphExecDestroy(e->gchunk);
        e->gchunk = nullptr;
    }
    e->ready = false;
}

}  // namespace

extern "C" int p3m_ensemble_create(p3m_ensemble **out, p3m_ctx *const *ctxs, int n, int own_streams)
{
    if (!out || !ctxs || n < 1) return p3m_fail_global(P3M_EINVAL, "p3m_ensemble_create: bad arguments");
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return p3m_fail_global(P3M_EINVAL, "p3m_ensemble_create: context %d is NULL", i);
    p3m_ensemble *e = (p3m_ensemble *)calloc(1, sizeof(p3m_ensemble));
    if (!e) return p3m_fail_global(P3M_ENOMEM, "p3m_ensemble_create: host allocation failed");
    e->n = n;
    e->c = (p3m_ctx **)calloc(n, sizeof(p3m_ctx *));
    e->join = (cudaEvent_t *)calloc(n, sizeof(cudaEvent_t));
    e->state[0] = (PtrState *)calloc(n, sizeof(PtrState));
    e->state[1] = (PtrState *)calloc(n, sizeof(PtrState));
    e->version = (int *)calloc(n, sizeof(int));
    if (own_streams) e->own = (cudaStream_t *)calloc(n, sizeof(cudaStream_t));
    cudaError_t err = (e->c && e->join && e->state[0] && e->state[1] && e->version &&
                       (!own_streams || e->own))
                          ? cudaSuccess
                          : cudaErrorMemoryAllocation;
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->parent, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming);
    for (int i = 0; i < n && err == cudaSuccess; ++i) {
        e->c[i] = ctxs[i];
        err = cudaEventCreateWithFlags(&e->join[i], cudaEventDisableTiming);
        if (err == cudaSuccess && own_streams) {
            err = cudaStreamCreateWithFlags(&e->own[i], cudaStreamNonBlocking);
            if (err == cudaSuccess && p3m_set_stream(ctxs[i], e->own[i]) != P3M_OK) err = cudaErrorUnknown;
        }
    }
    if (err != cudaSuccess) {
        p3m_ensemble_free(e);
        return p3m_fail_global(P3M_ECUDA, "p3m_ensemble_create: %s", cudaGetErrorString(err));
    }
    // batched pair launch over the FP32 P3M contexts (work items coded (slot << 24) | item)
    e->slot = (int *)malloc(sizeof(int) * n);
    e->base = (size_t *)calloc(n, sizeof(size_t));
    if (!e->slot || !e->base) err = cudaErrorMemoryAllocation;
    std::vector<const uint32_t *> nw;
    for (int i = 0; i < n && err == cudaSuccess; ++i) {
        p3m_ctx *c = ctxs[i];
        const bool ok = c->precision == P3M_PREC_MIXED && c->short_range &&
                        c->max_work < (1u << 24) && e->nb < 255;
        e->slot[i] = ok ? e->nb : -1;
        if (ok) {
            e->base[e->nb] = e->cap;
            e->cap += c->max_work;
            nw.push_back(c->work_off + c->g.n_cells);
            ++e->nb;
        }
    }
    if (err == cudaSuccess && e->nb > 0) {
        const size_t tiles = (e->cap + P3M_SORT_TILE - 1) / P3M_SORT_TILE;
        const size_t scan_n = 256 * tiles;
        err = cudaMalloc((void **)&e->descs, sizeof(PairArgs) * e->nb);
        if (err == cudaSuccess) err = cudaMalloc((void **)&e->nwork, sizeof(uint32_t *) * e->nb);
        for (int b = 0; b < 2 && err == cudaSuccess; ++b) {
            err = cudaMalloc((void **)&e->gkey[b], 4 * e->cap);
            if (err == cudaSuccess) err = cudaMalloc((void **)&e->gval[b], 4 * e->cap);
        }
        if (err == cudaSuccess) err = cudaMalloc((void **)&e->gcounts, 4 * 256 * tiles);
        if (err == cudaSuccess) err = cudaMalloc((void **)&e->gaux, 4 * (scan_n / P3M_SORT_TILE + 4));
        if (err == cudaSuccess) err = cudaMalloc((void **)&e->gtotal, 16);
        if (err == cudaSuccess) err = cudaMalloc((void **)&e->gcursor, 16);
        if (err == cudaSuccess)
            err = cudaMemcpy((void *)e->nwork, nw.data(), sizeof(uint32_t *) * e->nb, cudaMemcpyHostToDevice);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->after_pairs, cudaEventDisableTiming);
    }
    e->batched = false;  // measured slower than per-context branches on uneven ensembles
    if (err != cudaSuccess) {
        p3m_ensemble_free(e);
        return p3m_fail_global(P3M_ECUDA, "p3m_ensemble_create: %s", cudaGetErrorString(err));
    }
    *out = e;
    return P3M_OK;
}

extern "C" int p3m_ensemble_set_batched(p3m_ensemble *e, int enable)
{
    if (!e) return p3m_fail_global(P3M_EINVAL, "p3m_ensemble_set_batched: NULL ensemble");
    const bool want = enable && e->nb >= 1;
    if (want != e->batched) drop_graphs(e);
    e->batched = want;
    return P3M_OK;
}

extern "C" int p3m_ensemble_run(p3m_ensemble *e, const double *a_list, int n_steps, int use_graph)
{
    if (!e || !a_list || n_steps < 1)
        return p3m_fail_global(P3M_EINVAL, "p3m_ensemble_run: bad arguments");
    if (n_steps > P3M_MAX_GRAPH_STEPS)
        return p3m_fail_global(P3M_EINVAL, "p3m_ensemble_run: at most %d steps per call", P3M_MAX_GRAPH_STEPS);
    for (int k = 0; k < n_steps; ++k)
        if (!finite_pos(a_list[k]) || !(a_list[k + 1] > a_list[k]))
            return p3m_fail_global(P3M_EINVAL, "p3m_ensemble_run: a_list must increase");
    for (int i = 0; i < e->n; ++i) {
        p3m_ctx *c = e->c[i];
        if (!c->have_particles) return p3m_fail_global(P3M_ESTATE, "p3m_ensemble_run: context %d has no particles", i);
        if (use_graph && !c->stream)
            return p3m_fail_global(P3M_EINVAL, "p3m_ensemble_run: graph mode needs non-default streams");
        if (!c->forces_valid) {
            int rc = key_current(c);
            if (!rc) rc = evaluate(c, 0.0, nullptr);
            if (rc) return p3m_fail_global(rc, "p3m_ensemble_run: %s", c->err);
            c->forces_valid = true;
        }
    }
    if (!use_graph && e->batched) {
        for (int k = 0; k < n_steps; ++k) {
            int rc = ens_step(e, a_list[k], a_list[k + 1] - a_list[k], false);
            if (rc) return rc;
        }
        // later work on the contexts' own streams comes after the last batched launch
        cudaError_t err = cudaEventRecord(e->fork, e->parent);
        for (int i = 0; i < e->n && err == cudaSuccess; ++i)
            err = cudaStreamWaitEvent(e->c[i]->stream, e->fork, 0);
        if (err != cudaSuccess)
            return p3m_fail_global(P3M_ECUDA, "p3m_ensemble_run: %s", cudaGetErrorString(err));
    } else if (!use_graph) {
        for (int k = 0; k < n_steps; ++k)
            for (int i = 0; i < e->n; ++i) {
                int rc = step_body(e->c[i], a_list[k], a_list[k + 1] - a_list[k], false);
                if (rc) return p3m_fail_global(rc, "p3m_ensemble_run: %s", e->c[i]->err);
            }
    } else {
        // per-step factors of every context, and its step counter reset
        std::vector<double> fac(4 * (size_t)n_steps);
        for (int i = 0; i < e->n; ++i) {
            p3m_ctx *c = e->c[i];
            for (int k = 0; k < n_steps; ++k) {
                const double a = a_list[k], a2 = a_list[k + 1], am = a + 0.5 * (a2 - a);
                fac[4 * k] = c->mass * p3m_kick_factor(c->cosmo, a, am);
                fac[4 * k + 1] = p3m_drift_factor(c->cosmo, a, a2) / c->mass;
                fac[4 * k + 2] = c->mass * p3m_kick_factor(c->cosmo, am, a2);
                fac[4 * k + 3] = a2;
            }
            cudaError_t err = cudaMemcpyAsync(c->fac_table, fac.data(), sizeof(double) * fac.size(),
                                              cudaMemcpyHostToDevice, c->stream);
            if (err == cudaSuccess) err = cudaMemsetAsync(c->step_idx, 0, sizeof(uint32_t), c->stream);
            if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
            if (err != cudaSuccess)
                return p3m_fail_global(P3M_ECUDA, "p3m_ensemble_run: %s", cudaGetErrorString(err));
        }
        // the graphs bake buffer addresses and geometry: recapture when they no longer match
        if (e->ready) {
            int par = -1;
            for (int p = 0; p < 2 && par < 0; ++p) {
                bool all = true;
                for (int i = 0; i < e->n; ++i)
                    all = all && save_ptrs(e->c[i]) == e->state[p][i] &&
                          e->version[i] == e->c[i]->geom_version;
                if (all) par = p;
            }
            if (par < 0) drop_graphs(e);
            else e->parity = par;
        }
        if (!e->ready) {
            for (int i = 0; i < e->n; ++i) {
                e->state[0][i] = save_ptrs(e->c[i]);
                e->version[i] = e->c[i]->geom_version;
            }
            int rc = capture_steps(e, 1, &e->gexec[0]);
            for (int i = 0; i < e->n && rc == P3M_OK; ++i) e->state[1][i] = save_ptrs(e->c[i]);
            if (rc == P3M_OK) rc = capture_steps(e, 1, &e->gexec[1]);
            // back at the parity-0 roles: the chunk graph starts there and ends there
            for (int i = 0; i < e->n && rc == P3M_OK; ++i)
                if (!(save_ptrs(e->c[i]) == e->state[0][i])) rc = P3M_ESTATE;
            if (rc == P3M_OK) rc = capture_steps(e, kChunkSteps, &e->gchunk);
            if (rc != P3M_OK) {
                for (int i = 0; i < e->n; ++i) load_ptrs(e->c[i], e->state[0][i]);
                drop_graphs(e);
                return rc;
            }
            e->ready = true;
            e->parity = 0;
        }
        cudaError_t err = cudaSuccess;
        for (int k = 0; k < n_steps && err == cudaSuccess;) {
            if (e->parity == 0 && n_steps - k >= kChunkSteps) {
                err = cudaGraphLaunch(e->gchunk, e->parent);
                k += kChunkSteps;
            } else {
                err = cudaGraphLaunch(e->gexec[e->parity], e->parent);
                e->parity ^= 1;
                ++k;
            }
        }
        // later work on the contexts' own streams comes after the replayed steps
        if (err == cudaSuccess) err = cudaEventRecord(e->fork, e->parent);
        for (int i = 0; i < e->n; ++i) {
            load_ptrs(e->c[i], e->state[e->parity][i]);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(e->c[i]->stream, e->fork, 0);
        }
        if (err != cudaSuccess)
            return p3m_fail_global(P3M_ECUDA, "p3m_ensemble_run: %s", cudaGetErrorString(err));
    }
    for (int i = 0; i < e->n; ++i) {
        e->c[i]->a = a_list[n_steps];
        e->c[i]->forces_valid = true;
    }
    return P3M_OK;
}

extern "C" void p3m_ensemble_free(p3m_ensemble *e)
{
    if (!e) return;
    if (e->parent) cudaStreamSynchronize(e->parent);
    drop_graphs(e);
    for (int i = 0; i < e->n; ++i) {
        if (e->c && e->c[i] && e->own && e->own[i]) {
            p3m_set_stream(e->c[i], nullptr);
            cudaStreamDestroy(e->own[i]);
        }
        if (e->join && e->join[i]) cudaEventDestroy(e->join[i]);
    }
    if (e->fork) cudaEventDestroy(e->fork);
    if (e->after_pairs) cudaEventDestroy(e->after_pairs);
    void *dbufs[] = {e->descs, (void *)e->nwork, e->gkey[0], e->gkey[1], e->gval[0], e->gval[1],
                     e->gcounts,  e->gaux, e->gtotal, e->gcursor};
    for (void *q : dbufs)
        if (q) cudaFree(q);
    free(e->slot);
    free(e->base);
    if (e->parent) cudaStreamDestroy(e->parent);
    free(e->c);
    free(e->join);
    free(e->own);
    free(e->state[0]);
    free(e->state[1]);
    free(e->version);
    free(e);
}

extern "C" int p3m_run_steps(p3m_ctx *c, const double *a_list, int n_steps, int use_graph)
{
    if (!c) return P3M_EINVAL;
    if (!use_graph) {
        for (int k = 0; k < n_steps; ++k) {
            int rc = p3m_step(c, a_list[k], a_list[k + 1] - a_list[k]);
            if (rc) return rc;
        }
        return P3M_OK;
    }
    if (!c->self_ens) {
        int rc = p3m_ensemble_create(&c->self_ens, &c, 1, 0);
        if (rc) return fail(c, rc, "%s", g_init_err);
    }
    int rc = p3m_ensemble_run(c->self_ens, a_list, n_steps, 1);
    if (rc) return fail(c, rc, "%s", g_init_err);
    return P3M_OK;
}

// ---------------------------------------------------------------- autotuner

extern "C" int p3m_autotune(p3m_ctx *c, int *sub_bits_out, double *ms_out)
{
    if (!c) return P3M_EINVAL;
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_autotune: no particles loaded");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int saved_b = c->g.sub_bits;
    int best_b = saved_b;
    double best_ms = 1e300;
    for (int b = 0; b <= 3; ++b) {
        const uint64_t max_key = ((uint64_t)c->g.n_cells << (3 * b)) - 1;
        if (ms_out) ms_out[b] = NAN;
        if (max_key >= (1ull << 32)) continue;
        c->g.sub_bits = b;
        c->g.n_fine = c->g.n_c << b;
        c->g.inv_fine = (double)c->g.n_fine / c->g.box;
        c->key_bits = 1;
        while (c->key_bits < 32 && (max_key >> c->key_bits)) ++c->key_bits;
        ++c->geom_version;
        int rc = key_current(c);
        if (!rc) rc = evaluate(c, 0.0, nullptr);  // warm-up (and a sort from the previous order)
        if (rc) return rc;
        CK(cudaEventRecord(e0, c->stream));
        for (int r = 0; r < 2 && !rc; ++r) {
            rc = key_current(c);
            if (!rc) rc = evaluate(c, 0.0, nullptr);
        }
        if (rc) return rc;
        CK(cudaEventRecord(e1, c->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms_out) ms_out[b] = ms / 2.0;
        if (ms / 2.0 < best_ms) {
            best_ms = ms / 2.0;
            best_b = b;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const uint64_t max_key = ((uint64_t)c->g.n_cells << (3 * best_b)) - 1;
    c->g.sub_bits = best_b;
    c->g.n_fine = c->g.n_c << best_b;
    c->g.inv_fine = (double)c->g.n_fine / c->g.box;
    c->key_bits = 1;
    while (c->key_bits < 32 && (max_key >> c->key_bits)) ++c->key_bits;
    ++c->geom_version;
    int rc = key_current(c);
    if (!rc) rc = evaluate(c, 0.0, nullptr);
    if (rc) return rc;
    c->forces_valid = true;
    if (sub_bits_out) *sub_bits_out = best_b;
    return P3M_OK;
}

// ---------------------------------------------------------------- reverse-mode derivatives

extern "C" int p3m_step_factors(const p3m_ctx *c, double a, double da, double *k1, double *dfac,
                                double *k2)
{
    if (!c || !finite_pos(a) || !finite_pos(da)) return P3M_EINVAL;
    const double am = a + 0.5 * da, a2 = a + da;
    if (k1) *k1 = c->mass * p3m_kick_factor(c->cosmo, a, am);
    if (dfac) *dfac = p3m_drift_factor(c->cosmo, a, a2) / c->mass;
    if (k2) *k2 = c->mass * p3m_kick_factor(c->cosmo, am, a2);
    return P3M_OK;
}

extern "C" int p3m_axpy(p3m_ctx *c, double alpha, const double *x3n, double *y3n)
{
    if (!c || !x3n || !y3n) return fail(c, P3M_EINVAL, "p3m_axpy: NULL argument");
    CK(launch_axpy(c, y3n, x3n, alpha));
    return P3M_OK;
}

extern "C" int p3m_force_vjp(p3m_ctx *c, const double *v3n, double *out3n, int on_device)
{
    if (!c || !v3n || !out3n) return fail(c, P3M_EINVAL, "p3m_force_vjp: NULL argument");
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_force_vjp: no particles loaded");
    const size_t bytes = 3 * sizeof(double) * (size_t)c->g.n;
    // sort, cells and mesh fields at the current positions (the pair forces are not needed)
    int rc = key_current(c);
    if (!rc) rc = evaluate(c, 0.0, nullptr, false, false);
    if (rc) return rc;
    c->forces_valid = !c->short_range;
    const double *vin = v3n;
    if (!on_device) {
        CK(cudaMemcpyAsync(c->pos_alt, v3n, bytes, cudaMemcpyHostToDevice, c->stream));
        vin = c->pos_alt;
    }
    CK(launch_to_slots(c, vin, c->adj_vs));
    CK(launch_force_vjp(c, c->adj_vs, c->adj_out));
    if (on_device) {
        CK(launch_scatter_out(c, c->adj_out, out3n));
        return P3M_OK;
    }
    CK(launch_scatter_out(c, c->adj_out, c->pos_alt));
    CK(cudaMemcpyAsync(out3n, c->pos_alt, bytes, cudaMemcpyDeviceToHost, c->stream));
    return check_flags(c);
}

extern "C" int p3m_density_loss(p3m_ctx *c, const double *target, double *loss, double *grad3n,
                                int on_device)
{
    if (!c || !target || !loss) return fail(c, P3M_EINVAL, "p3m_density_loss: NULL argument");
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_density_loss: no particles loaded");
    const size_t M3 = (size_t)c->g.mesh * c->g.mesh * c->g.mesh;
    const size_t bytes = 3 * sizeof(double) * (size_t)c->g.n;
    const double *t = target;
    if (!on_device) {
        CK(cudaMemcpyAsync(c->adj_u, target, sizeof(double) * M3, cudaMemcpyHostToDevice, c->stream));
        t = (const double *)c->adj_u;
    }
    CK(launch_deposit(c));
    double *loss_dev = c->red + 1024 * 4 + 4;
    CK(launch_density_loss(c, t, loss_dev, grad3n ? c->adj_out : nullptr));
    if (grad3n) {
        if (on_device) {
            CK(launch_scatter_out(c, c->adj_out, grad3n));
        } else {
            CK(launch_scatter_out(c, c->adj_out, c->pos_alt));
            CK(cudaMemcpyAsync(grad3n, c->pos_alt, bytes, cudaMemcpyDeviceToHost, c->stream));
        }
    }
    CK(cudaMemcpyAsync(loss, loss_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return P3M_OK;
}

// ---------------------------------------------------------------- energies

namespace {

// phi_per - phi_iso: the long-range potential a particle feels from its own periodic images
// (with the neutralising background), by the Ewald identity at alpha = 2.6/L for the lattice
// sum and the split's alpha = 1/(2 r_s) for the short-range images:
//   (4 pi/L^3) sum_{k != 0} exp(-k^2 r_s^2)/k^2 = psi_self - sum_{n != 0} erfc(|n|L/(2 r_s))/(|n|L)
//                                                  + 4 pi r_s^2/L^3 + 1/(sqrt(pi) r_s),
// psi_self the alpha-independent Ewald self term of one particle per cell.
double image_potential(const P3MGeom &g)
{
    const double L = g.box, alpha = 2.6 / L, rs = g.r_s;
    double real = 0.0, recip = 0.0, srimg = 0.0;
    for (int x = -3; x <= 3; ++x)
        for (int y = -3; y <= 3; ++y)
            for (int z = -3; z <= 3; ++z) {
                if (!x && !y && !z) continue;
                const double r = L * sqrt((double)(x * x + y * y + z * z));
                real += erfc(alpha * r) / r;
                srimg += erfc(0.5 * r / rs) / r;
            }
    const double kf = 2.0 * M_PI / L;
    for (int x = -8; x <= 8; ++x)
        for (int y = -8; y <= 8; ++y)
            for (int z = -8; z <= 8; ++z) {
                if (!x && !y && !z) continue;
                const double k2 = kf * kf * (double)(x * x + y * y + z * z);
                recip += exp(-k2 / (4.0 * alpha * alpha)) / k2;
            }
    const double V = L * L * L;
    const double psi_self = real + 4.0 * M_PI / V * recip - M_PI / (alpha * alpha * V) -
                            2.0 * alpha / sqrt(M_PI);
    const double ksum = psi_self - srimg + 4.0 * M_PI * rs * rs / V + 1.0 / (sqrt(M_PI) * rs);
    return -g.gm * ksum + g.gm / (sqrt(M_PI) * rs);  // phi_per - phi_iso
}

int energy_now(p3m_ctx *c, double *kin, double *pot)
{
    int rc = key_current(c);
    if (!rc) rc = evaluate(c, 0.0, nullptr, false, false);
    if (rc) return rc;
    double cst = 0.0;
    if (c->short_range) {
        const double V = c->g.box * c->g.box * c->g.box;
        cst = image_potential(c->g) + 4.0 * M_PI * c->g.gm * ((double)c->g.n / V) * c->g.r_s * c->g.r_s;
    }
    double *sum_dev = c->red + 1024 * 4 + 5;
    CK(launch_potential(c, cst, c->adj_out, sum_dev));
    double sum = 0.0, r[4];
    CK(cudaMemcpyAsync(&sum, sum_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(launch_diag(c, r));  // synchronises
    *pot = 0.5 * c->mass * sum / c->a;
    *kin = r[3] / (2.0 * c->mass * c->a * c->a);
    c->forces_valid = !c->short_range;
    return P3M_OK;
}

}  // namespace

extern "C" int p3m_energy(p3m_ctx *c, double *kinetic, double *potential)
{
    if (!c || !kinetic || !potential) return fail(c, P3M_EINVAL, "p3m_energy: NULL argument");
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_energy: no particles loaded");
    return energy_now(c, kinetic, potential);
}

extern "C" int p3m_track_energy(p3m_ctx *c, int enable)
{
    if (!c) return P3M_EINVAL;
    if (!enable) {
        if (c->track_energy) ++c->geom_version;
        c->track_energy = false;
        return P3M_OK;
    }
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_track_energy: no particles loaded");
    double k0 = 0.0, w0 = 0.0;
    int rc = energy_now(c, &k0, &w0);
    if (rc) return rc;
    double p2 = 2.0 * c->mass * c->a * c->a * k0;
    const double li0[4] = {0.0, p2, c->a, 0.0};
    CK(cudaMemcpyAsync(c->li, li0, sizeof(li0), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->li_a0 = c->a;
    c->li_e0 = c->a * (k0 + w0);
    c->track_energy = true;
    ++c->geom_version;  // captured steps lack the tracking kernels
    return P3M_OK;
}
