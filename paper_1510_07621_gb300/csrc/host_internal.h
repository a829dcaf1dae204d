// Host-side internals shared by the C ABI's translation units (api.cu, ensemble.cu,
// derivatives.cu): error reporting, the phases of a force evaluation and of a step, and the
// buffer roles that captured graphs depend on.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <nvtx3/nvToolsExt.h>
#include <string.h>

#include "p3m_internal.cuh"

extern char g_init_err[512];  // message of the last failure without a context

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return p3m_host::fail(c, P3M_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define CKF(call)                                                                           \
    do {                                                                                    \
        cufftResult r_ = (call);                                                            \
        if (r_ != CUFFT_SUCCESS)                                                            \
            return p3m_host::fail(c, P3M_ECUFFT, "%s failed: cufft code %d", #call, (int)r_); \
    } while (0)

namespace p3m_host {

// Writes the message into c->err (or the global message when c is NULL); returns code.
int fail(p3m_ctx *c, int code, const char *fmt, ...);

extern const char *kPhaseNames[P3M_NPHASES];

// One phase on the context's stream: an NVTX range named after the phase (host-side, for
// profilers' timelines), and CUDA-event timing when enabled (skipped while capturing a graph).
struct Phase {
    p3m_ctx *c;
    int id;
    Phase(p3m_ctx *c_, int id_) : c(c_), id(id_)
    {
        nvtxRangePushA(kPhaseNames[id_]);
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
        nvtxRangePop();
    }
};

// An NVTX range over one call of the C ABI.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

// Reads the device flags (a bounded wait that gave up); synchronises.
int check_flags(p3m_ctx *c);
// Sort by cell, mesh force, pair force at the current (keyed) positions; see api.cu.
int evaluate(p3m_ctx *c, double kfac, double *sr_only_out, bool from_table = false,
             bool pairs = true);
// The phases of evaluate, in order: sort, permute and deposit; R2C; k-space pass; C2R; gather
// and pair force (with the fused kick).
int eval_pre(p3m_ctx *c);
int eval_r2c(p3m_ctx *c);
int eval_kspace(p3m_ctx *c);
int eval_c2r(p3m_ctx *c);
int eval_post(p3m_ctx *c, double kfac, double *sr_only_out, bool from_table, bool pairs);
// The parts of step_body: factors, first half kick and drift (second kick's factor in *k2), and
// the energy bookkeeping after the forces.
int step_kd(p3m_ctx *c, double a, double da, bool from_table, double *k2);
int step_tail(p3m_ctx *c, double a, double da, bool from_table);
// Wrap and key the current positions (no kick, no drift).
int key_current(p3m_ctx *c);
bool finite_pos(double x);
// One kick-drift-kick step with valid forces at a (from_table: factors from the device table).
int step_body(p3m_ctx *c, double a, double da, bool from_table);
// The part of a step before the pair sum, for the ensemble's batched pair launch.
int step_pre(p3m_ctx *c, double a, double da, bool from_table, int slot, PairArgs *desc,
             uint32_t *gk, uint32_t *gv);

// Buffers whose roles swap during a step (all return to their roles after two steps).
struct PtrState {
    double *pos, *mom, *pos_alt, *mom_alt;
    uint32_t *pid, *pid_alt, *keys, *keys_alt, *vals, *vals_alt;
    uint32_t *work_key, *work_key_alt, *work_order, *work_order_alt;
    bool operator==(const PtrState &o) const { return memcmp(this, &o, sizeof(*this)) == 0; }
};

PtrState save_ptrs(const p3m_ctx *c);
void load_ptrs(p3m_ctx *c, const PtrState &s);

// Kinetic and potential energy of the current state (sorts and evaluates the mesh).
int energy_now(p3m_ctx *c, double *kin, double *pot);

}  // namespace p3m_host
