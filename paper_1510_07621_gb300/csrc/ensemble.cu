// Streams, CUDA-graph replay of whole steps, ensembles of contexts (with the optional batched
// pair launch) and the sort-key autotuner.
#include <cuda_runtime.h>

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "host_internal.h"

using namespace p3m_host;

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

    // Size-grouped FFTs: contexts with the same mesh and precision whose density, spectrum and
    // force meshes are slices of one allocation, so that one batched R2C and one batched C2R
    // (on the parent stream) serve the whole group; the steps then run in phases (see ens_step_fft).
    bool grouped;             // on (default when some group has at least two contexts)
    int ngrp;
    struct FftGroup *grp;
    int *gi;                  // per context: its group, or -1 (its FFTs stay its own)
    void **saved;             // per context: its own rho, rho_k, frc_k, frc while grouped
    double *k2;               // per context: second half-kick factor of the current step
};

struct FftGroup {
    int mesh, precision, count;
    size_t rho_b, rhok_b, frck_b, frc_b;  // bytes of one member's slice of each buffer
    void *rho, *rho_k, *frc_k, *frc;
    cufftHandle r2c, c2r;
    bool plans;
};

namespace {

constexpr int kChunkSteps = 8;  // steps per chunk graph (even: buffer roles have period 2)

// Captures `steps` consecutive steps of every context as parallel branches of one graph
// (one branch per context, its steps in sequence) into *out.
int ens_step(p3m_ensemble *e, double a, double da, bool from_table);
int ens_step_fft(p3m_ensemble *e, double a, double da, bool from_table);

int capture_steps(p3m_ensemble *e, int steps, cudaGraphExec_t *out)
{
    p3m_ctx *c = nullptr;
    cudaGraph_t graph = nullptr;
    cudaError_t err = cudaStreamBeginCapture(e->parent, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess)
        return p3m_fail_global(P3M_ECUDA, "graph capture: %s", cudaGetErrorString(err));
    int rc = P3M_OK;
    if (e->batched || e->grouped) {  // the steps one after another, in lockstep
        for (int i = 0; i < e->n; ++i) e->c[i]->capturing = true;
        for (int k = 0; k < steps && rc == P3M_OK; ++k)
            rc = e->batched ? ens_step(e, 0.0, 0.0, true) : ens_step_fft(e, 0.0, 0.0, true);
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

// One lockstep step of every context with the FFTs of each group batched: (A) per context, the
// first half kick, drift, sort, permute and deposit (a context outside every group runs its whole
// step here); (B) one batched R2C per group; (C) per context, the k-space pass; (D) one batched
// C2R per group; (E) per context, the gather, the pair force with the second half kick and the
// energy bookkeeping.  Branches fork from and join the parent stream at each phase.
int ens_step_fft(p3m_ensemble *e, double a, double da, bool from_table)
{
    auto fork = [&]() { return cudaEventRecord(e->fork, e->parent); };
    cudaError_t err = fork();
    int rc = P3M_OK;
    for (int phase = 0; phase < 3 && err == cudaSuccess && rc == P3M_OK; ++phase) {
        if (phase > 0) err = fork();
        for (int i = 0; i < e->n && err == cudaSuccess && rc == P3M_OK; ++i) {
            p3m_ctx *c = e->c[i];
            if (phase > 0 && e->gi[i] < 0) continue;
            err = cudaStreamWaitEvent(c->stream, e->fork, 0);
            if (err != cudaSuccess) break;
            if (phase == 0) {
                if (e->gi[i] < 0) {
                    rc = step_body(c, a, da, from_table);
                } else {
                    rc = step_kd(c, a, da, from_table, &e->k2[i]);
                    if (!rc) rc = eval_pre(c);
                }
            } else if (phase == 1) {
                rc = eval_kspace(c);
            } else {
                rc = eval_post(c, e->k2[i], nullptr, from_table, true);
                if (!rc) rc = step_tail(c, a, da, from_table);
            }
            if (rc == P3M_OK) err = cudaEventRecord(e->join[i], c->stream);
            if (err == cudaSuccess && rc == P3M_OK) err = cudaStreamWaitEvent(e->parent, e->join[i], 0);
        }
        for (int g = 0; g < e->ngrp && phase < 2 && err == cudaSuccess && rc == P3M_OK; ++g) {
            FftGroup &G = e->grp[g];
            const bool f32 = G.precision == P3M_PREC_MIXED;
            const cufftResult r =
                phase == 0 ? (f32 ? cufftExecR2C(G.r2c, (cufftReal *)G.rho, (cufftComplex *)G.rho_k)
                                  : cufftExecD2Z(G.r2c, (cufftDoubleReal *)G.rho, (cufftDoubleComplex *)G.rho_k))
                           : (f32 ? cufftExecC2R(G.c2r, (cufftComplex *)G.frc_k, (cufftReal *)G.frc)
                                  : cufftExecZ2D(G.c2r, (cufftDoubleComplex *)G.frc_k, (cufftDoubleReal *)G.frc));
            if (r != CUFFT_SUCCESS) return p3m_fail_global(P3M_ECUFFT, "ensemble step: batched cuFFT code %d", (int)r);
            e->launches += 1;
        }
    }
    if (rc != P3M_OK) {
        for (int i = 0; i < e->n; ++i)
            if (e->c[i]->err[0] && strcmp(e->c[i]->err, "no error")) return p3m_fail_global(rc, "ensemble step: %s", e->c[i]->err);
        return p3m_fail_global(rc, "ensemble step failed");
    }
    if (err != cudaSuccess)
        return p3m_fail_global(P3M_ECUDA, "ensemble step: %s", cudaGetErrorString(err));
    return P3M_OK;
}

// Point every grouped context back at its own meshes (copying the group slices' contents there)
// and release the groups' buffers and plans.
void ungroup(p3m_ensemble *e)
{
    if (e->parent) cudaStreamSynchronize(e->parent);
    for (int i = 0; i < e->n && e->gi; ++i) {
        const int g = e->gi[i];
        if (g < 0) continue;
        p3m_ctx *c = e->c[i];
        FftGroup &G = e->grp[g];
        cudaStreamSynchronize(c->stream);
        void **own = e->saved + 4 * i;
        cudaMemcpy(own[0], c->rho, G.rho_b, cudaMemcpyDeviceToDevice);
        cudaMemcpy(own[1], c->rho_k, G.rhok_b, cudaMemcpyDeviceToDevice);
        cudaMemcpy(own[2], c->frc_k, G.frck_b, cudaMemcpyDeviceToDevice);
        cudaMemcpy(own[3], c->frc, G.frc_b, cudaMemcpyDeviceToDevice);
        c->rho = own[0];
        c->rho_k = own[1];
        c->frc_k = own[2];
        c->frc = own[3];
        c->fft_grouped = false;
        ++c->geom_version;  // graphs that baked the slices go stale
        e->gi[i] = -1;
    }
    for (int g = 0; g < e->ngrp; ++g) {
        FftGroup &G = e->grp[g];
        if (G.plans) {
            cufftDestroy(G.r2c);
            cufftDestroy(G.c2r);
        }
        void *bufs[] = {G.rho, G.rho_k, G.frc_k, G.frc};
        for (void *b : bufs)
            if (b) cudaFree(b);
    }
    free(e->grp);
    e->grp = nullptr;
    e->ngrp = 0;
    e->grouped = false;
}

// Groups the contexts by (mesh, precision); every group of at least two gets one allocation
// per mesh buffer, sliced among its members, and batched plans on the parent stream.
int group_ffts(p3m_ensemble *e)
{
    std::vector<FftGroup> gs;
    std::vector<std::vector<int>> members;
    for (int i = 0; i < e->n; ++i) {
        p3m_ctx *c = e->c[i];
        if (c->fft_grouped) continue;  // already in another ensemble's group: keeps its FFTs
        int g = -1;
        for (size_t k = 0; k < gs.size() && g < 0; ++k)
            if (gs[k].mesh == c->g.mesh && gs[k].precision == c->precision) g = (int)k;
        if (g < 0) {
            FftGroup G;
            memset(&G, 0, sizeof(G));
            G.mesh = c->g.mesh;
            G.precision = c->precision;
            gs.push_back(G);
            members.emplace_back();
            g = (int)gs.size() - 1;
        }
        members[g].push_back(i);
    }
    e->grp = (FftGroup *)calloc(gs.size() ? gs.size() : 1, sizeof(FftGroup));
    if (!e->grp) return P3M_ENOMEM;
    for (int i = 0; i < e->n; ++i) e->gi[i] = -1;
    for (size_t k = 0; k < gs.size(); ++k) {
        if (members[k].size() < 2) continue;
        FftGroup &G = e->grp[e->ngrp];
        G = gs[k];
        G.count = (int)members[k].size();
        const size_t M = (size_t)G.mesh, M3 = M * M * M, nk = M * M * (M / 2 + 1);
        const size_t real = G.precision == P3M_PREC_MIXED ? 4 : 8;
        G.rho_b = real * M3;
        G.rhok_b = 2 * real * nk;
        G.frck_b = 6 * real * nk;
        G.frc_b = 3 * real * M3;
        cudaError_t err = cudaMalloc(&G.rho, G.rho_b * G.count);
        if (err == cudaSuccess) err = cudaMalloc(&G.rho_k, G.rhok_b * G.count);
        if (err == cudaSuccess) err = cudaMalloc(&G.frc_k, G.frck_b * G.count);
        if (err == cudaSuccess) err = cudaMalloc(&G.frc, G.frc_b * G.count);
        ++e->ngrp;  // (released by ungroup on failure)
        if (err != cudaSuccess) return P3M_ENOMEM;
        int dims[3] = {G.mesh, G.mesh, G.mesh};
        const bool f32 = G.precision == P3M_PREC_MIXED;
        cufftResult r = cufftPlanMany(&G.r2c, 3, dims, nullptr, 1, (int)M3, nullptr, 1, (int)nk,
                                      f32 ? CUFFT_R2C : CUFFT_D2Z, G.count);
        if (r == CUFFT_SUCCESS) {
            r = cufftPlanMany(&G.c2r, 3, dims, nullptr, 1, (int)nk, nullptr, 1, (int)M3,
                              f32 ? CUFFT_C2R : CUFFT_Z2D, 3 * G.count);
            if (r != CUFFT_SUCCESS) cufftDestroy(G.r2c);
        }
        if (r != CUFFT_SUCCESS) return P3M_ECUFFT;
        G.plans = true;
        cufftSetStream(G.r2c, e->parent);
        cufftSetStream(G.c2r, e->parent);
        for (int s_ = 0; s_ < G.count; ++s_) {
            const int i = members[k][s_];
            p3m_ctx *c = e->c[i];
            CK(cudaStreamSynchronize(c->stream));
            void **own = e->saved + 4 * i;
            own[0] = c->rho;
            own[1] = c->rho_k;
            own[2] = c->frc_k;
            own[3] = c->frc;
            c->rho = (char *)G.rho + G.rho_b * s_;
            c->rho_k = (char *)G.rho_k + G.rhok_b * s_;
            c->frc_k = (char *)G.frc_k + G.frck_b * s_;
            c->frc = (char *)G.frc + G.frc_b * s_;
            ++c->geom_version;
            c->fft_grouped = true;
            e->gi[i] = e->ngrp - 1;
        }
    }
    e->grouped = e->ngrp > 0;
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
    e->batched = false;  // within 1 % of per-context branches on an uneven ensemble, which
                         // keep the contexts independent
    // size-grouped FFTs, on by default when some group has at least two contexts
    e->gi = (int *)malloc(sizeof(int) * n);
    e->saved = (void **)calloc(4 * (size_t)n, sizeof(void *));
    e->k2 = (double *)calloc(n, sizeof(double));
    if (err == cudaSuccess && (!e->gi || !e->saved || !e->k2)) err = cudaErrorMemoryAllocation;
    if (err == cudaSuccess) {
        const int rc = group_ffts(e);
        if (rc != P3M_OK) {
            ungroup(e);
            p3m_ensemble_free(e);
            return p3m_fail_global(rc, "p3m_ensemble_create: grouping the FFTs failed");
        }
    }
    if (err != cudaSuccess) {
        p3m_ensemble_free(e);
        return p3m_fail_global(P3M_ECUDA, "p3m_ensemble_create: %s", cudaGetErrorString(err));
    }
    *out = e;
    return P3M_OK;
}

extern "C" int p3m_ensemble_set_fft_groups(p3m_ensemble *e, int enable)
{
    if (!e) return p3m_fail_global(P3M_EINVAL, "p3m_ensemble_set_fft_groups: NULL ensemble");
    const bool want = enable != 0;
    if (want == (e->grp != nullptr)) return P3M_OK;
    drop_graphs(e);
    if (!want) {
        ungroup(e);
        return P3M_OK;
    }
    const int rc = group_ffts(e);
    if (rc != P3M_OK) {
        ungroup(e);
        return p3m_fail_global(rc, "p3m_ensemble_set_fft_groups: grouping the FFTs failed");
    }
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
    } else if (!use_graph && e->grouped) {
        for (int k = 0; k < n_steps; ++k) {
            int rc = ens_step_fft(e, a_list[k], a_list[k + 1] - a_list[k], false);
            if (rc) return rc;
        }
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
    if (e->grp) ungroup(e);
    free(e->gi);
    free(e->saved);
    free(e->k2);
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
    // then the FP32 pair kernel's tile length at that key (3 or 5 blocks of 32 j particles)
    if (c->precision == P3M_PREC_MIXED && c->short_range) {
        double best_t = 1e300;
        int best_tb = c->tile_blocks;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        for (int tb = 3; tb <= 5; tb += 2) {
            c->tile_blocks = tb;
            rc = key_current(c);
            if (!rc) rc = evaluate(c, 0.0, nullptr);  // warm-up
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
            if (ms < best_t) {
                best_t = ms;
                best_tb = tb;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->tile_blocks = best_tb;
        ++c->geom_version;  // captured graphs bake the kernel choice
        rc = key_current(c);
        if (!rc) rc = evaluate(c, 0.0, nullptr);
        if (rc) return rc;
    }
    c->forces_valid = true;
    if (sub_bits_out) *sub_bits_out = best_b;
    return P3M_OK;
}

extern "C" int p3m_get_tuning(const p3m_ctx *c, int *sub_bits, int *tile_blocks)
{
    if (!c) return P3M_EINVAL;
    if (sub_bits) *sub_bits = c->g.sub_bits;
    if (tile_blocks) *tile_blocks = c->tile_blocks;
    return P3M_OK;
}

