// Kick, particle load/unload in the caller's order, and FP64 diagnostics reductions.
#include <cuda_runtime.h>

#include "p3m_internal.cuh"

namespace {

inline int grid_for(int64_t n, int threads, int num_sms)
{
    int64_t b = (n + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

__global__ void k_kick(double *__restrict__ mom, const double *__restrict__ acc, int64_t n3,
                       double kfac, const double *__restrict__ kfac_dev)
{
    if (kfac_dev) kfac = *kfac_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3;
         i += (int64_t)gridDim.x * blockDim.x)
        mom[i] = __dadd_rn(mom[i], __dmul_rn(kfac, acc[i]));
}

__device__ __forceinline__ double wrap_box(double x, double L)
{
    // x = fmod(x, L); x < 0 -> x += L; x >= L -> x -= L.  Inside [0, L) (the common case after
    // a drift) every step leaves x unchanged, and fmod(x, L) == x for -L < x < L: the FP64
    // sequence, slow on GB300's FP64 pipe, runs only for the rest.
    // x in [0, L) as integer compares of the bit patterns (IEEE order of non-negative doubles;
    // -0.0 and NaN take the full sequence, which leaves -0.0 unchanged, as this test would)
    const long long xb = __double_as_longlong(x);
    if (xb >= 0 && xb < __double_as_longlong(L)) return x;
    if (!(x > -L && x < L)) x = fmod(x, L);
    if (x < 0.0) x = __dadd_rn(x, L);
    if (x >= L) x = __dadd_rn(x, -L);
    return x;
}

// Copies caller arrays into slot order = caller order, wraps positions, identity ids,
// and flags any NaN/Inf.
__global__ void k_load(const double *__restrict__ pos, const double *__restrict__ mom,
                       const double *__restrict__ acc, int64_t n, double L,
                       double *__restrict__ pos_out, double *__restrict__ mom_out,
                       double *__restrict__ acc_out, uint32_t *__restrict__ pid,
                       uint32_t *__restrict__ flags)
{
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double x = pos[d * n + i], p = mom[d * n + i];
            bad |= !isfinite(x) || !isfinite(p);
            pos_out[d * n + i] = isfinite(x) ? wrap_box(x, L) : 0.0;
            mom_out[d * n + i] = p;
            if (acc) {
                const double a = acc[d * n + i];
                bad |= !isfinite(a);
                acc_out[d * n + i] = a;
            }
        }
        pid[i] = (uint32_t)i;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, P3M_FLAG_NONFINITE);
}

// dst[d][pid[k]] = src[d][k]
__global__ void k_scatter(const double *__restrict__ src, const uint32_t *__restrict__ pid,
                          int64_t n, double *__restrict__ dst)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = pid[k];
        dst[j] = src[k];
        dst[n + j] = src[n + k];
        dst[2 * n + j] = src[2 * n + k];
    }
}

// inv[pid[k]] = k: the slot of each particle of the caller's order.
__global__ void k_inverse(const uint32_t *__restrict__ pid, int64_t n, uint32_t *__restrict__ inv)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        inv[pid[k]] = (uint32_t)k;
}

// dst (caller order) = src (slot order) through the inverse permutation: the writes are
// sequential, so dst may be host memory that the GPU writes over the CPU-GPU link.
__global__ void k_gather_out(const double *__restrict__ src, const uint32_t *__restrict__ inv,
                             int64_t n, double *__restrict__ dst)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = inv[j];
        dst[j] = src[k];
        dst[n + j] = src[n + k];
        dst[2 * n + j] = src[2 * n + k];
    }
}

// Per-block partial sums of (px, py, pz, |p|^2) in a fixed order; then one block adds the
// partials in block order.  Same result on every run.
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1024;

__global__ void __launch_bounds__(kRedThreads)
    k_diag_partial(const double *__restrict__ mom, int64_t n, double *__restrict__ part)
{
    __shared__ double s[4][kRedThreads];
    double acc[4] = {0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double px = mom[i], py = mom[n + i], pz = mom[2 * n + i];
        acc[0] += px;
        acc[1] += py;
        acc[2] += pz;
        acc[3] += px * px + py * py + pz * pz;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) part[blockIdx.x * 4 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void __launch_bounds__(kRedThreads) k_diag_final(double *part, int nb)
{
    __shared__ double s[4][kRedThreads];
    double acc[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += part[b * 4 + q];
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) part[kRedBlocks * 4 + threadIdx.x] = s[threadIdx.x][0];
}

}  // namespace

cudaError_t launch_axpy(p3m_ctx *c, double *y, const double *x, double alpha)
{
    c->launches += 1;
    const int64_t n3 = 3 * c->g.n;
    k_kick<<<grid_for(n3, 256, c->num_sms), 256, 0, c->stream>>>(y, x, n3, alpha, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_kick(p3m_ctx *c, double kfac, const double *kfac_dev)
{
    c->launches += 1;
    const int64_t n3 = 3 * c->g.n;
    k_kick<<<grid_for(n3, 256, c->num_sms), 256, 0, c->stream>>>(c->mom, c->acc, n3, kfac, kfac_dev);
    return cudaGetLastError();
}

namespace {
// First kernel of a graph-replayed step: the step's factors (K1, D, K2, a at the end) from the
// table into the fixed slot the other kernels read, and the step counter advanced.
__global__ void k_step_begin(const double *__restrict__ table, uint32_t *step_idx, double *cur)
{
    const uint32_t s = *step_idx;
    cur[0] = table[4 * s];
    cur[1] = table[4 * s + 1];
    cur[2] = table[4 * s + 2];
    cur[3] = table[4 * s + 3];
    *step_idx = s + 1;
}

// Trapezoid update of the Layzer-Irvine integral of K da from sum p^2 at the step's end.
__global__ void k_li_update(const double *__restrict__ p2, const double *__restrict__ a_dev,
                            double a_host, double mass, double *li)
{
    const double a = a_dev ? *a_dev : a_host;
    const double k_now = *p2 / (2.0 * mass * a * a);
    const double k_prev = li[1] / (2.0 * mass * li[2] * li[2]);
    li[0] += 0.5 * (k_prev + k_now) * (a - li[2]);
    li[1] = *p2;
    li[2] = a;
}
}  // namespace

cudaError_t launch_step_begin(p3m_ctx *c)
{
    c->launches += 1;
    k_step_begin<<<1, 1, 0, c->stream>>>(c->fac_table, c->step_idx, c->cur_fac);
    return cudaGetLastError();
}

cudaError_t launch_load_particles(p3m_ctx *c, const double *pos, const double *mom,
                                  const double *acc)
{
    c->launches += 1;
    k_load<<<grid_for(c->g.n, 256, c->num_sms), 256, 0, c->stream>>>(
        pos, mom, acc, c->g.n, c->g.box, c->pos, c->mom, c->acc, c->pid, c->counters + 1);
    return cudaGetLastError();
}

cudaError_t launch_scatter_out(p3m_ctx *c, const double *src, double *dst)
{
    c->launches += 1;
    k_scatter<<<grid_for(c->g.n, 256, c->num_sms), 256, 0, c->stream>>>(src, c->pid, c->g.n, dst);
    return cudaGetLastError();
}

cudaError_t launch_inverse_pid(p3m_ctx *c, uint32_t *inv)
{
    c->launches += 1;
    k_inverse<<<grid_for(c->g.n, 256, c->num_sms), 256, 0, c->stream>>>(c->pid, c->g.n, inv);
    return cudaGetLastError();
}

cudaError_t launch_gather_out(p3m_ctx *c, const double *src, const uint32_t *inv, double *dst)
{
    c->launches += 1;
    k_gather_out<<<grid_for(c->g.n, 256, c->num_sms), 256, 0, c->stream>>>(src, inv, c->g.n, dst);
    return cudaGetLastError();
}

cudaError_t launch_li_update(p3m_ctx *c, const double *a_now_dev, double a_now)
{
    c->launches += 3;
    k_diag_partial<<<kRedBlocks, kRedThreads, 0, c->stream>>>(c->mom, c->g.n, c->red);
    k_diag_final<<<1, kRedThreads, 0, c->stream>>>(c->red, kRedBlocks);
    k_li_update<<<1, 1, 0, c->stream>>>(c->red + kRedBlocks * 4 + 3, a_now_dev, a_now, c->mass, c->li);
    return cudaGetLastError();
}

cudaError_t launch_diag(p3m_ctx *c, double *host_out)
{
    c->launches += 2;
    k_diag_partial<<<kRedBlocks, kRedThreads, 0, c->stream>>>(c->mom, c->g.n, c->red);
    k_diag_final<<<1, kRedThreads, 0, c->stream>>>(c->red, kRedBlocks);
    cudaError_t e = cudaMemcpyAsync(host_out, c->red + kRedBlocks * 4, 4 * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(c->stream);
}

// ------------------------------------------------------------------ FMA throughput probe
// Independent multiply-add chains (8 per thread) over many resident warps: the measured
// FP32 / FP64 FMA rate of this GPU, for the roofline of the pair kernels.

namespace {

constexpr int kProbeChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, T seed, int iters)
{
    T a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = seed + (T)k;
    const T b = (T)0.9999999, c = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], b, c);
    }
    T t = 0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) t += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;  // keeps the chains alive
}

template <typename T>
int fma_probe(int iters, double *tflops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return P3M_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return P3M_ECUDA;
    const int threads = 256, blocks = sms * 8;
    const size_t nt = (size_t)threads * blocks;
    T *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, nt * sizeof(T));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.0f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {  // first launch warms up
        e = cudaEventRecord(e0, s);
        k_fma_probe<T><<<blocks, threads, 0, s>>>(out, (T)1, iters);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e == cudaSuccess && best > 0.0f)
        *tflops = 2.0 * kProbeChains * (double)iters * (double)nt / (best * 1e-3) / 1e12;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    return e == cudaSuccess ? P3M_OK : P3M_ECUDA;
}

}  // namespace

extern "C" int p3m_measure_fma_peak(int fp64, double *tflops)
{
    if (!tflops) return P3M_EINVAL;
    *tflops = NAN;
    return fp64 ? fma_probe<double>(256, tflops) : fma_probe<float>(8192, tflops);
}
