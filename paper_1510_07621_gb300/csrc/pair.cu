// Short-range particle-particle part of the P3M force (the guide's P3M kick algorithm with
// split scale PM_scale and cutoff P3M_cutoff, Ch. Parameters):
//
//   a_SR,i = G m * sum_{j: 0 < r_ij < r_c} g(r_ij / r_s) d_ij / (r_ij^2 + eps^2)^(3/2),
//   g(x) = erfc(x/2) + x/sqrt(pi) exp(-x^2/4),
//
// over the particles of the 27 chaining cells around particle i's cell (n_c >= 3 cells of
// side >= r_c, so each neighbour cell appears once and with the minimum image).
//
// Work item = up to 128 particles of one cell (one per thread).  The j particles of the 27
// neighbour cells stream through shared memory in tiles of 256, copied by the bulk-copy (TMA)
// engine into two alternating buffers (the next tile is in flight while the current one is
// used), completion tracked by one mbarrier per buffer.  Coordinates are relative to each
// particle's own cell origin (FP32 in the mixed mode), shifted per neighbour cell by the
// FP64 offset between the two cell origins, so no FP32 absolute coordinate ever appears.
// Per-tile FP32 partial sums are added into FP64 accumulators per particle.
// CTAs are persistent and take work items from an atomic cursor.
#include <cuda_runtime.h>

#include "p3m_internal.cuh"

namespace {

constexpr int kTI = P3M_PAIR_TI;
constexpr int kTJ = P3M_PAIR_TJ;

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = double4;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Plain (non-multicast) bulk copy global -> this CTA's shared memory; both addresses 16-byte
// aligned, size a multiple of 16 bytes.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity; gives up after ~2^31 clock cycles (about one
// second) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) return false;
    }
    return true;
}

// Pair kernel g(x) * (r^2 + eps^2)^-3/2 for one pair with r2 = |d|^2 (0 < r2 < r_c^2).
__device__ __forceinline__ float pair_factor(float r2, float eps2, float inv_rs)
{
    const float s = rsqrtf(r2 + eps2);
    const float x = r2 * rsqrtf(r2) * inv_rs;
    const float g = erfcf(0.5f * x) + x * 0.564189583547756287f * expf(-0.25f * x * x);
    return g * s * s * s;
}

__device__ __forceinline__ double pair_factor(double r2, double eps2, double inv_rs)
{
    const double s = 1.0 / sqrt(r2 + eps2);
    const double x = sqrt(r2) * inv_rs;
    const double g = erfc(0.5 * x) + x * 0.56418958354775628695 * exp(-0.25 * x * x);
    return g * s * s * s;
}

struct Neighbour {
    uint32_t start, end;
    double sx, sy, sz;  // origin(neighbour, unwrapped image) - origin(own cell)
};

template <typename T>
__global__ void __launch_bounds__(kTI)
    k_pairs(const typename Vec4<T>::type *__restrict__ rel, const uint32_t *__restrict__ cell_start,
            const uint32_t *__restrict__ work, const uint32_t *__restrict__ n_work_ptr, P3MGeom g,
            const double *__restrict__ acc_in, double *__restrict__ acc_out,
            double *__restrict__ mom, double kfac, uint32_t *__restrict__ counters,
            unsigned long long *__restrict__ pair_count)
{
    using V4 = typename Vec4<T>::type;
    // FP64 mode keeps absolute coordinates (d = (x_j - x_i) + image, the same operations as a
    // plain minimum-image difference); FP32 mode uses cell-relative coordinates.
    constexpr bool kAbsolute = sizeof(T) == 8;
    __shared__ __align__(128) V4 sj[2][kTJ];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ Neighbour nbr[27];
    __shared__ uint32_t s_item;

    const int tid = threadIdx.x;
    const int64_t n = g.n;
    const uint32_t n_work = *n_work_ptr;
    const T rc2 = (T)(g.r_c * g.r_c);
    const T eps2 = (T)(g.eps * g.eps);
    const T inv_rs = (T)(1.0 / g.r_s);
    const int nc = g.n_c;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t parity[2] = {0u, 0u};
    unsigned long long my_pairs = 0;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(&counters[0], 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_work) break;
        const uint32_t cell = work[2 * (size_t)item];
        const uint32_t first = work[2 * (size_t)item + 1];
        const uint32_t cend = cell_start[cell + 1];
        const int cx = (int)(cell % nc), cy = (int)((cell / nc) % nc), cz = (int)(cell / (nc * nc));
        if (tid < 27) {
            const int ox = tid % 3 - 1, oy = (tid / 3) % 3 - 1, oz = tid / 9 - 1;
            int ux = cx + ox, uy = cy + oy, uz = cz + oz;  // unwrapped neighbour index
            const int wx = (ux + nc) % nc, wy = (uy + nc) % nc, wz = (uz + nc) % nc;
            const uint32_t nb = ((uint32_t)wz * nc + wy) * nc + wx;
            Neighbour q;
            q.start = cell_start[nb];
            q.end = cell_start[nb + 1];
            const double L = g.box, cs = g.cs;
            const double ix = ux < 0 ? -L : (ux >= nc ? L : 0.0);
            const double iy = uy < 0 ? -L : (uy >= nc ? L : 0.0);
            const double iz = uz < 0 ? -L : (uz >= nc ? L : 0.0);
            if (kAbsolute) {  // periodic image only
                q.sx = ix;
                q.sy = iy;
                q.sz = iz;
            } else {  // offset between the two cell origins (image included)
                q.sx = ((double)wx * cs + ix) - (double)cx * cs;
                q.sy = ((double)wy * cs + iy) - (double)cy * cs;
                q.sz = ((double)wz * cs + iz) - (double)cz * cs;
            }
            nbr[tid] = q;
        }
        __syncthreads();

        const uint32_t i = first + tid;
        const bool valid = i < cend;
        V4 xi = valid ? rel[i] : V4{};
        double ax = 0.0, ay = 0.0, az = 0.0;

        // tile sequence: neighbour nb, tile start js; (27, *) = done
        int nb_c = 0;
        uint32_t js_c = nbr[0].start;
        auto advance = [&](int &nb, uint32_t &js) {
            // move (nb, js) to the next non-empty tile position at or after it
            while (nb < 27 && js >= nbr[nb].end) {
                ++nb;
                if (nb < 27) js = nbr[nb].start;
            }
        };
        advance(nb_c, js_c);
        int buf = 0;
        if (nb_c < 27 && tid == 0) {
            const uint32_t len = min((uint32_t)kTJ, nbr[nb_c].end - js_c);
            mbar_expect_tx(&bar[0], len * (uint32_t)sizeof(V4));
            bulk_load(&sj[0][0], rel + js_c, len * (uint32_t)sizeof(V4), &bar[0]);
        }
        bool timed_out = false;
        while (nb_c < 27) {
            const uint32_t len = min((uint32_t)kTJ, nbr[nb_c].end - js_c);
            int nb_n = nb_c;
            uint32_t js_n = js_c + len;
            advance(nb_n, js_n);
            if (nb_n < 27 && tid == 0) {
                const uint32_t ln = min((uint32_t)kTJ, nbr[nb_n].end - js_n);
                mbar_expect_tx(&bar[buf ^ 1], ln * (uint32_t)sizeof(V4));
                bulk_load(&sj[buf ^ 1][0], rel + js_n, ln * (uint32_t)sizeof(V4), &bar[buf ^ 1]);
            }
            const bool ok = mbar_wait_bounded(&bar[buf], parity[buf]);
            parity[buf] ^= 1u;
            if (__syncthreads_or(!ok)) {
                timed_out = true;
                if (nb_n < 27) {  // drain the copy in flight into the other buffer
                    mbar_wait_bounded(&bar[buf ^ 1], parity[buf ^ 1]);
                }
                break;
            }
            // FP32: xs = x_i - shift, d = x_j - xs;  FP64: d = (x_j - x_i) + image
            const T xs = kAbsolute ? (T)xi.x : (T)((double)xi.x - nbr[nb_c].sx);
            const T ys = kAbsolute ? (T)xi.y : (T)((double)xi.y - nbr[nb_c].sy);
            const T zs = kAbsolute ? (T)xi.z : (T)((double)xi.z - nbr[nb_c].sz);
            const T ix = kAbsolute ? (T)nbr[nb_c].sx : T(0);
            const T iy = kAbsolute ? (T)nbr[nb_c].sy : T(0);
            const T iz = kAbsolute ? (T)nbr[nb_c].sz : T(0);
            T px = 0, py = 0, pz = 0;
            uint32_t cnt = 0;
            const V4 *tile = sj[buf];
            for (uint32_t j = 0; j < len; ++j) {
                const V4 q = tile[j];
                T dx = q.x - xs, dy = q.y - ys, dz = q.z - zs;
                if (kAbsolute) {
                    dx += ix;
                    dy += iy;
                    dz += iz;
                }
                const T r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < rc2 && r2 > T(0)) {
                    const T f = pair_factor(r2, eps2, inv_rs);
                    px += f * dx;
                    py += f * dy;
                    pz += f * dz;
                    ++cnt;
                }
            }
            ax += (double)px;
            ay += (double)py;
            az += (double)pz;
            if (valid) my_pairs += cnt;
            __syncthreads();  // every thread is done with sj[buf] before it is refilled
            buf ^= 1;
            nb_c = nb_n;
            js_c = js_n;
        }
        if (timed_out) {
            if (tid == 0) atomicOr(&counters[1], P3M_FLAG_TIMEOUT);
            break;
        }
        if (valid) {
            double a3[3] = {g.gm * ax, g.gm * ay, g.gm * az};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double tot = (acc_in ? acc_in[d * n + i] : 0.0) + a3[d];
                acc_out[d * n + i] = tot;
                if (kfac != 0.0) mom[d * n + i] = __dadd_rn(mom[d * n + i], __dmul_rn(kfac, tot));
            }
        }
    }
    // pair count: warp sum, one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_pairs += __shfl_down_sync(0xffffffffu, my_pairs, o);
    if ((tid & 31) == 0 && my_pairs) {
        atomicAdd(pair_count, my_pairs);
        atomicAdd(pair_count + 1, my_pairs);
    }
}

template <typename T>
cudaError_t pairs_impl(p3m_ctx *c, const double *acc_in, double *acc_out, double kfac)
{
    cudaMemsetAsync(c->counters, 0, sizeof(uint32_t), c->stream);
    cudaMemsetAsync(c->pair_count, 0, sizeof(unsigned long long), c->stream);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs<T>, kTI, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int grid = c->num_sms * per_sm;
    c->launches += 1;
    k_pairs<T><<<grid, kTI, 0, c->stream>>>((const typename Vec4<T>::type *)c->rel, c->cell_start,
                                            c->work, c->work_off + c->g.n_cells, c->g, acc_in,
                                            acc_out, c->mom, kfac, c->counters, c->pair_count);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pairs(p3m_ctx *c, const double *acc_in, double *acc_out, double kfac)
{
    return c->precision == P3M_PREC_MIXED ? pairs_impl<float>(c, acc_in, acc_out, kfac)
                                          : pairs_impl<double>(c, acc_in, acc_out, kfac);
}
