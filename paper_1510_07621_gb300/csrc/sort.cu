// Chaining-cell keys, stable LSD radix sort, particle permutation, cell ranges and the
// pair work list.
//
// Key of a particle (the chaining-mesh binning of P3M; the guide only fixes the cutoff that
// sets the cell size, Ch. Parameters "P3M_cutoff"): with n_f = n_c 2^b fine cells per side,
//   f_d = min(trunc(x_d * (n_f / L)), n_f - 1)   (one correctly rounded FP64 multiply)
//   cell = (c_z n_c + c_y) n_c + c_x,  c_d = f_d >> b
//   key  = (cell << 3b) | Hilbert(f_x mod 2^b, f_y mod 2^b, f_z mod 2^b)
// (Hilbert: the index along the 3-D Hilbert curve of order b, after Skilling, "Programming the
// Hilbert curve", AIP Conf. Proc. 707, 2004; consecutive indices are face neighbours, so runs of
// consecutive particles are more compact than along a Morton order)
// Particles are ordered by key, ties by their current slot (a stable sort), so the order is
// reproducible bit for bit.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "p3m_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = P3M_SORT_TILE / kThreads;  // 16
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

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

__device__ __forceinline__ uint32_t fine_index(double x, double inv, int nf)
{
    int f = (int)__dmul_rn(x, inv);  // x >= 0: truncation is floor
    return (uint32_t)min(f, nf - 1);
}

// The same index without FP64 arithmetic in almost every case.  x_f = x truncated to its
// leading 24 significant bits (bit operations), inv_f = inv rounded to FP32: the FP32 product
// p = x_f inv_f is within 2^-22 x inv < 2^-22 n_f of x inv, and the correctly rounded FP64
// product within 2^-53 n_f of it.  So when p lies more than tol = 2^-21 n_f from every
// integer, floor(p) is floor of the FP64 product; otherwise the FP64 product decides.
__device__ __forceinline__ uint32_t fine_index_fast(double x, double inv, float inv_f, float tol, int nf)
{
    const long long xb = __double_as_longlong(x);
    const int e = (int)((xb >> 52) & 0x7FF) - 1023 + 127;  // x >= 0: no sign bit
    const float xf = e >= 1 ? __int_as_float((e << 23) | (int)((xb >> 29) & 0x7FFFFF)) : 0.0f;
    const float p = xf * inv_f;
    const float k = truncf(p);
    if (p - k > tol && p - k < 1.0f - tol) return (uint32_t)min((int)k, nf - 1);
    return fine_index(x, inv, nf);
}

__device__ __forceinline__ uint32_t make_key(uint32_t fx, uint32_t fy, uint32_t fz,
                                             const P3MGeom &g)
{
    const int b = g.sub_bits;
    const uint32_t cell = ((fz >> b) * (uint32_t)g.n_c + (fy >> b)) * (uint32_t)g.n_c + (fx >> b);
    const uint32_t m = (1u << b) - 1u;
    uint32_t x[3] = {fx & m, fy & m, fz & m}, code = 0;
    if (b > 0) {
        const uint32_t top = 1u << (b - 1);
        for (uint32_t q = top; q > 1; q >>= 1) {  // undo the excess rotations and reflections
            const uint32_t low = q - 1;
            for (int i = 0; i < 3; ++i) {
                if (x[i] & q) {
                    x[0] ^= low;
                } else {
                    const uint32_t t = (x[0] ^ x[i]) & low;
                    x[0] ^= t;
                    x[i] ^= t;
                }
            }
        }
        x[1] ^= x[0];  // Gray encode
        x[2] ^= x[1];
        uint32_t t = 0;
        for (uint32_t q = top; q > 1; q >>= 1)
            if (x[2] & q) t ^= q - 1;
        for (int i = 0; i < 3; ++i) x[i] ^= t;
        for (int level = b - 1; level >= 0; --level)
            for (int i = 0; i < 3; ++i) code = (code << 1) | ((x[i] >> level) & 1u);
    }
    return (cell << (3 * b)) | code;
}

// Half kick + drift (optional), periodic wrap, key.  Kick and drift are one FMA each (a single
// rounding): p += (m K) a; x += p (D / m).  With fac_dev the two factors are read from
// fac_dev[0], fac_dev[1] (graph-replayed steps).
__global__ void k_kick_drift_keys(double *__restrict__ pos, double *__restrict__ mom,
                                  const double *__restrict__ acc, P3MGeom g, int kick_drift,
                                  double kfac, double dfac, uint32_t *__restrict__ keys,
                                  const double *__restrict__ fac_dev)
{
    const int64_t n = g.n;
    if (fac_dev) {
        kfac = fac_dev[0];
        dfac = fac_dev[1];
    }
    const float inv_f = (float)g.inv_fine, tol = (float)g.n_fine * 0x1p-21f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t f[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double x = pos[d * n + i];
            if (kick_drift) {
                const double p = __fma_rn(kfac, acc[d * n + i], mom[d * n + i]);
                mom[d * n + i] = p;
                x = __fma_rn(p, dfac, x);
            }
            x = wrap_box(x, g.box);
            pos[d * n + i] = x;
            f[d] = fine_index_fast(x, g.inv_fine, inv_f, tol, g.n_fine);
        }
        const uint32_t key = make_key(f[0], f[1], f[2], g);
        p3m_in_bounds((key >> (3 * g.sub_bits)) < (uint32_t)g.n_cells, g.flags);
        keys[i] = key;
    }
}

// ------------------------------------------------------------------ radix sort, 8-bit digits
// Tile t holds keys [t*4096, (t+1)*4096), visited in 16 rounds of 256 consecutive keys;
// within a round warp w holds keys [w*32, w*32+32).  That visiting order is the input order,
// so ranks assigned round by round, warp by warp, lane by lane make each pass stable.

__global__ void __launch_bounds__(kThreads)
    k_radix_upsweep(const uint32_t *__restrict__ keys, int64_t n, int shift,
                    uint32_t *__restrict__ counts, int n_tiles)
{
    __shared__ uint32_t hist[kRadix];
    const int tid = threadIdx.x, lane = tid & 31;
    hist[tid] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * P3M_SORT_TILE;
    for (int r = 0; r < kItems; ++r) {
        const int64_t idx = base + r * kThreads + tid;
        const bool valid = idx < n;
        const uint32_t d = valid ? (keys[idx] >> shift) & (kRadix - 1) : (uint32_t)kRadix;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&hist[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    counts[(size_t)tid * n_tiles + blockIdx.x] = hist[tid];
}

__global__ void __launch_bounds__(kThreads)
    k_radix_downsweep(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                      int64_t n, int shift, const uint32_t *__restrict__ offsets, int n_tiles,
                      uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out)
{
    __shared__ uint32_t s_base[kRadix];
    __shared__ uint32_t s_cnt[kThreads / 32][kRadix];
    __shared__ uint32_t s_pos[kThreads / 32][kRadix];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_base[tid] = offsets[(size_t)tid * n_tiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s_cnt[w][tid] = 0;
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * P3M_SORT_TILE;
    for (int r = 0; r < kItems; ++r) {
        const int64_t idx = base + r * kThreads + tid;
        const bool valid = idx < n;
        uint32_t key = 0, val = 0;
        if (valid) {
            key = keys_in[idx];
            val = vals_in ? vals_in[idx] : (uint32_t)idx;
        }
        const uint32_t d = valid ? (key >> shift) & (kRadix - 1) : (uint32_t)kRadix;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) s_cnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t run = s_base[tid];
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) {
                const uint32_t c = s_cnt[w][tid];
                s_cnt[w][tid] = 0;
                s_pos[w][tid] = run;
                run += c;
            }
            s_base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t p = s_pos[warp][d] + rank;
            keys_out[p] = key;
            vals_out[p] = val;
        }
    }
}

// ------------------------------------------------------------------ one-sweep LSD radix sort
// The particle sort: one histogram kernel for all passes, then one kernel per 8-bit pass.  A
// pass's CTAs take 4096-key tiles in launch order from an atomic counter; each ranks its tile
// (warp w the keys [512 w, 512 w + 512), round by round and lane by lane, so ranks are
// stable), publishes its per-digit counts, and finds the count of each digit in all earlier
// tiles by walking back over their published values (decoupled look-back: an entry holds a
// tile's own count, flag kAgg, or the running total through that tile, flag kInc).  A tile
// publishes kAgg before it waits for anything, and waits only on tiles taken before it, so
// every wait ends; each is still bounded (about a second) and sets P3M_FLAG_TIMEOUT when it
// gives up.  The tile is then reordered in shared memory by digit and written out in runs,
// coalesced, at global position = (keys of smaller digits) + (keys of the digit in earlier
// tiles) + (rank in the tile).

constexpr int kWarps = kThreads / 32;
constexpr int kWarpItems = P3M_SORT_TILE / kWarps;  // 512
constexpr unsigned long long kAgg = 1ull << 62, kInc = 2ull << 62, kCountMask = (1ull << 62) - 1;

// hist[p * 256 + d] += number of keys whose digit p is d, for p < passes (<= 4)
__global__ void __launch_bounds__(kThreads)
    k_digit_hist(const uint32_t *__restrict__ keys, int64_t n, int passes, uint32_t *__restrict__ hist)
{
    __shared__ uint32_t h[4 * kRadix];
    for (int i = threadIdx.x; i < 4 * kRadix; i += kThreads) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i0 = (int64_t)blockIdx.x * kThreads; i0 < n; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const bool valid = i < n;
        const uint32_t k = valid ? keys[i] : 0u;
        for (int p = 0; p < passes; ++p) {
            const uint32_t d = valid ? (k >> (p * kRadixBits)) & (kRadix - 1) : (uint32_t)kRadix;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[p * kRadix + d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kThreads)
        if (h[i]) atomicAdd(hist + i, h[i]);
}

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total);

__global__ void __launch_bounds__(kThreads, 3)
    k_onesweep(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, int64_t n,
               int shift, const uint32_t *__restrict__ hist, unsigned long long *status,
               uint32_t *tile_counter, uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
               uint32_t *flags, const unsigned long long *lookback, long long wait_limit)
{
    __shared__ uint32_t s_key[P3M_SORT_TILE];
    __shared__ uint32_t s_val[P3M_SORT_TILE];
    __shared__ uint32_t s_wcnt[kWarps][kRadix];  // per-warp digit counts, then offsets
    __shared__ uint32_t s_off[kRadix];           // first tile slot of each digit
    __shared__ uint32_t s_out[kRadix];           // global position of the digit's first key
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s_wcnt[w][tid] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t wbase = (int64_t)tile * P3M_SORT_TILE + (int64_t)warp * kWarpItems;
    const uint32_t lt = (1u << lane) - 1u;

    // the warp's 512 keys and values (all loads in flight at once), then their ranks
    uint32_t key[kItems], val[kItems], rank[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t idx = wbase + r * 32 + lane;
        const bool valid = idx < n;
        key[r] = valid ? kin[idx] : 0u;
        val[r] = valid ? (vin ? vin[idx] : (uint32_t)idx) : 0u;
    }
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const bool valid = wbase + r * 32 + lane < n;
        const uint32_t d = valid ? (key[r] >> shift) & (kRadix - 1) : (uint32_t)kRadix;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const int lead = __ffs(peers) - 1;
        uint32_t before = 0;
        if (valid && lane == lead) {
            before = s_wcnt[warp][d];
            s_wcnt[warp][d] = before + __popc(peers);
        }
        before = __shfl_sync(0xffffffffu, before, lead);
        rank[r] = before + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();

    // thread tid = digit d: the tile's count, published at once; per-warp offsets
    const int d = tid;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = s_wcnt[w][d];
        s_wcnt[w][d] = cnt;
        cnt += c;
    }
    unsigned long long *mine = status + (size_t)tile * kRadix + d;
    if (tile == 0)
        atomicExch(mine, kInc | cnt);
    else
        atomicExch(mine, kAgg | cnt);
    s_off[d] = block_exclusive_scan(cnt, nullptr);
    const uint32_t first = block_exclusive_scan(hist[d], nullptr);
    // keys of digit d in the tiles before this one
    unsigned long long before = 0;
    if (tile > 0) {
        long long t = (long long)tile - 1;
        const long long t0 = clock64();
        for (;;) {
            // lookback is status itself, except under an injected timeout (a zeroed copy)
            const unsigned long long v = *(volatile const unsigned long long *)(lookback + (size_t)t * kRadix + d);
            const unsigned long long f = v & ~kCountMask;
            if (f == 0ull) {
                if (clock64() - t0 > wait_limit) {
                    atomicOr(flags, P3M_FLAG_TIMEOUT);
                    break;
                }
                __nanosleep(32);
                continue;
            }
            before += v & kCountMask;
            if (f == kInc) break;
            --t;
        }
        atomicExch(mine, kInc | (before + cnt));
    }
    s_out[d] = first + (uint32_t)before;
    __syncthreads();

    // the tile in digit order in shared memory, then written out in runs
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t idx = wbase + r * 32 + lane;
        if (idx < n) {
            const uint32_t dd = (key[r] >> shift) & (kRadix - 1);
            const uint32_t slot = s_off[dd] + s_wcnt[warp][dd] + rank[r];
            s_key[slot] = key[r];
            s_val[slot] = val[r];
        }
    }
    __syncthreads();
    const int64_t left = n - (int64_t)tile * P3M_SORT_TILE;
    const int count = left < P3M_SORT_TILE ? (int)left : P3M_SORT_TILE;
    for (int j = tid; j < count; j += kThreads) {
        const uint32_t k = s_key[j];
        const uint32_t dd = (k >> shift) & (kRadix - 1);
        const uint32_t p = s_out[dd] + (uint32_t)j - s_off[dd];
        if (p < n) {  // (always, unless a look-back wait gave up)
            kout[p] = k;
            vout[p] = s_val[j];
        }
    }
}

// ------------------------------------------------------------------ exclusive scan (uint32)

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < kThreads / 32 ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    const uint32_t before = warp ? warp_sums[warp - 1] : 0u;
    if (total) *total = warp_sums[kThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kThreads)
    k_scan_reduce(const uint32_t *__restrict__ in, size_t n, uint32_t *__restrict__ aux)
{
    const size_t base = (size_t)blockIdx.x * P3M_SORT_TILE;
    uint32_t s = 0;
    for (int r = 0; r < kItems; ++r) {
        const size_t i = base + r * kThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    uint32_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) aux[blockIdx.x] = total;
}

// Single block: exclusive scan of aux[0..nb) in place, aux[nb] = total.
__global__ void __launch_bounds__(kThreads) k_scan_aux(uint32_t *aux, size_t nb)
{
    uint32_t carry = 0;
    for (size_t base = 0; base < nb; base += kThreads) {
        const size_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? aux[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, &total);
        if (i < nb) aux[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) aux[nb] = carry;
}

// Each thread owns 16 consecutive items of the block's 4096 (read before any write, so
// in == out is allowed).
__global__ void __launch_bounds__(kThreads)
    k_scan_down(const uint32_t *in, uint32_t *out, size_t n, const uint32_t *__restrict__ aux)
{
    const size_t base = (size_t)blockIdx.x * P3M_SORT_TILE + (size_t)threadIdx.x * kItems;
    uint32_t v[kItems];
    uint32_t s = 0;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        v[r] = (base + r < n) ? in[base + r] : 0u;
        s += v[r];
    }
    uint32_t run = aux[blockIdx.x] + block_exclusive_scan(s, nullptr);
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        if (base + r < n) out[base + r] = run;
        run += v[r];
    }
}

// ------------------------------------------------------------------ permutation and cells

template <typename R4>
__device__ __forceinline__ R4 make_rel(double x, double y, double z);
template <>
__device__ __forceinline__ float4 make_rel<float4>(double x, double y, double z)
{
    return make_float4((float)x, (float)y, (float)z, 0.0f);
}
template <>
__device__ __forceinline__ double4_16a make_rel<double4_16a>(double x, double y, double z)
{
    return make_double4_16a(x, y, z, 0.0);
}

// FP32 mode: position minus its cell origin (no FP32 absolute coordinate).  FP64 mode: the
// absolute position itself, so that the pair kernel forms x_j - x_i exactly like a plain
// minimum-image difference.
// (origin[c] = c * cs, a host table: the same correctly rounded products without the FP64
// multiply and conversion per particle)
template <typename R4>
__device__ __forceinline__ R4 rel_coords(double x, double y, double z, uint32_t cx, uint32_t cy,
                                         uint32_t cz, const double *origin)
{
    return make_rel<R4>(x - __ldg(origin + cx), y - __ldg(origin + cy), z - __ldg(origin + cz));
}
template <>
__device__ __forceinline__ double4_16a rel_coords<double4_16a>(double x, double y, double z, uint32_t,
                                                       uint32_t, uint32_t, const double *)
{
    return make_double4_16a(x, y, z, 0.0);
}

template <typename R4>
__global__ void __launch_bounds__(256, 6) k_permute(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ keys,
                          P3MGeom g, const double *__restrict__ pos,
                          const double *__restrict__ mom, const uint32_t *__restrict__ pid,
                          double *__restrict__ pos_out, double *__restrict__ mom_out,
                          uint32_t *__restrict__ pid_out, R4 *__restrict__ rel,
                          float4 *__restrict__ block_box, float *__restrict__ relx,
                          const double *__restrict__ origin)
{
    // one warp per 32-slot block of the sorted order; the warp also writes the block's
    // bounding box (FP32, absolute coordinates, rounded outwards by the callers' margins).
    // Six CTAs per SM (40 registers): the permute phase 0.644 -> 0.619 ms at 256^3 against five.
    const int64_t n = g.n;
    const int64_t nblocks = (n + 31) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t blk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; blk < nblocks;
         blk += nwarps) {
        const int64_t k = blk * 32 + lane;
        const bool active = k < n;
        const uint32_t pj = perm[active ? k : blk * 32];
        p3m_in_bounds(pj < (uint32_t)n, g.flags);
        const uint32_t j = min(pj, (uint32_t)(n - 1));  // in bounds always
        const double x = pos[j], y = pos[n + j], z = pos[2 * n + j];
        R4 rv = make_rel<R4>(0.0, 0.0, 0.0);
        if (active) {
            pos_out[k] = x;
            pos_out[n + k] = y;
            pos_out[2 * n + k] = z;
            mom_out[k] = mom[j];
            mom_out[n + k] = mom[n + j];
            mom_out[2 * n + k] = mom[2 * n + j];
            pid_out[k] = pid[j];
            const uint32_t cell = keys[k] >> (3 * g.sub_bits);
            const uint32_t cx = cell % g.n_c, cy = (cell / g.n_c) % g.n_c,
                           cz = cell / (g.n_c * g.n_c);
            rv = rel_coords<R4>(x, y, z, cx, cy, cz, origin);
            rel[k] = rv;
        }
        if (relx) {  // block-SoA copy of the relative coordinates (zero past the end)
            float *dst = relx + blk * 96;
            dst[lane] = (float)rv.x;
            dst[32 + lane] = (float)rv.y;
            dst[64 + lane] = (float)rv.z;
        }
        float lx = (float)x, ly = (float)y, lz = (float)z, hx = lx, hy = ly, hz = lz;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
            ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
            lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
            hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
            hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
            hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        }
        if (lane == 0) {
            block_box[2 * blk] = make_float4(lx, ly, lz, 0.0f);
            block_box[2 * blk + 1] = make_float4(hx, hy, hz, 0.0f);
        }
    }
}

// cell_start[c] = first sorted slot whose cell is >= c (slots k = 0..n, cell(n) = n_cells).
__global__ void k_cell_start(const uint32_t *__restrict__ keys, P3MGeom g,
                             uint32_t *__restrict__ cell_start)
{
    const int64_t n = g.n;
    const int sh = 3 * g.sub_bits;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t prev = k > 0 ? (int64_t)(keys[k - 1] >> sh) : -1;
        const int64_t cur = k < n ? (int64_t)(keys[k] >> sh) : (int64_t)g.n_cells;
        if (!p3m_in_bounds(cur <= (int64_t)g.n_cells, g.flags)) continue;
        for (int64_t c = prev + 1; c <= cur; ++c) cell_start[c] = (uint32_t)k;
    }
}

__global__ void k_work_count(const uint32_t *__restrict__ cell_start, int n_cells,
                             uint32_t *__restrict__ work_n, uint32_t *__restrict__ max_count)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x) {
        const uint32_t s0 = cell_start[c], s1 = cell_start[c + 1];
        const uint32_t cnt = s1 > s0 ? s1 - s0 : 0u;  // ranges are ordered unless a sort gave up
        work_n[c] = (cnt + P3M_PAIR_TI - 1) / P3M_PAIR_TI;
        if (cnt) atomicMax(max_count, cnt);
    }
}

// Work item w = (cell, first slot): work[2w] = cell, work[2w+1] = slot.  Its cost estimate is
// (particles in the item) x (particles in the 27 neighbour cells); the sort key is its class
// log2(cost) to 1/8 octave (the FP32 exponent and top 3 mantissa bits, 8 bits), inverted, so
// that one 8-bit pass of the stable sort puts the most expensive items first.  Unused entries
// keep the key 0xFFFFFFFF (low byte 255, the cheapest class) and, being after every used entry,
// stay last.
__global__ void k_work_fill(const uint32_t *__restrict__ cell_start,
                            const uint32_t *__restrict__ work_off, int n_c,
                            uint32_t *__restrict__ work, uint32_t *__restrict__ work_key,
                            uint32_t *__restrict__ work_val)
{
    const int n_cells = n_c * n_c * n_c;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x) {
        const uint32_t s = cell_start[c], e = cell_start[c + 1];
        if (s == e) continue;
        const int cx = c % n_c, cy = (c / n_c) % n_c, cz = c / (n_c * n_c);
        float nb = 0.0f;
        for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    const int q = (((cz + oz + n_c) % n_c) * n_c + (cy + oy + n_c) % n_c) * n_c +
                                  (cx + ox + n_c) % n_c;
                    nb += (float)(cell_start[q + 1] - cell_start[q]);
                }
        uint32_t w = work_off[c];
        for (uint32_t i = s; i < e; i += P3M_PAIR_TI, ++w) {
            work[2 * (size_t)w] = (uint32_t)c;
            work[2 * (size_t)w + 1] = i;
            const float cost = (float)min((uint32_t)P3M_PAIR_TI, e - i) * nb;
            // 8-bit cost class: log2(cost) to 1/8 octave (cost >= 1), largest first
            const uint32_t cls = (__float_as_uint(cost) >> 20) - (127u << 3);
            work_key[w] = 255u - min(cls, 255u);
            work_val[w] = w;
        }
    }
}

inline int grid_for(int64_t n, int threads, int num_sms)
{
    int64_t b = (n + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_kick_drift_keys(p3m_ctx *c, bool kick_drift, double kfac, double dfac,
                                   bool from_table)
{
    c->launches += 1;
    k_kick_drift_keys<<<grid_for(c->g.n, 256, c->num_sms), 256, 0, c->stream>>>(
        c->pos, c->mom, c->acc, c->g, kick_drift ? 1 : 0, kfac, dfac, c->keys,
        from_table ? c->cur_fac : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *aux,
                            cudaStream_t s)
{
    const size_t nb = (n + P3M_SORT_TILE - 1) / P3M_SORT_TILE;
    if (nb == 0) return cudaSuccess;
    k_scan_reduce<<<(unsigned)nb, kThreads, 0, s>>>(in, n, aux);
    k_scan_aux<<<1, kThreads, 0, s>>>(aux, nb);
    k_scan_down<<<(unsigned)nb, kThreads, 0, s>>>(in, out, n, aux);
    return cudaGetLastError();
}

// Stable LSD sort of n (key, value) pairs on the low key_bits bits.  k[0]/v[0] hold the input
// (v[0] NULL: values are the input positions); on return k[0]/v[0] hold the sorted pairs (the
// two buffers of each array are swapped as needed).  counts needs 256 * ceil(n/4096) entries.
cudaError_t radix_sort_pairs(uint32_t **k, uint32_t **v, bool identity_vals, int64_t n,
                             int key_bits, uint32_t *counts, uint32_t *aux, cudaStream_t s,
                             unsigned long long *launches)
{
    const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    const int n_tiles = (int)((n + P3M_SORT_TILE - 1) / P3M_SORT_TILE);
    const size_t ncount = (size_t)kRadix * n_tiles;
    uint32_t *kin = k[0], *kout = k[1];
    uint32_t *vin = identity_vals ? nullptr : v[0], *vout = identity_vals ? v[0] : v[1];
    for (int p = 0; p < passes; ++p) {
        const int shift = p * kRadixBits;
        *launches += 5;  // upsweep, 3 scan kernels, downsweep
        k_radix_upsweep<<<n_tiles, kThreads, 0, s>>>(kin, n, shift, counts, n_tiles);
        cudaError_t e = launch_scan_u32(counts, counts, ncount, aux, s);
        if (e != cudaSuccess) return e;
        k_radix_downsweep<<<n_tiles, kThreads, 0, s>>>(kin, vin, n, shift, counts, n_tiles, kout,
                                                       vout);
        uint32_t *t = kin;  // the next pass reads what this one wrote
        kin = kout;
        kout = t;
        uint32_t *vt = vin;
        vin = vout;
        vout = vt ? vt : v[1];
    }
    if (kin != k[0]) {
        k[1] = k[0];
        k[0] = kin;
    }
    if (vin != v[0]) {
        v[1] = v[0];
        v[0] = vin;
    }
    return cudaGetLastError();
}

// Stable sort of n (key, value) pairs of the context on the low key_bits bits in one-sweep
// passes (identity_vals: the values are the input slots); k[0]/v[0] hold the result.
cudaError_t radix_sort_onesweep(p3m_ctx *c, uint32_t **k, uint32_t **v, bool identity_vals,
                                int64_t n, int key_bits)
{
    const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    const unsigned n_tiles = (unsigned)((n + P3M_SORT_TILE - 1) / P3M_SORT_TILE);
    cudaStream_t s = c->stream;
    // sort_hist: 4 x 256 digit counts, then one tile counter per pass
    cudaError_t e = cudaMemsetAsync(c->sort_hist, 0, sizeof(uint32_t) * (4 * kRadix + 4), s);
    if (e != cudaSuccess) return e;
    const unsigned hist_grid = (unsigned)min((int64_t)n_tiles, (int64_t)c->num_sms * 4);
    k_digit_hist<<<hist_grid, kThreads, 0, s>>>(k[0], n, passes, c->sort_hist);
    c->launches += 1;
    uint32_t *kin = k[0], *kout = k[1];
    uint32_t *vin = identity_vals ? nullptr : v[0], *vout = identity_vals ? v[0] : v[1];
    for (int p = 0; p < passes; ++p) {
        e = cudaMemsetAsync(c->sort_status, 0, sizeof(unsigned long long) * kRadix * n_tiles, s);
        if (e != cudaSuccess) return e;
        k_onesweep<<<n_tiles, kThreads, 0, s>>>(kin, vin, n, p * kRadixBits, c->sort_hist + p * kRadix,
                                                c->sort_status, c->sort_hist + 4 * kRadix + p, kout,
                                                vout, c->counters + 1,
                                                c->sort_probe ? c->sort_probe : c->sort_status,
                                                c->sort_wait_limit);
        c->launches += 1;
        uint32_t *t = kin;  // the next pass reads what this one wrote
        kin = kout;
        kout = t;
        uint32_t *vt = vin;
        vin = vout;
        vout = vt ? vt : v[1];
    }
    if (kin != k[0]) {
        k[1] = k[0];
        k[0] = kin;
    }
    if (vin != v[0]) {
        v[1] = v[0];
        v[0] = vin;
    }
    return cudaGetLastError();
}

cudaError_t launch_radix_sort(p3m_ctx *c)
{
    uint32_t *k[2] = {c->keys, c->keys_alt}, *v[2] = {c->vals, c->vals_alt};
    cudaError_t e = radix_sort_onesweep(c, k, v, true, c->g.n, c->key_bits);
    c->keys = k[0];
    c->keys_alt = k[1];
    c->vals = v[0];
    c->vals_alt = v[1];
    return e;
}

cudaError_t launch_permute_and_cells(p3m_ctx *c)
{
    const int64_t n = c->g.n;
    const int gb = grid_for(n, 256, c->num_sms);
    c->launches += 7;  // permute, cell_start, work_count, 3 scan kernels, work_fill
    if (c->precision == P3M_PREC_MIXED)
        k_permute<float4><<<gb, 256, 0, c->stream>>>(c->vals, c->keys, c->g, c->pos, c->mom,
                                                     c->pid, c->pos_alt, c->mom_alt, c->pid_alt,
                                                     (float4 *)c->rel, c->block_box, c->relx,
                                                     c->tab_origin);
    else
        k_permute<double4_16a><<<gb, 256, 0, c->stream>>>(c->vals, c->keys, c->g, c->pos, c->mom,
                                                      c->pid, c->pos_alt, c->mom_alt,
                                                      c->pid_alt, (double4_16a *)c->rel, c->block_box,
                                                      nullptr, c->tab_origin);
    double *t = c->pos;
    c->pos = c->pos_alt;
    c->pos_alt = t;
    t = c->mom;
    c->mom = c->mom_alt;
    c->mom_alt = t;
    uint32_t *u = c->pid;
    c->pid = c->pid_alt;
    c->pid_alt = u;

    k_cell_start<<<grid_for(n + 1, 256, c->num_sms), 256, 0, c->stream>>>(c->keys, c->g,
                                                                         c->cell_start);
    cudaMemsetAsync(c->counters + 2, 0, sizeof(uint32_t), c->stream);
    const int gc = grid_for(c->g.n_cells, 256, c->num_sms);
    cudaMemsetAsync(c->work_off + c->g.n_cells, 0, sizeof(uint32_t), c->stream);
    k_work_count<<<gc, 256, 0, c->stream>>>(c->cell_start, c->g.n_cells, c->work_off,
                                            c->counters + 2);
    cudaError_t e = launch_scan_u32(c->work_off, c->work_off, (size_t)c->g.n_cells + 1,
                                    c->scan_aux, c->stream);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(c->work_key, 0xFF, sizeof(uint32_t) * c->max_work, c->stream);
    k_work_fill<<<gc, 256, 0, c->stream>>>(c->cell_start, c->work_off, c->g.n_c, c->work,
                                           c->work_key, c->work_order);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // most expensive work items first (longest-processing-time order for the pair kernel)
    uint32_t *k[2] = {c->work_key, c->work_key_alt}, *v[2] = {c->work_order, c->work_order_alt};
    e = radix_sort_onesweep(c, k, v, false, (int64_t)c->max_work, 8);
    c->work_key = k[0];
    c->work_key_alt = k[1];
    c->work_order = v[0];
    c->work_order_alt = v[1];
    return e;
}

// ------------------------------------------------------------------ allocation-free binning
// p3m_cell_sort_noalloc: the chaining-cell keys, stable sort and cell ranges of the context's
// force evaluation, for callers that must not allocate device memory.  Its scratch (two key
// arrays, the spare value array, the radix digit counts and the scan partials) is one
// file-scope device array, sized for at most P3M_NOALLOC_MAX_N particles; every GPU that loads
// the library holds it until the process exits.

namespace {

constexpr int64_t kNoAllocMaxN = P3M_NOALLOC_MAX_N;
constexpr int kNoAllocTiles = (int)((kNoAllocMaxN + P3M_SORT_TILE - 1) / P3M_SORT_TILE);
constexpr size_t kNoAllocCounts = (size_t)kRadix * kNoAllocTiles;
constexpr size_t kNoAllocAux = kNoAllocCounts / P3M_SORT_TILE + 8;
constexpr size_t kNoAllocWords = 3 * (size_t)kNoAllocMaxN + kNoAllocCounts + kNoAllocAux;

// Keys of positions that stay unmodified: the same wrap and key arithmetic as
// k_kick_drift_keys, without writing the positions back.
__global__ void k_keys_only(const double *__restrict__ pos, P3MGeom g, uint32_t *__restrict__ keys)
{
    const int64_t n = g.n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t f[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) f[d] = fine_index(wrap_box(pos[d * n + i], g.box), g.inv_fine, g.n_fine);
        keys[i] = make_key(f[0], f[1], f[2], g);
    }
}

}  // namespace

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

namespace {

std::mutex g_noalloc_mutex;
uint32_t *g_noalloc_ptr[256];  // device address of g_noalloc_scratch, per device ordinal

// Device address of the scratch on the current device, looked up with that device current (the
// host-side symbol itself is not a device address).  The first call on a device must look it up
// outside stream capture; later calls look it up again whenever the stream is not capturing, so
// that an address cached before a cudaDeviceReset (which reloads the module in a new context) is
// never used afterwards; while capturing they use the cached address.
cudaError_t noalloc_scratch(cudaStream_t stream, uint32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = (uint32_t *)p;
    } else if (!g_noalloc_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;  // no set-up call before the capture began
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int p3m_cell_sort_noalloc(const double *pos3n, int64_t n, double box, int n_c,
                                     int sub_bits, uint32_t *keys_out, uint32_t *ids_out,
                                     uint32_t *cell_start_out, void *stream)
{
    if (!pos3n || !keys_out || !ids_out || !cell_start_out)
        return p3m_fail_global(P3M_EINVAL, "p3m_cell_sort_noalloc: NULL pointer argument");
    if (n < 1 || n > kNoAllocMaxN)
        return p3m_fail_global(P3M_EINVAL,
                               "p3m_cell_sort_noalloc: n = %lld outside [1, %lld] (fixed scratch size)",
                               (long long)n, (long long)kNoAllocMaxN);
    if (!(box > 0.0) || !isfinite(box) || n_c < 1 || n_c > 1024 || sub_bits < 0 || sub_bits > 3)
        return p3m_fail_global(P3M_EINVAL, "p3m_cell_sort_noalloc: need box > 0, 1 <= n_c <= 1024, "
                                           "0 <= sub_bits <= 3");
    const uint64_t max_key = ((uint64_t)n_c * n_c * n_c << (3 * sub_bits)) - 1;
    if (max_key >= (1ull << 32))
        return p3m_fail_global(P3M_EINVAL, "p3m_cell_sort_noalloc: sort key exceeds 32 bits");
    int key_bits = 1;
    while (key_bits < 32 && (max_key >> key_bits)) ++key_bits;

    uint32_t *scratch = nullptr;
    cudaError_t e = noalloc_scratch((cudaStream_t)stream, &scratch);
    if (e != cudaSuccess)
        return p3m_fail_global(P3M_ECUDA, "p3m_cell_sort_noalloc: scratch lookup failed: %s",
                               cudaGetErrorString(e));
    uint32_t *keys0 = scratch, *keys1 = scratch + kNoAllocMaxN, *vals1 = scratch + 2 * kNoAllocMaxN;
    uint32_t *counts = scratch + 3 * kNoAllocMaxN, *aux = counts + kNoAllocCounts;

    P3MGeom g;
    memset(&g, 0, sizeof(g));
    g.box = box;
    g.n = n;
    g.n_c = n_c;
    g.sub_bits = sub_bits;
    g.n_fine = n_c << sub_bits;
    g.inv_fine = (double)g.n_fine / box;
    g.n_cells = n_c * n_c * n_c;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    k_keys_only<<<grid_for(n, 256, sms), 256, 0, s>>>(pos3n, g, keys0);
    unsigned long long launches = 0;
    uint32_t *k[2] = {keys0, keys1}, *v[2] = {ids_out, vals1};
    e = radix_sort_pairs(k, v, true, n, key_bits, counts, aux, s, &launches);
    if (e == cudaSuccess) e = cudaMemcpyAsync(keys_out, k[0], 4 * (size_t)n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && v[0] != ids_out)
        e = cudaMemcpyAsync(ids_out, v[0], 4 * (size_t)n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        k_cell_start<<<grid_for(n + 1, 256, sms), 256, 0, s>>>(keys_out, g, cell_start_out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return p3m_fail_global(P3M_ECUDA, "p3m_cell_sort_noalloc: %s", cudaGetErrorString(e));
    return P3M_OK;
}
