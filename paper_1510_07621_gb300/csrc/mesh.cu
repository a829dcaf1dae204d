// Particle-mesh part of the P3M force (the guide's PM_gridsize mesh, Ch. Parameters):
// CIC mass assignment, the fused k-space pass (Green's function with the Gaussian long-range
// filter of scale PM_scale, CIC deconvolution, spectral gradient) and the CIC interpolation
// of the three mesh accelerations back to the particles.  cuFFT does the transforms.
//
// Mesh layout: M^3 values, node (ix, iy, iz) at ((ix*M + iy)*M + iz), node positions i*h.
// Spectrum layout (cuFFT R2C): M * M * (M/2+1) complex values, z fastest.
#include <cuda_runtime.h>
#include <cufft.h>
#include <limits.h>
#include <math.h>

#include <mutex>

#include "p3m_internal.cuh"

namespace {

__device__ __forceinline__ int wrap_index(int i, int M)
{
    i %= M;
    return i < 0 ? i + M : i;
}

// CIC stencil of a wrapped position: base node i0 = floor(x M/L) and fraction f.
template <typename T>
__device__ __forceinline__ void cic_stencil(double x, double inv_h, int &i0, T &f)
{
    const double u = __dmul_rn(x, inv_h);
    const double fl = floor(u);
    i0 = (int)fl;
    f = (T)(u - fl);
}

// CIC stencil of a sorted particle in FP32 from its cell-relative coordinates (FP32 mode).  The
// node coordinate is u = c M/n_c + rel M/L for cell coordinate c; c M = q n_c + r is split in
// integers, so only v = r/n_c + rel M/L (below 1 + M/n_c) is rounded to FP32: i0 = q + floor(v),
// f = v - floor(v).  CIC weights are continuous across node planes, so a rounding that moves
// floor(v) by one at a plane changes the weights by the same rounding only.
__device__ __forceinline__ void cic_stencil_rel(const float4 rv, uint32_t cell, const P3MGeom &g,
                                                float inv_h, float inv_nc, int i0[3], float f[3])
{
    const int nc = g.n_c, M = g.mesh;
    const int cc[3] = {(int)(cell % (uint32_t)nc), (int)((cell / (uint32_t)nc) % (uint32_t)nc),
                       (int)(cell / (uint32_t)(nc * nc))};
    const float rr[3] = {rv.x, rv.y, rv.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int cm = cc[d] * M;
        const int q = cm / nc, r = cm - q * nc;
        const float v = fmaf(rr[d], inv_h, (float)r * inv_nc);
        const float fl = floorf(v);
        i0[d] = q + (int)fl;
        f[d] = v - fl;
    }
}

// Fixed-point mass: every CIC weight (or run sum of weights) is rounded once to an integer
// multiple of 2^-S and added as a 64-bit integer.  Integer addition is associative, so the
// mesh does not depend on the order in which the atomics land: two runs give the same bits.
// FP32 mode: S = 32 (weights are FP32 values, so 2^-33 is below their own rounding); FP64
// mode: S = 62 - bit length of N, the finest scale at which N unit masses on one node still fit.
template <typename T>
__device__ __forceinline__ unsigned long long to_fixed(T w, T scale);
template <>
__device__ __forceinline__ unsigned long long to_fixed<float>(float w, float scale)
{
    return __float2ull_rn(w * scale);
}
template <>
__device__ __forceinline__ unsigned long long to_fixed<double>(double w, double scale)
{
    return __double2ull_rn(w * scale);
}

// Fixed-size chunks of the sorted particles (CTA b takes slots [b*512, (b+1)*512)), so that a
// dense cell is spread over many CTAs.  The chunk's CIC nodes are accumulated in a shared-memory
// tile spanning the chunk's node bounding box (found by a block reduction); the tile is then
// added to the mesh with one global atomic per non-zero node.  A chunk whose box exceeds the
// tile capacity (e.g. one that straddles the periodic boundary) adds its 8 weights per particle
// straight to the mesh.  All sums are 64-bit fixed-point integers (to_fixed).  64-bit
// shared-memory atomics are slow, so in the FP32 mode every 2^-32 fixed-point addend v is split
// into v >> 16 and v & 0xFFFF, added by 32-bit atomics to two tiles (high and low); the tile
// node is then (high << 16) + low, exactly the 64-bit sum.  Neither tile can overflow: a node
// takes at most one addend per particle of the chunk (runs of equal-base lanes are summed first),
// at most 512 of weight at most 1 + 2^-20 each, so high < 2^26 and low < 2^25.  With the split
// tiles every chunk that fits uses its tile; against 64-bit tiles for dense chunks only (sparse
// chunks through global atomics): evolved 128^3 0.151 -> 0.079 ms, synthetic clustered 0.155 ->
// 0.083 ms, 256^3 near-uniform 0.480 -> 0.417 ms, 512^3 3.73 -> 3.13 ms (64-bit tiles for every
// chunk were slower than the global atomics: 0.187, 0.190 and 0.594 ms).  The FP64 mode (2^-S
// with S up to 62 - bit length of N) keeps 64-bit tiles, for dense chunks only.
// Six CTAs per SM (at most 40 registers, a few bytes of spills, and the largest shared-memory
// carveout, set once per process by mesh_set_attributes): 256^3 near-uniform 0.415 -> 0.370 ms,
// evolved 128^3 0.079 -> 0.077 ms against four CTAs per SM.
constexpr int kDepChunk = 512;
constexpr int kDepTileMax = 4096;  // nodes

template <typename T>
__global__ void __launch_bounds__(256, 6)
    k_deposit_chunks(const double *__restrict__ pos, const float4 *__restrict__ rel,
                     const uint32_t *__restrict__ keys, P3MGeom g, T scale,
                     unsigned long long *__restrict__ fix)
{
    // rel != nullptr (FP32 mode, sorted state fresh): FP32 stencils from rel and the keys' cells
    const float inv_h_f = (float)g.inv_h, inv_nc = 1.0f / (float)g.n_c;
    const int csh = 3 * g.sub_bits;
    __shared__ union {
        unsigned long long u64[kDepTileMax];    // FP64 mode: 64-bit tile
        unsigned int u32[2][kDepTileMax];       // FP32 mode: high and low tiles
    } tiles;
    unsigned long long *const tile = tiles.u64;
    __shared__ int s_lo[3][8], s_hi[3][8];
    constexpr bool k32 = sizeof(T) == 4;  // split 32-bit tiles (FP32 mode)
    unsigned int *const tile_hi = tiles.u32[0], *const tile_lo = tiles.u32[1];
    const int M = g.mesh;
    const int64_t n = g.n;
    const int64_t base = (int64_t)blockIdx.x * kDepChunk;
    constexpr int per = kDepChunk / 256;
    int i0[per][3];
    T f[per][3];
    bool act[per];
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
#pragma unroll
    for (int r = 0; r < per; ++r) {
        const int64_t k = base + r * 256 + threadIdx.x;
        act[r] = k < n;
        if (act[r] && sizeof(T) == 4 && rel) {
            int ii[3];
            float ff[3];
            cic_stencil_rel(rel[k], keys[k] >> csh, g, inv_h_f, inv_nc, ii, ff);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                i0[r][d] = ii[d];
                f[r][d] = (T)ff[d];
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (act[r]) {
                if (!(sizeof(T) == 4 && rel)) cic_stencil(pos[d * n + k], g.inv_h, i0[r][d], f[r][d]);
                lo[d] = min(lo[d], i0[r][d]);
                hi[d] = max(hi[d], i0[r][d] + 1);
            } else {
                i0[r][d] = 0;
                f[r][d] = T(0);
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
        if (lane == 0) {
            s_lo[d][warp] = lo[d];
            s_hi[d][warp] = hi[d];
        }
    }
    __syncthreads();
    int blo[3], bdim[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int a = INT_MAX, b = INT_MIN;
        for (int w = 0; w < 8; ++w) {
            a = min(a, s_lo[d][w]);
            b = max(b, s_hi[d][w]);
        }
        blo[d] = a;
        bdim[d] = b - a + 1;
    }
    const long long vol = (long long)bdim[0] * bdim[1] * bdim[2];
    if (vol <= kDepTileMax && (k32 || vol <= kDepChunk)) {
        for (int t = threadIdx.x; t < vol; t += 256) {
            if (k32)
                tile_hi[t] = tile_lo[t] = 0u;
            else
                tile[t] = 0ull;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < per; ++r) {
            // the warp's 32 particles are consecutive in the sorted order; lanes whose base
            // nodes agree form runs of consecutive lanes
            const int lx = i0[r][0] - blo[0], ly = i0[r][1] - blo[1], lz = i0[r][2] - blo[2];
            const int key = act[r] ? (lx * bdim[1] + ly) * bdim[2] + lz : -1 - lane;
            const int prev = __shfl_up_sync(0xffffffffu, key, 1);
            const uint32_t heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
            const T wx[2] = {T(1) - f[r][0], f[r][0]}, wy[2] = {T(1) - f[r][1], f[r][1]};
            const T wz[2] = {T(1) - f[r][2], f[r][2]};
            T w[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) w[c] = wx[c >> 2] * wy[(c >> 1) & 1] * wz[c & 1];
            if (__popc(heads) <= 8) {
                // few runs (dense region): each run's weights summed onto its first lane by a
                // segmented reduction (a fixed order of additions for a given particle order),
                // then one set of 8 shared-memory atomics per run
                const int rid = __popc(heads & ((2u << lane) - 1u));
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int rid_o = __shfl_down_sync(0xffffffffu, rid, off);
                    const bool same = lane + off < 32 && rid_o == rid;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const T o = __shfl_down_sync(0xffffffffu, w[c], off);
                        if (same) w[c] += o;
                    }
                }
                if (!(act[r] && ((heads >> lane) & 1u))) continue;
            } else if (!act[r]) {
                continue;
            }
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const long long t = ((lx + a) * bdim[1] + (ly + b)) * bdim[2] + lz;
                    if (!p3m_in_bounds(t >= 0 && t + 1 < vol, g.flags)) continue;
                    const unsigned long long v0 = to_fixed(w[(a << 2) | (b << 1)], scale);
                    const unsigned long long v1 = to_fixed(w[(a << 2) | (b << 1) | 1], scale);
                    if (k32) {
                        atomicAdd(tile_hi + t, (unsigned int)(v0 >> 16));
                        atomicAdd(tile_lo + t, (unsigned int)(v0 & 0xFFFFu));
                        atomicAdd(tile_hi + t + 1, (unsigned int)(v1 >> 16));
                        atomicAdd(tile_lo + t + 1, (unsigned int)(v1 & 0xFFFFu));
                    } else {
                        atomicAdd(tile + t, v0);
                        atomicAdd(tile + t + 1, v1);
                    }
                }
        }
        __syncthreads();
        // t -> (lx, ly, lz) by FP32 reciprocals: for t, bdim < 2^12 the rounded quotient
        // (t + 1/2) / bdim is off by far less than its distance 1/(2 bdim) to an integer.  Node
        // indices lie in [-1, M + 1], so one conditional add or subtract wraps them.
        const float inv_z = 1.0f / (float)bdim[2], inv_y = 1.0f / (float)bdim[1];
        for (int t = threadIdx.x; t < vol; t += 256) {
            const unsigned long long v =
                k32 ? ((unsigned long long)tile_hi[t] << 16) + tile_lo[t] : tile[t];
            if (v == 0ull) continue;
            const int row = (int)(((float)t + 0.5f) * inv_z), lz = t - row * bdim[2];
            const int lx = (int)(((float)row + 0.5f) * inv_y), ly = row - lx * bdim[1];
            int wx = blo[0] + lx, wy = blo[1] + ly, wz = blo[2] + lz;
            wx += wx < 0 ? M : (wx >= M ? -M : 0);
            wy += wy < 0 ? M : (wy >= M ? -M : 0);
            wz += wz < 0 ? M : (wz >= M ? -M : 0);
            const size_t node = ((size_t)wx * M + wy) * M + wz;
            if (p3m_in_bounds(node < (size_t)M * M * M, g.flags)) atomicAdd(fix + node, v);
        }
    } else {
#pragma unroll
        for (int r = 0; r < per; ++r) {
            if (!act[r]) continue;
            const T wx[2] = {T(1) - f[r][0], f[r][0]}, wy[2] = {T(1) - f[r][1], f[r][1]};
            const T wz[2] = {T(1) - f[r][2], f[r][2]};
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const size_t node = ((size_t)wrap_index(i0[r][0] + a, M) * M +
                                             wrap_index(i0[r][1] + b, M)) * M + wrap_index(i0[r][2] + c, M);
                        if (p3m_in_bounds(node < (size_t)M * M * M, g.flags))
                            atomicAdd(fix + node, to_fixed(wx[a] * wy[b] * wz[c], scale));
                    }
        }
    }
}

// mesh = fix 2^-S - mean, two nodes per thread (M^3 is even), one pass over the mesh.  FP32
// mode (S = 32): the high and low 32-bit words convert exactly or with one rounding each,
// (hi - mean) + lo 2^-32 rounds twice, so the result is within about one FP32 unit of the exact
// value.  FP64 mode: one conversion and one FMA.  The accumulator is only read here; the
// deposit clears it beforehand.
__global__ void __launch_bounds__(256)
    k_fix_to_mesh_f32(const ulonglong2 *__restrict__ fix, size_t n2, float mean, float2 *__restrict__ mesh)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n2) return;
    const ulonglong2 v = fix[i];
    float2 o;
    o.x = fmaf(__uint2float_rn((uint32_t)v.x), 0x1p-32f, __uint2float_rn((uint32_t)(v.x >> 32)) - mean);
    o.y = fmaf(__uint2float_rn((uint32_t)v.y), 0x1p-32f, __uint2float_rn((uint32_t)(v.y >> 32)) - mean);
    mesh[i] = o;
}

__global__ void __launch_bounds__(256)
    k_fix_to_mesh_f64(const ulonglong2 *__restrict__ fix, size_t n2, double inv_scale, double mean,
                      double2 *__restrict__ mesh)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n2) return;
    const ulonglong2 v = fix[i];
    mesh[i] = make_double2(fma(__ull2double_rn(v.x), inv_scale, -mean),
                           fma(__ull2double_rn(v.y), inv_scale, -mean));
}

// Fused k-space pass: G(k) = C * t(kx) t(ky) t(kz) / k^2 with t the per-axis Gaussian filter
// and deconvolution factor, then F_d = -i kg_d G rho_k for the three axes.
template <typename T, typename C2>
__global__ void __launch_bounds__(256)
    k_kspace(const C2 *__restrict__ rho_k, const T *__restrict__ tk, const T *__restrict__ tkg,
             const T *__restrict__ tg, int M, T gconst, C2 *__restrict__ fx,
             C2 *__restrict__ fy, C2 *__restrict__ fz)
{
    const int nz = M / 2 + 1;
    const size_t total = (size_t)M * M * nz;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int iz = (int)(idx % nz);
        const size_t t = idx / nz;
        const int iy = (int)(t % M), ix = (int)(t / M);
        const T kx = tk[ix], ky = tk[iy], kz = tk[iz];
        const T k2 = kx * kx + ky * ky + kz * kz;
        const T G = idx == 0 ? T(0) : gconst * (tg[ix] * tg[iy] * tg[iz]) / k2;
        const C2 r = rho_k[idx];
        const T gx = G * tkg[ix], gy = G * tkg[iy], gz = G * tkg[iz];
        C2 o;
        o.x = gx * r.y;
        o.y = -gx * r.x;
        fx[idx] = o;
        o.x = gy * r.y;
        o.y = -gy * r.x;
        fy[idx] = o;
        o.x = gz * r.y;
        o.y = -gz * r.x;
        fz[idx] = o;
    }
}

// CIC interpolation of the three mesh accelerations at the particles.  FP32 mode: the stencil
// comes from the cell-relative coordinates (right after the permute).  When the three force
// meshes do not fit in L2, k_gather_f32_staged takes a chunk of 512 consecutive sorted
// particles per CTA: it finds the chunk's node bounding box (block reduction), copies that box
// of the three meshes into shared memory, and interpolates from there.  24 scattered global
// loads per particle (8 nodes x 3 meshes) kept the L1 request pipeline saturated at large
// meshes (256^3: 0.51 -> 0.38 ms, 512^3: 4.6 -> 3.3 ms).  With the meshes in L2, the direct
// loads of k_gather_f32 were faster (evolved 128^3: 0.047 against 0.051 ms); a chunk whose box
// exceeds the tile (one that straddles the periodic boundary or spans sparse cells) reads the
// meshes directly too.  Every path adds the same products in the same order, so the result
// does not depend on the path.  FP64 mode: the stencil from the FP64 positions.  (Writing the
// three C2R outputs interleaved per node, so that a node is one 16-byte load, made a direct
// gather 34 % faster at 256^3 but the strided C2R 2.3x slower: not kept.)
constexpr int kGatherChunk = 512;
constexpr int kGatherTileMax = 2048;  // nodes (three FP32 meshes: 24 KB)

// the chunk's node bounding box (origin blo, extent bdim) from the threads' stencil bounds
__device__ __forceinline__ void chunk_box(int lo[3], int hi[3], int blo[3], int bdim[3])
{
    __shared__ int s_lo[3][8], s_hi[3][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
        if (lane == 0) {
            s_lo[d][warp] = lo[d];
            s_hi[d][warp] = hi[d];
        }
    }
    __syncthreads();
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int a = INT_MAX, b = INT_MIN;
        for (int w = 0; w < 8; ++w) {
            a = min(a, s_lo[d][w]);
            b = max(b, s_hi[d][w]);
        }
        blo[d] = a;
        bdim[d] = b - a + 1;  // (no active particle: a > b, bdim <= 0)
    }
}

__global__ void __launch_bounds__(256)
    k_gather_f32_staged(const float4 *__restrict__ rel, const uint32_t *__restrict__ keys, P3MGeom g,
                        const float *__restrict__ fxm, const float *__restrict__ fym,
                        const float *__restrict__ fzm, double *__restrict__ acc)
{
    __shared__ float tile[3][kGatherTileMax];
    const int M = g.mesh;
    const int64_t n = g.n;
    const float inv_h_f = (float)g.inv_h, inv_nc = 1.0f / (float)g.n_c;
    const int csh = 3 * g.sub_bits;
    const int64_t base = (int64_t)blockIdx.x * kGatherChunk;
    constexpr int per = kGatherChunk / 256;
    int i0[per][3];
    float f[per][3];
    bool act[per];
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
#pragma unroll
    for (int r = 0; r < per; ++r) {
        const int64_t k = base + r * 256 + threadIdx.x;
        act[r] = k < n;
        int ii[3] = {0, 0, 0};
        float ff[3] = {0.0f, 0.0f, 0.0f};
        if (act[r]) cic_stencil_rel(rel[k], keys[k] >> csh, g, inv_h_f, inv_nc, ii, ff);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            i0[r][d] = ii[d];
            f[r][d] = ff[d];
            if (act[r]) {
                lo[d] = min(lo[d], ii[d]);
                hi[d] = max(hi[d], ii[d] + 1);
            }
        }
    }
    int blo[3], bdim[3];
    chunk_box(lo, hi, blo, bdim);
    const long long vol = (long long)bdim[0] * bdim[1] * bdim[2];
    if (bdim[0] > 0 && vol <= kGatherTileMax) {
        // t -> (lx, ly, lz) by FP32 reciprocals: for t, bdim < 2^11 the rounded quotient
        // (t + 1/2) / bdim is off by far less than its distance 1/(2 bdim) to an integer.  Node
        // indices lie in [-1, M + 1], so one conditional add or subtract wraps them.
        const float inv_z = 1.0f / (float)bdim[2], inv_y = 1.0f / (float)bdim[1];
        for (int t = threadIdx.x; t < vol; t += 256) {
            const int row = (int)(((float)t + 0.5f) * inv_z), lz = t - row * bdim[2];
            const int lx = (int)(((float)row + 0.5f) * inv_y), ly = row - lx * bdim[1];
            int wx = blo[0] + lx, wy = blo[1] + ly, wz = blo[2] + lz;
            wx += wx < 0 ? M : (wx >= M ? -M : 0);
            wy += wy < 0 ? M : (wy >= M ? -M : 0);
            wz += wz < 0 ? M : (wz >= M ? -M : 0);
            const size_t node = ((size_t)wx * M + wy) * M + wz;
            const bool ok = p3m_in_bounds(node < (size_t)M * M * M, g.flags);
            tile[0][t] = ok ? __ldg(fxm + node) : 0.0f;
            tile[1][t] = ok ? __ldg(fym + node) : 0.0f;
            tile[2][t] = ok ? __ldg(fzm + node) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < per; ++r) {
            if (!act[r]) continue;
            const int64_t k = base + r * 256 + threadIdx.x;
            const float wx[2] = {1.0f - f[r][0], f[r][0]}, wy[2] = {1.0f - f[r][1], f[r][1]},
                        wz[2] = {1.0f - f[r][2], f[r][2]};
            const int lx = i0[r][0] - blo[0], ly = i0[r][1] - blo[1], lz = i0[r][2] - blo[2];
            float ax = 0.0f, ay = 0.0f, az = 0.0f;
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const float w = wx[a] * wy[b] * wz[c];
                        const int t = ((lx + a) * bdim[1] + (ly + b)) * bdim[2] + lz + c;
                        if (!p3m_in_bounds(t >= 0 && t < vol, g.flags)) continue;
                        ax += w * tile[0][t];
                        ay += w * tile[1][t];
                        az += w * tile[2][t];
                    }
            acc[k] = (double)ax;
            acc[n + k] = (double)ay;
            acc[2 * n + k] = (double)az;
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < per; ++r) {
        if (!act[r]) continue;
        const int64_t k = base + r * 256 + threadIdx.x;
        const float wx[2] = {1.0f - f[r][0], f[r][0]}, wy[2] = {1.0f - f[r][1], f[r][1]},
                    wz[2] = {1.0f - f[r][2], f[r][2]};
        const int jx[2] = {wrap_index(i0[r][0], M), wrap_index(i0[r][0] + 1, M)};
        const int jy[2] = {wrap_index(i0[r][1], M), wrap_index(i0[r][1] + 1, M)};
        const int jz[2] = {wrap_index(i0[r][2], M), wrap_index(i0[r][2] + 1, M)};
        float ax = 0.0f, ay = 0.0f, az = 0.0f;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float w = wx[a] * wy[b] * wz[c];
                    const size_t node = ((size_t)jx[a] * M + jy[b]) * M + jz[c];
                    if (!p3m_in_bounds(node < (size_t)M * M * M, g.flags)) continue;
                    ax += w * __ldg(fxm + node);
                    ay += w * __ldg(fym + node);
                    az += w * __ldg(fzm + node);
                }
        acc[k] = (double)ax;
        acc[n + k] = (double)ay;
        acc[2 * n + k] = (double)az;
    }
}

// The direct FP32 gather (meshes in L2): one particle per thread, grid-stride.
__global__ void __launch_bounds__(256)
    k_gather_f32(const float4 *__restrict__ rel, const uint32_t *__restrict__ keys, P3MGeom g,
                 const float *__restrict__ fxm, const float *__restrict__ fym,
                 const float *__restrict__ fzm, double *__restrict__ acc)
{
    const int M = g.mesh;
    const int64_t n = g.n;
    const float inv_h_f = (float)g.inv_h, inv_nc = 1.0f / (float)g.n_c;
    const int csh = 3 * g.sub_bits;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int ii[3];
        float ff[3];
        cic_stencil_rel(rel[k], keys[k] >> csh, g, inv_h_f, inv_nc, ii, ff);
        const float wx[2] = {1.0f - ff[0], ff[0]}, wy[2] = {1.0f - ff[1], ff[1]},
                    wz[2] = {1.0f - ff[2], ff[2]};
        const int jx[2] = {wrap_index(ii[0], M), wrap_index(ii[0] + 1, M)};
        const int jy[2] = {wrap_index(ii[1], M), wrap_index(ii[1] + 1, M)};
        const int jz[2] = {wrap_index(ii[2], M), wrap_index(ii[2] + 1, M)};
        float ax = 0.0f, ay = 0.0f, az = 0.0f;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float w = wx[a] * wy[b] * wz[c];
                    const size_t node = ((size_t)jx[a] * M + jy[b]) * M + jz[c];
                    if (!p3m_in_bounds(node < (size_t)M * M * M, g.flags)) continue;
                    ax += w * __ldg(fxm + node);
                    ay += w * __ldg(fym + node);
                    az += w * __ldg(fzm + node);
                }
        acc[k] = (double)ax;
        acc[n + k] = (double)ay;
        acc[2 * n + k] = (double)az;
    }
}

__global__ void __launch_bounds__(256)
    k_gather_f64(const double *__restrict__ pos, P3MGeom g, const double *__restrict__ fxm,
                 const double *__restrict__ fym, const double *__restrict__ fzm, double *__restrict__ acc)
{
    const int M = g.mesh;
    const int64_t n = g.n;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        double fx, fy, fz;
        cic_stencil(pos[k], g.inv_h, ix, fx);
        cic_stencil(pos[n + k], g.inv_h, iy, fy);
        cic_stencil(pos[2 * n + k], g.inv_h, iz, fz);
        const double wx[2] = {1.0 - fx, fx}, wy[2] = {1.0 - fy, fy}, wz[2] = {1.0 - fz, fz};
        const int jx[2] = {wrap_index(ix, M), wrap_index(ix + 1, M)};
        const int jy[2] = {wrap_index(iy, M), wrap_index(iy + 1, M)};
        const int jz[2] = {wrap_index(iz, M), wrap_index(iz + 1, M)};
        double ax = 0, ay = 0, az = 0;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const double w = wx[a] * wy[b] * wz[c];
                    const size_t node = ((size_t)jx[a] * M + jy[b]) * M + jz[c];
                    if (!p3m_in_bounds(node < (size_t)M * M * M, g.flags)) continue;
                    ax += w * __ldg(fxm + node);
                    ay += w * __ldg(fym + node);
                    az += w * __ldg(fzm + node);
                }
        acc[k] = ax;
        acc[n + k] = ay;
        acc[2 * n + k] = az;
    }
}

// Power spectrum binning over the R2C half spectrum of the count mesh minus its mean:
// delta_k = rho_k / N; every mode (ix, iy, iz) stands for itself and, for 0 < iz < M/2, for its
// conjugate partner (weight 2).  Shell b = round(|n|) - 1 accumulates w |delta_k|^2 / W^2,
// w |k| and w; with radius > 0 the top-hat sum w |delta_k|^2 / W^2 W_TH(|k| R)^2 goes to
// row entry 3 n_bins.  The additions happen in an order fixed by the launch shape alone: the
// lanes of a warp that hold modes of one shell are summed in lane order by the lowest of them,
// which adds the sums to its warp's private shared-memory row; the block adds its warps' rows in
// warp order into its row of part[], and k_powspec_final adds the blocks' rows in block order.
// So every run gives the same bits.
template <typename C2>
__global__ void __launch_bounds__(128)
    k_powspec(const C2 *__restrict__ rk, int M, const double *__restrict__ inv_w2, double kf,
              double inv_n2, double radius, int n_bins, double *__restrict__ part)
{
    extern __shared__ double sacc[];  // (blockDim / 32) rows of 3 n_bins + 1
    const int nacc = 3 * n_bins + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double *mine = sacc + (size_t)warp * nacc;
    for (int t = lane; t < nacc; t += 32) mine[t] = 0.0;
    __syncwarp();
    const int nz = M / 2 + 1;
    const size_t total = (size_t)M * M * nz;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = ((size_t)blockIdx.x * nw + warp) * 32; base < total; base += stride) {
        const size_t idx = base + lane;
        int b = -1;
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, vt = 0.0;
        if (idx < total && idx != 0) {
            const int iz = (int)(idx % nz);
            const size_t t = idx / nz;
            const int iy = (int)(t % M), ix = (int)(t / M);
            const int sx = ix <= M / 2 ? ix : ix - M, sy = iy <= M / 2 ? iy : iy - M;
            const double w = (iz == 0 || iz == M / 2) ? 1.0 : 2.0;
            const double nk = sqrt((double)sx * sx + (double)sy * sy + (double)iz * iz);
            const C2 r = rk[idx];
            const double p = ((double)r.x * r.x + (double)r.y * r.y) * inv_n2 * inv_w2[ix] *
                             inv_w2[iy] * inv_w2[iz];
            b = (int)floor(nk + 0.5) - 1;
            if (b >= n_bins) b = -1;
            v0 = w * p;
            v1 = w * nk * kf;
            v2 = w;
            if (radius > 0.0) {
                const double x = nk * kf * radius;
                const double wt = x < 1e-3 ? 1.0 - x * x / 10.0 : 3.0 * (sin(x) - x * cos(x)) / (x * x * x);
                vt = w * p * wt * wt;
            }
        }
        const unsigned grp = __match_any_sync(0xffffffffu, b);
        if (b >= 0) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            for (unsigned m = grp; m; m &= m - 1u) {
                const int src = __ffs(m) - 1;
                s0 += __shfl_sync(grp, v0, src);
                s1 += __shfl_sync(grp, v1, src);
                s2 += __shfl_sync(grp, v2, src);
            }
            if (lane == __ffs(grp) - 1) {
                mine[3 * b] += s0;
                mine[3 * b + 1] += s1;
                mine[3 * b + 2] += s2;
            }
        }
        if (radius > 0.0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) vt += __shfl_xor_sync(0xffffffffu, vt, o);
            if (lane == 0) mine[3 * n_bins] += vt;
        }
        __syncwarp();
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nacc; t += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sacc[(size_t)w * nacc + t];
        part[(size_t)blockIdx.x * nacc + t] = s;
    }
}

__global__ void k_powspec_final(const double *__restrict__ part, int blocks, int nacc,
                                double *__restrict__ acc)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nacc; t += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < blocks; ++b) s += part[(size_t)b * nacc + t];
        acc[t] = s;
    }
}

inline int grid_for(size_t n, int threads, int num_sms)
{
    size_t b = (n + threads - 1) / threads;
    size_t cap = (size_t)num_sms * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

// Bit length of n (the S of the FP64 mode's fixed point is 62 minus it).
int bit_length(int64_t n)
{
    int b = 0;
    while (b < 63 && (n >> b)) ++b;
    return b;
}

template <typename T>
cudaError_t deposit_impl(p3m_ctx *c, bool from_rel)
{
    const size_t M3 = (size_t)c->g.mesh * c->g.mesh * c->g.mesh;
    const bool f32 = sizeof(T) == 4;
    const int S = f32 ? 32 : 62 - bit_length(c->g.n);
    c->launches += 2;  // deposit, conversion (and the clearing memset)
    cudaError_t e = cudaMemsetAsync(c->rho_fix, 0, sizeof(unsigned long long) * M3, c->stream);
    if (e != cudaSuccess) return e;
    const int64_t chunks = (c->g.n + kDepChunk - 1) / kDepChunk;
    k_deposit_chunks<T><<<(unsigned)chunks, 256, 0, c->stream>>>(
        c->pos, from_rel && c->precision == P3M_PREC_MIXED ? (const float4 *)c->rel : nullptr,
        c->keys, c->g, (T)ldexp(1.0, S), c->rho_fix);
    const size_t n2 = M3 / 2;  // M is even
    const unsigned grid = (unsigned)((n2 + 255) / 256);
    if (f32)
        k_fix_to_mesh_f32<<<grid, 256, 0, c->stream>>>((const ulonglong2 *)c->rho_fix, n2,
                                                       (float)c->g.mean_count, (float2 *)c->rho);
    else
        k_fix_to_mesh_f64<<<grid, 256, 0, c->stream>>>((const ulonglong2 *)c->rho_fix, n2, ldexp(1.0, -S),
                                                       c->g.mean_count, (double2 *)c->rho);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_deposit(p3m_ctx *c, bool from_rel)
{
    return c->precision == P3M_PREC_MIXED ? deposit_impl<float>(c, from_rel) : deposit_impl<double>(c, false);
}

cudaError_t launch_kspace(p3m_ctx *c)
{
    const int M = c->g.mesh;
    const size_t nk = (size_t)M * M * (M / 2 + 1);
    const int grid = grid_for(nk, 256, c->num_sms);
    c->launches += 1;
    if (c->precision == P3M_PREC_MIXED) {
        cufftComplex *f = (cufftComplex *)c->frc_k;
        k_kspace<float, cufftComplex><<<grid, 256, 0, c->stream>>>(
            (const cufftComplex *)c->rho_k, (const float *)c->tab_k, (const float *)c->tab_kg,
            (const float *)c->tab_g, M, (float)c->green_const, f, f + nk, f + 2 * nk);
    } else {
        cufftDoubleComplex *f = (cufftDoubleComplex *)c->frc_k;
        k_kspace<double, cufftDoubleComplex><<<grid, 256, 0, c->stream>>>(
            (const cufftDoubleComplex *)c->rho_k, (const double *)c->tab_k,
            (const double *)c->tab_kg, (const double *)c->tab_g, M, c->green_const, f, f + nk,
            f + 2 * nk);
    }
    return cudaGetLastError();
}

cudaError_t launch_powspec(p3m_ctx *c, const double *inv_w2, double radius, int n_bins, double *acc)
{
    const int M = c->g.mesh;
    const int nacc = 3 * n_bins + 1, threads = 128;
    const size_t smem = sizeof(double) * (size_t)nacc * (threads / 32);
    const double kf = 2.0 * M_PI / c->g.box;
    const double inv_n2 = 1.0 / ((double)c->g.n * (double)c->g.n);
    c->launches += 2;
    cudaError_t e = cudaSuccess;
    if (c->precision == P3M_PREC_MIXED) {
        if (smem > 48 * 1024)
            e = cudaFuncSetAttribute(k_powspec<cufftComplex>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        if (e != cudaSuccess) return e;
        k_powspec<cufftComplex><<<c->ps_blocks, threads, smem, c->stream>>>(
            (const cufftComplex *)c->rho_k, M, inv_w2, kf, inv_n2, radius, n_bins, c->ps_part);
    } else {
        if (smem > 48 * 1024)
            e = cudaFuncSetAttribute(k_powspec<cufftDoubleComplex>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_powspec<cufftDoubleComplex><<<c->ps_blocks, threads, smem, c->stream>>>(
            (const cufftDoubleComplex *)c->rho_k, M, inv_w2, kf, inv_n2, radius, n_bins, c->ps_part);
    }
    k_powspec_final<<<(nacc + 255) / 256, 256, 0, c->stream>>>(c->ps_part, c->ps_blocks, nacc, acc);
    return cudaGetLastError();
}

cudaError_t mesh_set_attributes()
{
    static cudaError_t done = cudaErrorNotReady;  // once per process; never inside a capture
    static std::once_flag once;
    std::call_once(once, [] {
        done = cudaFuncSetAttribute(k_deposit_chunks<float>,
                                    cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared);
        if (done == cudaSuccess)
            done = cudaFuncSetAttribute(k_deposit_chunks<double>,
                                        cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared);
    });
    return done;
}

cudaError_t launch_gather(p3m_ctx *c, double *acc_out)
{
    const size_t M3 = (size_t)c->g.mesh * c->g.mesh * c->g.mesh;
    const int grid = grid_for(c->g.n, 256, c->num_sms);
    c->launches += 1;
    if (c->precision == P3M_PREC_MIXED) {
        const float *f = (const float *)c->frc;
        if (3 * sizeof(float) * M3 > (size_t)c->l2_bytes) {  // the meshes do not fit in L2
            const unsigned chunks = (unsigned)((c->g.n + kGatherChunk - 1) / kGatherChunk);
            k_gather_f32_staged<<<chunks, 256, 0, c->stream>>>((const float4 *)c->rel, c->keys, c->g, f,
                                                               f + M3, f + 2 * M3, acc_out);
        } else {
            k_gather_f32<<<grid, 256, 0, c->stream>>>((const float4 *)c->rel, c->keys, c->g, f, f + M3,
                                                      f + 2 * M3, acc_out);
        }
    } else {
        const double *f = (const double *)c->frc;
        k_gather_f64<<<grid, 256, 0, c->stream>>>(c->pos, c->g, f, f + M3, f + 2 * M3, acc_out);
    }
    return cudaGetLastError();
}
