// Short-range particle-particle part of the P3M force (the guide's P3M kick algorithm with
// split scale PM_scale and cutoff P3M_cutoff, Ch. Parameters):
//
//   a_SR,i = G m * sum_{j: 0 < r_ij < r_c} g(r_ij / r_s) d_ij / (r_ij^2 + eps^2)^(3/2),
//   g(x) = erfc(x/2) + x/sqrt(pi) exp(-x^2/4),
//
// over the particles of the 27 chaining cells around particle i's cell (n_c >= 3 cells of
// side >= r_c, so each neighbour cell appears once and with the minimum image).
//
// Layout of the work: a CTA is one warp and a work item is up to 32 particles of one cell (one
// per lane).  The warp streams the j particles of the 27 neighbour cells through shared memory
// in tiles of up to five 32-slot blocks of the sorted order, copied by the bulk-copy (TMA)
// engine into two alternating buffers (the next tile in flight while the current one is used;
// one mbarrier per buffer; every wait bounded).  The warp skips a block when no lane's particle
// is within r_c of the block's bounding box, evaluates it without per-pair tests when the box
// lies within r_c of every lane's particle, and otherwise tests each pair, skipping j's that
// no lane accepts.  CTAs are persistent and take work items, most expensive first, from an
// atomic cursor.  No CTA-wide barrier: warps never wait for each other.
//
// Two kernels share that traversal.  k_pairs_x2 (FP32 mode) uses coordinates relative to each
// particle's own cell origin in FP32, shifted per neighbour cell by the difference of the two
// cell origins (an FP32 value plus its FP32 residual), evaluates two j particles per lane with
// packed f32x2 arithmetic and g from a fitted polynomial, and adds each tile's FP32 partial sums
// into FP64 sums per particle (one conversion and one FP64 add per coordinate and tile; measured
// as fast as FP32 TwoSum compensation, and as accurate).  k_pairs64 (FP64 mode) keeps absolute
// coordinates (d = (x_j - x_i) + image, like a plain minimum-image difference) and
// evaluates g with erfc/exp.
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "p3m_device.cuh"
#include "p3m_internal.cuh"

namespace {

constexpr int kTJ = P3M_PAIR_TJ;  // 128
constexpr int kBlocksPerTile = kTJ / 32;
constexpr int kMaxBlocksPerTileX2 = 5;  // FP32 kernel: up to 160 j particles (1.9 KB) per tile
constexpr int kShortTileX2 = 3;        // the autotuner's other choice

// Coefficients of the FP64 split factor (the context's gpoly64): g = 1 + r^3 sum_k c[k] tau^k
// (k <= P3M_SPLIT_DEG64), tau = r^2 c[P3M_SPLIT_DEG64 + 1] - 1.
struct GPoly64 {
    double c[P3M_SPLIT_DEG64 + 2];
};

// g(r/r_s) (r^2 + eps^2)^-3/2 for one pair in FP64, g from the FP64 fit (largest error about
// 4e-14 relative): rsqrt and a Horner chain instead of sqrt, a division, erfc and exp, which
// all run on GB300's narrow FP64 pipe.  For r2 = 0 the result is not finite; callers select
// such pairs out.
__device__ __forceinline__ double pair_factor64(double r2, double eps2, const GPoly64 &gp)
{
    const double s = rsqrt(r2 + eps2);
    const double r3 = r2 * (r2 * rsqrt(r2));
    const double tau = fma(r2, gp.c[P3M_SPLIT_DEG64 + 1], -1.0);
    double p = gp.c[P3M_SPLIT_DEG64];
#pragma unroll
    for (int k = P3M_SPLIT_DEG64 - 1; k >= 0; --k) p = fma(p, tau, gp.c[k]);
    const double gval = fma(r3, p, 1.0);
    return gval * (s * s * s);
}

struct Neighbour {
    uint32_t start, end;
    double imx, imy, imz;  // periodic image of the neighbour cell
};

__global__ void __launch_bounds__(32)
    k_pairs64(const double4_16a *__restrict__ rel, const double *__restrict__ pos,
            const float4 *__restrict__ block_box, const uint32_t *__restrict__ cell_start,
            const uint32_t *__restrict__ work, const uint32_t *__restrict__ order,
            const uint32_t *__restrict__ n_work_ptr, P3MGeom g, GPoly64 gp, float rcull2, float rin2,
            const double *__restrict__ acc_in, double *__restrict__ acc_out,
            double *__restrict__ mom, double kfac, const double *__restrict__ kfac_dev,
            uint32_t *__restrict__ counters, unsigned long long *__restrict__ pair_count)
{
    if (kfac_dev) kfac = *kfac_dev;  // graph-replayed steps read the factor from the device
    __shared__ __align__(128) double4_16a sj[2][kTJ];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ Neighbour nbr[27];

    const int lane = threadIdx.x;
    const int64_t n = g.n;
    const uint32_t n_work = *n_work_ptr;
    const double rc2 = g.r_c * g.r_c;
    const double eps2 = g.eps * g.eps;
    const int nc = g.n_c;

    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncwarp();
    uint32_t parity = 0u;  // bit b: parity of the next phase of bar[b]
    unsigned long long my_pairs = 0, st_fast = 0, st_tested = 0, st_eval = 0, st_culled = 0,
                       st_tiles = 0, st_empty_tiles = 0;
    bool timed_out = false;

    for (;;) {
        uint32_t slot = 0;
        if (lane == 0) slot = atomicAdd(&counters[0], 1u);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot >= n_work) break;
        const uint32_t item = order[slot];
        const uint32_t cell = work[2 * (size_t)item];
        const uint32_t first = work[2 * (size_t)item + 1];
        const uint32_t cend = cell_start[cell + 1];
        const int cx = (int)(cell % nc), cy = (int)((cell / nc) % nc), cz = (int)(cell / (nc * nc));
        if (lane < 27) {
            const int ox = lane % 3 - 1, oy = (lane / 3) % 3 - 1, oz = lane / 9 - 1;
            const int ux = cx + ox, uy = cy + oy, uz = cz + oz;  // unwrapped neighbour index
            const int wx = (ux + nc) % nc, wy = (uy + nc) % nc, wz = (uz + nc) % nc;
            const uint32_t nb = ((uint32_t)wz * nc + wy) * nc + wx;
            Neighbour q;
            q.start = cell_start[nb];
            q.end = cell_start[nb + 1];
            if (q.start == q.end) q.start = q.end = 0;  // empty: the tile walk skips it
            const double L = g.box;
            q.imx = ux < 0 ? -L : (ux >= nc ? L : 0.0);
            q.imy = uy < 0 ? -L : (uy >= nc ? L : 0.0);
            q.imz = uz < 0 ? -L : (uz >= nc ? L : 0.0);
            nbr[lane] = q;
        }
        __syncwarp();

        const uint32_t i = first + lane;
        const bool valid = i < cend;
        const uint32_t ii = valid ? i : first;
        const double4_16a xi = rel[ii];
        const double xa = pos[ii], ya = pos[n + ii], za = pos[2 * n + ii];  // absolute, FP64
        double ax = 0.0, ay = 0.0, az = 0.0;

        // Tile sequence over (neighbour nb, first block b); a tile is the blocks [b, b + 4)
        // clipped to the neighbour's range of slots; nb == 27 ends the sequence.
        auto next_tile = [&](int &nb, uint32_t &b) {
            while (nb < 27 && b * 32u >= nbr[nb].end) {
                ++nb;
                if (nb < 27) b = nbr[nb].start >> 5;
            }
        };
        auto issue = [&](int nb, uint32_t b, int to) {
            const uint32_t bend = min(b + kBlocksPerTile, (nbr[nb].end + 31) >> 5);
            const uint32_t j0 = b * 32;
            const uint32_t j1 = min((uint32_t)n, bend * 32);
            const uint32_t bytes = (j1 - j0) * (uint32_t)sizeof(double4_16a);
            mbar_expect_tx(&bar[to], bytes);
            bulk_load(&sj[to][0], rel + j0, bytes, &bar[to]);
        };

        int nb_c = 0;
        uint32_t b_c = nbr[0].start >> 5;
        next_tile(nb_c, b_c);
        int buf = 0;
        if (nb_c < 27 && lane == 0) issue(nb_c, b_c, 0);
        while (nb_c < 27) {
            const uint32_t nstart = nbr[nb_c].start, nend = nbr[nb_c].end;
            const uint32_t bend = min(b_c + kBlocksPerTile, (nend + 31) >> 5);
            int nb_n = nb_c;
            uint32_t b_n = bend;
            next_tile(nb_n, b_n);
            __syncwarp();  // every lane is done with sj[buf ^ 1] before it is refilled
            if (nb_n < 27 && lane == 0) issue(nb_n, b_n, buf ^ 1);
            const bool ok = mbar_wait_bounded(&bar[buf], (parity >> buf) & 1u);
            parity ^= 1u << buf;
            if (__any_sync(0xffffffffu, !ok)) {
                timed_out = true;
                if (nb_n < 27) mbar_wait_bounded(&bar[buf ^ 1], (parity >> (buf ^ 1)) & 1u);
                break;
            }
            const Neighbour &q = nbr[nb_c];
            // d = (x_j - x_i) + image, like a plain minimum-image difference
            const double xs = xi.x, ys = xi.y, zs = xi.z;
            const double ix = q.imx, iy = q.imy, iz = q.imz;
            // particle i in the frame of the block boxes (absolute, image removed)
            const float cxs = (float)(xa - q.imx), cys = (float)(ya - q.imy), czs = (float)(za - q.imz);
            const double4_16a *tile = sj[buf];
            double px = 0, py = 0, pz = 0;
            uint32_t cnt = 0, n_fast = 0, n_tested = 0, n_eval = 0, n_culled = 0;
            for (uint32_t b = b_c; b < bend; ++b) {
                const float4 lo = __ldg(block_box + 2 * b), hi = __ldg(block_box + 2 * b + 1);
                const float ex = fmaxf(fmaxf(lo.x - cxs, cxs - hi.x), 0.0f);
                const float ey = fmaxf(fmaxf(lo.y - cys, cys - hi.y), 0.0f);
                const float ez = fmaxf(fmaxf(lo.z - czs, czs - hi.z), 0.0f);
                const bool near = valid && ex * ex + ey * ey + ez * ez < rcull2;
                if (!__any_sync(0xffffffffu, near)) {
                    ++n_culled;
                    continue;
                }
                // the block's slots that belong to the neighbour cell, as tile offsets
                const uint32_t j0 = max(b * 32, nstart) - b_c * 32;
                const uint32_t j1 = min(b * 32 + 32, nend) - b_c * 32;
                const float fx = fmaxf(cxs - lo.x, hi.x - cxs);
                const float fy = fmaxf(cys - lo.y, hi.y - cys);
                const float fz = fmaxf(czs - lo.z, hi.z - czs);
                if (__all_sync(0xffffffffu, !valid || fx * fx + fy * fy + fz * fz < rin2)) {
                    // the block lies within r_c of every particle of the warp
                    n_fast += j1 - j0;
#pragma unroll 2
                    for (uint32_t j = j0; j < j1; ++j) {
                        const double4_16a qj = tile[j];
                        const double dx = (qj.x - xs) + ix, dy = (qj.y - ys) + iy, dz = (qj.z - zs) + iz;
                        const double r2 = dx * dx + dy * dy + dz * dz;
                        const bool in = valid && r2 > 0.0;
                        double f = pair_factor64(r2, eps2, gp);
                        f = in ? f : 0.0;
                        px += f * dx;
                        py += f * dy;
                        pz += f * dz;
                        cnt += in ? 1u : 0u;
                    }
                    continue;
                }
                n_tested += j1 - j0;
                for (uint32_t j = j0; j < j1; ++j) {
                    const double4_16a qj = tile[j];
                    const double dx = (qj.x - xs) + ix, dy = (qj.y - ys) + iy, dz = (qj.z - zs) + iz;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    const bool in = valid && r2 < rc2 && r2 > 0.0;
                    if (!__any_sync(0xffffffffu, in)) continue;
                    ++n_eval;
                    double f = pair_factor64(r2, eps2, gp);
                    f = in ? f : 0.0;
                    px += f * dx;
                    py += f * dy;
                    pz += f * dz;
                    cnt += in ? 1u : 0u;
                }
            }
            ax += (double)px;
            ay += (double)py;
            az += (double)pz;
            my_pairs += cnt;
            st_fast += n_fast;
            st_tested += n_tested;
            st_eval += n_eval;
            st_culled += n_culled;
            ++st_tiles;
            if (n_culled == bend - b_c) ++st_empty_tiles;
            buf ^= 1;
            nb_c = nb_n;
            b_c = b_n;
        }
        if (timed_out) break;
        if (valid) {
            const double a3[3] = {g.gm * ax, g.gm * ay, g.gm * az};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double tot = (acc_in ? acc_in[d * n + i] : 0.0) + a3[d];
                acc_out[d * n + i] = tot;
                if (kfac != 0.0) mom[d * n + i] = __dadd_rn(mom[d * n + i], __dmul_rn(kfac, tot));
            }
        }
        __syncwarp();  // nbr is rewritten by the next item
    }
    if (timed_out && lane == 0) atomicOr(&counters[1], P3M_FLAG_TIMEOUT);
    // pair count: warp sum, one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_pairs += __shfl_down_sync(0xffffffffu, my_pairs, o);
    if (lane == 0) {
        if (my_pairs) {
            atomicAdd(pair_count, my_pairs);
            atomicAdd(pair_count + 1, my_pairs);
        }
        if (st_fast) atomicAdd(pair_count + 2, st_fast);
        if (st_tested) atomicAdd(pair_count + 3, st_tested);
        if (st_eval) atomicAdd(pair_count + 4, st_eval);
        if (st_culled) atomicAdd(pair_count + 5, st_culled);
        if (st_tiles) atomicAdd(pair_count + 6, st_tiles);
        if (st_empty_tiles) atomicAdd(pair_count + 7, st_empty_tiles);
    }
}

// ------------------------------------------------------------------ FP32 mode, packed lanes
// The FP32 kernel proper.  Same traversal as k_pairs64 (one-warp CTAs, work items of one cell's
// particles, 27 neighbour cells streamed through two bulk-copy buffers, block culling and the
// all-inside fast path), but every lane evaluates two j particles at once with the packed
// f32x2 arithmetic of sm_100-class GPUs: one instruction issues both halves, so the FP32 pipe
// rather than instruction issue bounds the loop.  The j coordinates come from the block-SoA
// copy relx (per 32-slot block x[32] y[32] z[32]), so the pairs (j, j+1) and (j+2, j+3), j a
// multiple of 4, are one 16-byte shared-memory load per coordinate; the tile's block bounding
// boxes travel with it in the same bulk-copy transaction.
//
// r^2 starts its sum at kTiny = 1e-20: a pair at r = 0 (the particle itself, or a coincident
// one) then gets a finite factor, and its contribution f * d is exactly 0 without a select;
// for r^2 > 1e-12 the addend is absorbed by FP32 rounding.  Pairs are counted when
// kTiny < r^2 < r_c^2 (the kTiny test is made in the own cell only, the one place where r^2 can
// be exactly kTiny).

constexpr float kTiny = 1e-20f;

// Per-lane constants of the packed evaluation.
struct PairConst2 {
    f2 c[P3M_SPLIT_DEG + 1];  // polynomial coefficients, both halves equal
    f2 c11, m1, one, eps2, tiny;
};

// The factor g(r/r_s) (r^2 + eps^2)^-3/2 of both halves of r2 (r2 includes kTiny).
__device__ __forceinline__ f2 pair_factor2(f2 r2, const PairConst2 &k)
{
    float r2l, r2h, s2l, s2h;
    const f2 s2 = f2_add(r2, k.eps2);
    f2_unpack(r2, r2l, r2h);
    f2_unpack(s2, s2l, s2h);
    // s^3 = (r^2 + eps^2)^-3/2 as rsqrt * rcp: one FP32 multiply instead of two (the MUFU
    // pipe has room to spare)
    const f2 s3 = f2_mul(f2_pack(rsqrt_approx(s2l), rsqrt_approx(s2h)),
                         f2_pack(rcp_approx(s2l), rcp_approx(s2h)));
    const f2 r3 = f2_mul(r2, f2_pack(sqrt_approx(r2l), sqrt_approx(r2h)));
    const f2 tau = f2_fma(r2, k.c11, k.m1);
    f2 p = k.c[P3M_SPLIT_DEG];
#pragma unroll
    for (int q = P3M_SPLIT_DEG - 1; q >= 0; --q) p = f2_fma(p, tau, k.c[q]);
    const f2 gval = f2_fma(r3, p, k.one);
    return f2_mul(gval, s3);
}

template <bool kBatched, int kTileBlocks>
__global__ void __launch_bounds__(32, 32)
    k_pairs_x2(PairArgs a0, const PairArgs *__restrict__ descs, const uint32_t *__restrict__ order,
               const uint32_t *__restrict__ n_work_ptr, uint32_t *__restrict__ cursor)
{
    constexpr int kBlockFloats = 96;  // x[32] y[32] z[32]
    constexpr int kArgWords = sizeof(PairArgs) / 8;
    static_assert(sizeof(PairArgs) % 8 == 0, "PairArgs is copied in 8-byte words");
    __shared__ __align__(128) float sj[2][kTileBlocks * kBlockFloats];
    __shared__ __align__(16) float4 sbox[2][2 * kTileBlocks];  // the tile's block boxes (lo, hi)
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ NeighbourF nbr[27];
    __shared__ __align__(16) PairArgs sA;  // the current work item's context
    const PairArgs &A = sA;

    const int lane = threadIdx.x;
    const uint32_t n_work = *n_work_ptr;
    int cur_sim = -1;
    double kfac = 0.0;
    PairConst2 kc;
    kc.m1 = f2_pack(-1.0f, -1.0f);
    kc.one = f2_pack(1.0f, 1.0f);
    kc.tiny = f2_pack(kTiny, kTiny);
    // (re)load the context's arguments into shared memory and the per-lane constants
    auto load_args = [&](const PairArgs *src) {
        __syncwarp();  // every lane is done with the previous arguments
        const uint64_t *from = (const uint64_t *)src;
        uint64_t *to = (uint64_t *)&sA;
        for (int w = lane; w < kArgWords; w += 32) to[w] = from[w];
        __syncwarp();
        kfac = A.kfac_dev ? *A.kfac_dev : A.kfac;
#pragma unroll
        for (int q = 0; q <= P3M_SPLIT_DEG; ++q) kc.c[q] = f2_pack(A.gpoly[q], A.gpoly[q]);
        kc.c11 = f2_pack(A.gpoly[11], A.gpoly[11]);
        const float e2 = (float)(A.g.eps * A.g.eps);
        kc.eps2 = f2_pack(e2, e2);
    };
    if (!kBatched) load_args(&a0);

    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncwarp();
    uint32_t parity = 0u;
    bool timed_out = false;

    for (;;) {
        uint32_t slot = 0;
        if (lane == 0) slot = atomicAdd(cursor, 1u);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot >= n_work) break;
        uint32_t item = order[slot];
        if (kBatched) {
            const int sim = (int)(item >> 24);
            item &= 0xFFFFFFu;
            if (sim != cur_sim) {
                load_args(descs + sim);
                cur_sim = sim;
            }
        }
        const P3MGeom &g = A.g;
        const int64_t n = g.n;
        const int nc = g.n_c;
        const float rc2 = (float)(g.r_c * g.r_c), rcull2 = A.rcull2, rin2 = A.rin2;
        const float *__restrict__ relx = A.relx;
        const float4 *__restrict__ block_box = A.block_box;
        const uint32_t cell = A.work[2 * (size_t)item];
        const uint32_t first = A.work[2 * (size_t)item + 1];
        const uint32_t cend = A.cell_start[cell + 1];
        const int cx = (int)(cell % nc), cy = (int)((cell / nc) % nc), cz = (int)(cell / (nc * nc));
        __syncwarp();  // the previous item is done with nbr
        if (lane < 27) nbr[lane] = make_neighbour(g, A.cell_start, cx, cy, cz, lane);
        __syncwarp();
        // the item's pair count (this lane) and work counters (warp-uniform)
        uint32_t cnt = 0, n_fast = 0, n_tested = 0, n_eval = 0, n_culled = 0, n_tiles = 0,
                 n_empty = 0;

        const uint32_t i = first + lane;
        const bool valid = i < cend;
        const uint32_t ii = valid ? i : first;
        const float4 xi = A.rel[ii];
        // absolute position in FP32, for the bounding-box tests only (their margins cover
        // the FP32 rounding of coordinates up to the box size)
        const double *__restrict__ pos = A.pos;
        const float xa = (float)pos[ii], ya = (float)pos[n + ii], za = (float)pos[2 * n + ii];
        double sax = 0.0, say = 0.0, saz = 0.0;

        auto next_tile = [&](int &nb, uint32_t &b) {
            while (nb < 27 && b * 32u >= nbr[nb].end) {
                ++nb;
                if (nb < 27) b = nbr[nb].start >> 5;
            }
        };
        auto issue = [&](int nb, uint32_t b, int to) {
            const uint32_t bend = min(b + kTileBlocks, (nbr[nb].end + 31) >> 5);
            const uint32_t bytes = (bend - b) * (uint32_t)(kBlockFloats * sizeof(float));
            const uint32_t box_bytes = (bend - b) * (uint32_t)(2 * sizeof(float4));
            mbar_expect_tx(&bar[to], bytes + box_bytes);
            bulk_load(&sj[to][0], relx + (size_t)b * kBlockFloats, bytes, &bar[to]);
            bulk_load(&sbox[to][0], block_box + 2 * (size_t)b, box_bytes, &bar[to]);
        };

        int nb_c = 0;
        uint32_t b_c = nbr[0].start >> 5;
        next_tile(nb_c, b_c);
        int buf = 0;
        if (nb_c < 27 && lane == 0) issue(nb_c, b_c, 0);
        // x_i in the current neighbour cell's frame, set when the tile walk enters the cell
        int nb_frame = -1;
        f2 xs2 = make_float2(0.0f, 0.0f), ys2 = xs2, zs2 = xs2;
        float cxs = 0.0f, cys = 0.0f, czs = 0.0f;
        while (nb_c < 27) {
            const uint32_t nstart = nbr[nb_c].start, nend = nbr[nb_c].end;
            const uint32_t bend = min(b_c + kTileBlocks, (nend + 31) >> 5);
            int nb_n = nb_c;
            uint32_t b_n = bend;
            next_tile(nb_n, b_n);
            __syncwarp();
            if (nb_n < 27 && lane == 0) issue(nb_n, b_n, buf ^ 1);
            const bool ok = mbar_wait_bounded(&bar[buf], (parity >> buf) & 1u);
            parity ^= 1u << buf;
            if (__any_sync(0xffffffffu, !ok)) {
                timed_out = true;
                if (nb_n < 27) mbar_wait_bounded(&bar[buf ^ 1], (parity >> (buf ^ 1)) & 1u);
                break;
            }
            if (nb_c != nb_frame) {
                nb_frame = nb_c;
                const NeighbourF &q = nbr[nb_c];
                // x_i in the neighbour cell's frame: (x_i - s) with s = sx + rx
                const float xs = (xi.x - q.sx) - q.rx;
                const float ys = (xi.y - q.sy) - q.ry;
                const float zs = (xi.z - q.sz) - q.rz;
                xs2 = f2_pack(xs, xs);
                ys2 = f2_pack(ys, ys);
                zs2 = f2_pack(zs, zs);
                cxs = xa - q.imx;
                cys = ya - q.imy;
                czs = za - q.imz;
            }
            f2 px = make_float2(0.0f, 0.0f), py = px, pz = px;
            const uint32_t culled0 = n_culled;

            // Pair counts: a pair is counted when kTiny < r^2 < r_c^2.  r^2 = kTiny (all three
            // FP32 differences zero) happens for the particle itself and for coincident
            // particles, which always share a cell, so only the own cell (neighbour 13) tests
            // r^2 > kTiny; elsewhere every pair with r^2 < r_c^2 counts, and an all-inside block
            // adds its slot count without per-pair tests.

            // the pair (j, j+1) from its packed coordinates in an all-inside block, where every
            // lane accepts both; lo/hi (warp-uniform): which halves belong to the neighbour cell
            auto eval_inside = [&](auto own, f2 xj, f2 yj, f2 zj, bool lo, bool hi) {
                const f2 dx = f2_sub(xj, xs2), dy = f2_sub(yj, ys2), dz = f2_sub(zj, zs2);
                const f2 r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_fma(dx, dx, kc.tiny)));
                f2 f = pair_factor2(r2, kc);
                if (!(lo && hi)) {
                    float fl, fh;
                    f2_unpack(f, fl, fh);
                    f = f2_pack(lo ? fl : 0.0f, hi ? fh : 0.0f);
                }
                px = f2_fma(f, dx, px);
                py = f2_fma(f, dy, py);
                pz = f2_fma(f, dz, pz);
                if (decltype(own)::value) {
                    float r2l, r2h;
                    f2_unpack(r2, r2l, r2h);
                    cnt += (lo && r2l > kTiny) + (hi && r2h > kTiny);
                }
            };

            // one aligned pair (p, p+1) of the block at bx; lo/hi: which halves take part
            auto pair_tested = [&](auto own, const float *bx, uint32_t p, bool lo, bool hi) {
                const f2 dx = f2_sub(*(const f2 *)(bx + p), xs2);
                const f2 dy = f2_sub(*(const f2 *)(bx + 32 + p), ys2);
                const f2 dz = f2_sub(*(const f2 *)(bx + 64 + p), zs2);
                const f2 r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_fma(dx, dx, kc.tiny)));
                float r2l, r2h;
                f2_unpack(r2, r2l, r2h);
                const bool inl = lo && r2l < rc2, inh = hi && r2h < rc2;
                if (!__any_sync(0xffffffffu, inl || inh)) return;
                ++n_eval;
                float fl, fh;
                f2_unpack(pair_factor2(r2, kc), fl, fh);
                const f2 f = f2_pack(inl ? fl : 0.0f, inh ? fh : 0.0f);
                px = f2_fma(f, dx, px);
                py = f2_fma(f, dy, py);
                pz = f2_fma(f, dz, pz);
                if (decltype(own)::value)
                    cnt += (inl && r2l > kTiny) + (inh && r2h > kTiny);
                else
                    cnt += inl + inh;
            };

            // four slots p .. p+3 (p a multiple of 4) as two pairs, all halves taking part: each
            // pair is skipped when no lane accepts it, and when both are needed their
            // evaluations interleave
            auto pairs_tested2 = [&](auto own, const float *bx, uint32_t p) {
                const float4 X = *(const float4 *)(bx + p), Y = *(const float4 *)(bx + 32 + p),
                             Z = *(const float4 *)(bx + 64 + p);
                f2 d[2][3], r2[2];
                bool in[2][2], any[2];
                d[0][0] = f2_sub(f2_pack(X.x, X.y), xs2);
                d[0][1] = f2_sub(f2_pack(Y.x, Y.y), ys2);
                d[0][2] = f2_sub(f2_pack(Z.x, Z.y), zs2);
                d[1][0] = f2_sub(f2_pack(X.z, X.w), xs2);
                d[1][1] = f2_sub(f2_pack(Y.z, Y.w), ys2);
                d[1][2] = f2_sub(f2_pack(Z.z, Z.w), zs2);
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    r2[u] = f2_fma(d[u][2], d[u][2], f2_fma(d[u][1], d[u][1], f2_fma(d[u][0], d[u][0], kc.tiny)));
                    float l, h;
                    f2_unpack(r2[u], l, h);
                    in[u][0] = l < rc2;
                    in[u][1] = h < rc2;
                    any[u] = __any_sync(0xffffffffu, in[u][0] || in[u][1]);
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (!any[u]) continue;  // (then no lane counts a pair either)
                    ++n_eval;
                    float l, h;
                    f2_unpack(r2[u], l, h);
                    if (decltype(own)::value)
                        cnt += (in[u][0] && l > kTiny) + (in[u][1] && h > kTiny);
                    else
                        cnt += in[u][0] + in[u][1];
                    float fl, fh;
                    f2_unpack(pair_factor2(r2[u], kc), fl, fh);
                    const f2 f = f2_pack(in[u][0] ? fl : 0.0f, in[u][1] ? fh : 0.0f);
                    px = f2_fma(f, d[u][0], px);
                    py = f2_fma(f, d[u][1], py);
                    pz = f2_fma(f, d[u][2], pz);
                }
            };

            // the blocks of the tile; own: the neighbour is the work item's own cell
            auto blocks = [&](auto own) {
                for (uint32_t b = b_c; b < bend; ++b) {
                    const float4 lo = sbox[buf][2 * (b - b_c)], hi = sbox[buf][2 * (b - b_c) + 1];
                    const float ex = fmaxf(fmaxf(lo.x - cxs, cxs - hi.x), 0.0f);
                    const float ey = fmaxf(fmaxf(lo.y - cys, cys - hi.y), 0.0f);
                    const float ez = fmaxf(fmaxf(lo.z - czs, czs - hi.z), 0.0f);
                    const bool near = valid && ex * ex + ey * ey + ez * ez < rcull2;
                    if (!__any_sync(0xffffffffu, near)) {
                        ++n_culled;
                        continue;
                    }
                    const uint32_t j0 = max(b * 32, nstart) - b * 32;  // block-relative range
                    const uint32_t j1 = min(b * 32 + 32, nend) - b * 32;
                    const float *bx = sj[buf] + (b - b_c) * kBlockFloats;
                    const float fx = fmaxf(cxs - lo.x, hi.x - cxs);
                    const float fy = fmaxf(cys - lo.y, hi.y - cys);
                    const float fz = fmaxf(czs - lo.z, hi.z - czs);
                    uint32_t p = j0 & ~1u;
                    if (__all_sync(0xffffffffu, !valid || fx * fx + fy * fy + fz * fz < rin2)) {
                        // the block lies within r_c of every particle of the warp
                        n_fast += j1 - j0;
                        if (!decltype(own)::value) cnt += j1 - j0;
                        const f2 *px2 = (const f2 *)bx;  // (p, p+1) as one 8-byte load
                        if ((j0 & 1u) && j0 < j1) {
                            eval_inside(own, px2[p / 2], px2[16 + p / 2], px2[32 + p / 2], false, true);
                            p += 2;
                        }
                        if ((p & 2u) && p + 1 < j1) {
                            eval_inside(own, px2[p / 2], px2[16 + p / 2], px2[32 + p / 2], true, true);
                            p += 2;
                        }
                        for (; p + 3 < j1; p += 4) {
                            const float4 X = *(const float4 *)(bx + p), Y = *(const float4 *)(bx + 32 + p),
                                         Z = *(const float4 *)(bx + 64 + p);
                            eval_inside(own, f2_pack(X.x, X.y), f2_pack(Y.x, Y.y), f2_pack(Z.x, Z.y), true, true);
                            eval_inside(own, f2_pack(X.z, X.w), f2_pack(Y.z, Y.w), f2_pack(Z.z, Z.w), true, true);
                        }
                        if (p + 1 < j1) {
                            eval_inside(own, px2[p / 2], px2[16 + p / 2], px2[32 + p / 2], true, true);
                            p += 2;
                        }
                        if (p < j1) eval_inside(own, px2[p / 2], px2[16 + p / 2], px2[32 + p / 2], true, false);
                        continue;
                    }
                    n_tested += j1 - j0;
                    if ((j0 & 1u) && j0 < j1) {
                        pair_tested(own, bx, p, false, true);
                        p += 2;
                    }
                    if ((p & 2u) && p + 1 < j1) {
                        pair_tested(own, bx, p, true, true);
                        p += 2;
                    }
                    for (; p + 3 < j1; p += 4) pairs_tested2(own, bx, p);
                    for (; p + 1 < j1; p += 2) pair_tested(own, bx, p, true, true);
                    if (p < j1) pair_tested(own, bx, p, true, false);
                }
            };
            if (nb_c == 13)
                blocks(std::true_type{});
            else
                blocks(std::false_type{});
            float lo_, hi_;
            f2_unpack(px, lo_, hi_);
            sax += (double)(lo_ + hi_);
            f2_unpack(py, lo_, hi_);
            say += (double)(lo_ + hi_);
            f2_unpack(pz, lo_, hi_);
            saz += (double)(lo_ + hi_);
            ++n_tiles;
            if (n_culled - culled0 == bend - b_c) ++n_empty;
            buf ^= 1;
            nb_c = nb_n;
            b_c = b_n;
        }
        if (timed_out) {
            if (lane == 0) atomicOr(&A.counters[1], P3M_FLAG_TIMEOUT);
            break;
        }
        if (valid) {
            const double a3[3] = {g.gm * sax, g.gm * say, g.gm * saz};
            const double *__restrict__ acc_in = A.acc_in;
            double *__restrict__ acc_out = A.acc_out;
            double *__restrict__ mom = A.mom;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double tot = (acc_in ? acc_in[d * n + i] : 0.0) + a3[d];
                acc_out[d * n + i] = tot;
                if (kfac != 0.0) mom[d * n + i] = __dadd_rn(mom[d * n + i], __dmul_rn(kfac, tot));
            }
        }
        // the item's pair count (warp sum) and work counters, into its context
        unsigned long long my_pairs = valid ? cnt : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_pairs += __shfl_down_sync(0xffffffffu, my_pairs, o);
        if (lane == 0) {
            unsigned long long *pc = A.pair_count;
            if (my_pairs) {
                atomicAdd(pc, my_pairs);
                atomicAdd(pc + 1, my_pairs);
            }
            if (n_fast) atomicAdd(pc + 2, (unsigned long long)n_fast);
            if (n_tested) atomicAdd(pc + 3, (unsigned long long)n_tested);
            if (n_eval) atomicAdd(pc + 4, 2ull * n_eval);
            if (n_culled) atomicAdd(pc + 5, (unsigned long long)n_culled);
            if (n_tiles) atomicAdd(pc + 6, (unsigned long long)n_tiles);
            if (n_empty) atomicAdd(pc + 7, (unsigned long long)n_empty);
        }
    }
}

cudaError_t pairs64_impl(p3m_ctx *c, const double *acc_in, double *acc_out, double kfac,
                       const double *kfac_dev)
{
    cudaMemsetAsync(c->counters, 0, sizeof(uint32_t), c->stream);
    cudaMemsetAsync(c->pair_count, 0, sizeof(unsigned long long), c->stream);  // last evaluation
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs64, 32, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int grid = c->num_sms * per_sm;
    GPoly64 gp;
    for (int k = 0; k < P3M_SPLIT_DEG64 + 2; ++k) gp.c[k] = c->gpoly64[k];
    // culling radii: r_c widened (narrowed) by more than the FP32 rounding of absolute
    // coordinates up to the box size
    const double rcull = c->g.r_c * (1.0 + 1e-4) + c->g.box * 1e-6;
    const double rin = c->g.r_c * (1.0 - 1e-4) - c->g.box * 1e-6;
    c->launches += 1;
    k_pairs64<<<grid, 32, 0, c->stream>>>(
        (const double4_16a *)c->rel, c->pos, c->block_box, c->cell_start, c->work,
        c->work_order, c->work_off + c->g.n_cells, c->g, gp, (float)(rcull * rcull),
        rin > 0.0 ? (float)(rin * rin) : 0.0f, acc_in, acc_out, c->mom, kfac, kfac_dev,
        c->counters, c->pair_count);
    return cudaGetLastError();
}

cudaError_t pairs_x2_impl(p3m_ctx *c, const double *acc_in, double *acc_out, double kfac,
                          const double *kfac_dev)
{
    cudaMemsetAsync(c->counters, 0, sizeof(uint32_t), c->stream);
    cudaMemsetAsync(c->pair_count, 0, sizeof(unsigned long long), c->stream);  // last evaluation
    int per_sm = 0;
    auto kern = c->tile_blocks == kShortTileX2 ? k_pairs_x2<false, kShortTileX2>
                                                : k_pairs_x2<false, kMaxBlocksPerTileX2>;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    c->launches += 1;
    kern<<<c->num_sms * per_sm, 32, 0, c->stream>>>(pair_args(c, acc_in, acc_out, kfac, kfac_dev),
                                                    nullptr, c->work_order,
                                                    c->work_off + c->g.n_cells, c->counters);
    return cudaGetLastError();
}

__global__ void k_store_pair_args(PairArgs *dst, PairArgs a) { *dst = a; }

__global__ void k_ens_gather(uint32_t slot, const uint32_t *__restrict__ key,
                             const uint32_t *__restrict__ order, size_t n, uint32_t *__restrict__ gk,
                             uint32_t *__restrict__ gv)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        gk[k] = key[k];
        gv[k] = (slot << 24) | (order[k] & 0xFFFFFFu);
    }
}

__global__ void k_ens_total(const uint32_t *const *nwork, int nb, uint32_t *total)
{
    uint32_t t = 0;
    for (int k = 0; k < nb; ++k) t += *nwork[k];
    *total = t;
}

}  // namespace

PairArgs pair_args(const p3m_ctx *c, const double *acc_in, double *acc_out, double kfac,
                   const double *kfac_dev)
{
    PairArgs a;
    memset(&a, 0, sizeof(a));
    a.relx = c->relx;
    a.rel = (const float4 *)c->rel;
    a.pos = c->pos;
    a.block_box = c->block_box;
    a.cell_start = c->cell_start;
    a.work = c->work;
    a.acc_in = acc_in;
    a.acc_out = acc_out;
    a.mom = c->mom;
    a.kfac_dev = kfac_dev;
    a.counters = c->counters;
    a.pair_count = c->pair_count;
    a.kfac = kfac;
    a.g = c->g;
    for (int k = 0; k < 12; ++k) a.gpoly[k] = c->gpoly[k];
    // culling radii: r_c widened (narrowed) by more than the FP32 rounding of absolute
    // coordinates up to the box size
    const double rcull = c->g.r_c * (1.0 + 1e-4) + c->g.box * 1e-6;
    const double rin = c->g.r_c * (1.0 - 1e-4) - c->g.box * 1e-6;
    a.rcull2 = (float)(rcull * rcull);
    a.rin2 = rin > 0.0 ? (float)(rin * rin) : 0.0f;
    return a;
}

cudaError_t launch_pairs_batched(const PairArgs *descs, const uint32_t *order,
                                 const uint32_t *n_total, uint32_t *cursor, int num_sms,
                                 cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs_x2<true, kMaxBlocksPerTileX2>,
                                                      32, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    PairArgs unused;
    memset(&unused, 0, sizeof(unused));
    k_pairs_x2<true, kMaxBlocksPerTileX2><<<num_sms * per_sm, 32, 0, s>>>(unused, descs, order,
                                                                          n_total, cursor);
    return cudaGetLastError();
}

cudaError_t launch_store_pair_args(PairArgs *dst, const PairArgs &a, cudaStream_t s)
{
    k_store_pair_args<<<1, 1, 0, s>>>(dst, a);
    return cudaGetLastError();
}

cudaError_t launch_ens_gather(int slot, const uint32_t *key, const uint32_t *order, size_t n,
                              uint32_t *gkey, uint32_t *gval, cudaStream_t s)
{
    const size_t blocks = (n + 255) / 256;
    k_ens_gather<<<(unsigned)(blocks < 1 ? 1 : (blocks > 1024 ? 1024 : blocks)), 256, 0, s>>>(
        (uint32_t)slot, key, order, n, gkey, gval);
    return cudaGetLastError();
}

cudaError_t launch_ens_total(const uint32_t *const *nwork, int nb, uint32_t *total, cudaStream_t s)
{
    k_ens_total<<<1, 1, 0, s>>>(nwork, nb, total);
    return cudaGetLastError();
}

cudaError_t launch_pairs(p3m_ctx *c, const double *acc_in, double *acc_out, double kfac,
                         const double *kfac_dev)
{
    return c->precision == P3M_PREC_MIXED ? pairs_x2_impl(c, acc_in, acc_out, kfac, kfac_dev)
                                          : pairs64_impl(c, acc_in, acc_out, kfac, kfac_dev);
}
