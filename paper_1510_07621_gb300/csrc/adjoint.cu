// Reverse-mode derivative of the P3M force: the transposed Jacobian of the accelerations
// applied to a vector field v, (dA/dx)^T v, and the gradient of a mesh density loss.  These
// are the pieces of the adjoint of the kick-drift-kick step (the reverse sweep itself runs on
// the host side).
//
// Mesh part, with E_b = D_b rho the three mesh accelerations (D_b = IFFT(-i k_b G FFT), real,
// D_b^T = IFFT(+i k_b G FFT)) and rho(n) = sum_j W(x_j - n) the CIC counts:
//   out_k = sum_n grad W(x_k - n) [ sum_b v_k,b E_b(n) + psi(n) ],
//   psi = sum_b D_b^T u_b,  u_b(n) = sum_i W(x_i - n) v_i,b.
// Pair part, J(d) = h(r) I + (h'(r)/r) d d^T with h(r) = Gm g(r/r_s) (r^2 + eps^2)^-3/2:
//   out_k = sum_{j: 0 < r_kj < r_c} J(d_kj) (v_j - v_k).
#include <cuda_runtime.h>
#include <cufft.h>
#include <math.h>

#include <type_traits>
#include <vector>

#include "p3m_device.cuh"
#include "p3m_internal.cuh"

namespace {

inline int grid_for(int64_t n, int threads, int num_sms)
{
    int64_t b = (n + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ int wrap_index(int i, int M)
{
    i %= M;
    return i < 0 ? i + M : i;
}

// CIC stencil in FP64: base node i0 = floor(x M/L), fraction f.
__device__ __forceinline__ void stencil64(double x, double inv_h, int &i0, double &f)
{
    const double u = __dmul_rn(x, inv_h);
    const double fl = floor(u);
    i0 = (int)fl;
    f = u - fl;
}

// v_sorted[k] = v[pid[k]] (caller order -> slot order), also an FP32 copy with w = 0.
__global__ void k_to_slots(const double *__restrict__ v, const uint32_t *__restrict__ pid,
                           int64_t n, double *__restrict__ vs, float *__restrict__ vfx)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = pid[k];
        const double a = v[j], b = v[n + j], c = v[2 * n + j];
        vs[k] = a;
        vs[n + k] = b;
        vs[2 * n + k] = c;
        if (vfx) {  // FP32 block-SoA copy (per 32-slot block vx[32] vy[32] vz[32])
            float *dst = vfx + (k >> 5) * 96 + (k & 31);
            dst[0] = (float)a;
            dst[32] = (float)b;
            dst[64] = (float)c;
        }
    }
}

// The vector deposit u_b(node) = sum_k W(x_k - node) v_k,b accumulates in signed 64-bit fixed
// point, like the mass deposit, so that its result does not depend on the order of the atomic
// additions.  The scale 2^S comes from the largest |v|: with |v| < 2^e and N < 2^nb, every
// partial sum stays below 2^61 in magnitude for S = 61 - nb - e.

// *out = max |v| over n values, as the bit pattern of a non-negative double (those order like
// unsigned integers, so the maximum does not depend on the order of the atomics either).
__global__ void k_absmax_bits(const double *__restrict__ v, int64_t n, unsigned long long *__restrict__ out)
{
    unsigned long long m = 0ull;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v[k]));
        m = b > m ? b : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, m, o);
        m = x > m ? x : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// s_out[0] = S for the largest |v| in *maxbits (0 when v is all zero or not finite).
__global__ void k_fix_exponent(const unsigned long long *__restrict__ maxbits, int nb, int *__restrict__ s_out)
{
    const double m = __longlong_as_double((long long)*maxbits);
    int S = 0;
    if (m > 0.0 && m <= 1.7976931348623157e308) {
        int e = 0;
        frexp(m, &e);  // m < 2^e
        S = 61 - nb - e;
        S = S > 1000 ? 1000 : S;
    }
    s_out[0] = S;
}

// u_b(node) += W(x_k - node) v_k,b as round(W v 2^S) on three fixed-point meshes.
__global__ void k_deposit_vec(const double *__restrict__ pos, const double *__restrict__ v,
                              P3MGeom g, const int *__restrict__ s_dev,
                              unsigned long long *__restrict__ fix)
{
    const int M = g.mesh;
    const int64_t n = g.n;
    const size_t M3 = (size_t)M * M * M;
    const double scale = ldexp(1.0, *s_dev);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        double fx, fy, fz;
        stencil64(pos[k], g.inv_h, ix, fx);
        stencil64(pos[n + k], g.inv_h, iy, fy);
        stencil64(pos[2 * n + k], g.inv_h, iz, fz);
        const double wx[2] = {1.0 - fx, fx}, wy[2] = {1.0 - fy, fy}, wz[2] = {1.0 - fz, fz};
        const double vb[3] = {v[k] * scale, v[n + k] * scale, v[2 * n + k] * scale};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const double w = wx[a] * wy[b] * wz[c];
                    const size_t node = ((size_t)wrap_index(ix + a, M) * M + wrap_index(iy + b, M)) * M +
                                        wrap_index(iz + c, M);
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        atomicAdd(fix + d * M3 + node, (unsigned long long)__double2ll_rn(w * vb[d]));
                }
    }
}

// u = fix 2^-S (signed).
template <typename T>
__global__ void k_fix_to_vec(const unsigned long long *__restrict__ fix, size_t n,
                             const int *__restrict__ s_dev, T *__restrict__ u)
{
    const double inv_scale = ldexp(1.0, -*s_dev);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        u[i] = (T)(__ll2double_rn((long long)fix[i]) * inv_scale);
}

// psi_k = sum_b (+i kg_b G(k)) u_b,k with G as in the forward pass (constants included).
template <typename T, typename C2>
__global__ void k_kspace_adjoint(const C2 *__restrict__ ux, const C2 *__restrict__ uy,
                                 const C2 *__restrict__ uz, const T *__restrict__ tk,
                                 const T *__restrict__ tkg, const T *__restrict__ tg, int M,
                                 T gconst, C2 *__restrict__ psi)
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
        const C2 a = ux[idx], b = uy[idx], c = uz[idx];
        // i kg G u = G kg (-u.y, u.x)
        const T gx = G * tkg[ix], gy = G * tkg[iy], gz = G * tkg[iz];
        C2 o;
        o.x = -(gx * a.y + gy * b.y + gz * c.y);
        o.y = gx * a.x + gy * b.x + gz * c.x;
        psi[idx] = o;
    }
}

// out_k += scale sum_corners grad W(x_k - node) [ sum_b v_k,b E_b(node) + psi(node) ]
// (E or v NULL: no first term; psi NULL: no second term).
template <typename T>
__global__ void k_gather_grad(const double *__restrict__ pos, P3MGeom g, const T *__restrict__ E,
                              const double *__restrict__ v, const T *__restrict__ psi,
                              double scale, double *__restrict__ out)
{
    const int M = g.mesh;
    const int64_t n = g.n;
    const size_t M3 = (size_t)M * M * M;
    const double ih = g.inv_h;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        double fx, fy, fz;
        stencil64(pos[k], ih, ix, fx);
        stencil64(pos[n + k], ih, iy, fy);
        stencil64(pos[2 * n + k], ih, iz, fz);
        const double wx[2] = {1.0 - fx, fx}, wy[2] = {1.0 - fy, fy}, wz[2] = {1.0 - fz, fz};
        const double dx[2] = {-ih, ih};
        double vb[3] = {0.0, 0.0, 0.0};
        if (E && v) {
            vb[0] = v[k];
            vb[1] = v[n + k];
            vb[2] = v[2 * n + k];
        }
        double o0 = 0.0, o1 = 0.0, o2 = 0.0;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const size_t node = ((size_t)wrap_index(ix + a, M) * M + wrap_index(iy + b, M)) * M +
                                        wrap_index(iz + c, M);
                    double s = psi ? (double)psi[node] : 0.0;
                    if (E && v)
                        s += vb[0] * (double)E[node] + vb[1] * (double)E[M3 + node] +
                             vb[2] * (double)E[2 * M3 + node];
                    o0 += dx[a] * wy[b] * wz[c] * s;
                    o1 += wx[a] * dx[b] * wz[c] * s;
                    o2 += wx[a] * wy[b] * dx[c] * s;
                }
        out[k] += scale * o0;
        out[n + k] += scale * o1;
        out[2 * n + k] += scale * o2;
    }
}

// Density loss on the mesh: rho holds counts - mean; delta = rho / n_bar; per node
// r = delta - target; loss partial sums per block; ell = 2 r / n_bar written over rho.
template <typename T>
__global__ void __launch_bounds__(256)
    k_loss_mesh(T *__restrict__ rho, const double *__restrict__ target, size_t M3, double inv_nbar,
                double *__restrict__ part)
{
    __shared__ double s[256];
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M3;
         i += (size_t)gridDim.x * blockDim.x) {
        const double r = (double)rho[i] * inv_nbar - target[i];
        acc += r * r;
        rho[i] = (T)(2.0 * r * inv_nbar);
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_sum_parts(double *part, int nb, double *out)
{
    __shared__ double s[256];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[b];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// ------------------------------------------------------------------ pair part

// Coefficients of the FP32 split factor (the context's fitted polynomial, see p3m_ctx::gpoly).
struct GPolyA {
    float c[12];
};

// h(r)/Gm and h'(r)/(Gm r) for one pair in FP64, g and g' in closed form.
__device__ __forceinline__ void pair_jac(double r2, double eps2, double inv_rs, double &h,
                                         double &hr)
{
    const double r = sqrt(r2), x = r * inv_rs;
    const double s2 = r2 + eps2, s3 = s2 * sqrt(s2);
    const double gval = erfc(0.5 * x) + x * 0.56418958354775628695 * exp(-0.25 * x * x);
    const double gder = -x * x * exp(-0.25 * x * x) * 0.28209479177387814347;
    h = gval / s3;
    hr = (gder * inv_rs / s3 - 3.0 * r * gval / (s3 * s2)) / r;
}

template <typename T>
struct V4Of;
template <>
struct V4Of<float> {
    using type = float4;
};
template <>
struct V4Of<double> {
    using type = double4_16a;
};

// FP64 mode: one warp per work item (up to 32 particles of one cell, most expensive items first),
// like the force pair kernel: the j particles of the 27 neighbour cells in 32-slot blocks, a
// block skipped when no lane's particle is within r_c of its bounding box, evaluated without
// pair tests when it lies within r_c of every lane's particle; j data read through the cache
// and broadcast by shuffles.  out_k += Gm sum_j J(d_kj) (v_j - v_k).
__global__ void __launch_bounds__(32)
    k_pairs_vjp64(const double4_16a *__restrict__ rel, const double *__restrict__ pos,
                  const float4 *__restrict__ block_box, const double *__restrict__ vs,
                  const uint32_t *__restrict__ cell_start, const uint32_t *__restrict__ work,
                  const uint32_t *__restrict__ order, const uint32_t *__restrict__ n_work_ptr,
                  P3MGeom g, float rcull2, float rin2, uint32_t *__restrict__ cursor,
                  double *__restrict__ out)
{
    const int lane = threadIdx.x;
    const int64_t n = g.n;
    const uint32_t n_work = *n_work_ptr;
    const double rc2 = g.r_c * g.r_c, eps2 = g.eps * g.eps, inv_rs = 1.0 / g.r_s;
    const int nc = g.n_c;
    for (;;) {
        uint32_t slot = 0;
        if (lane == 0) slot = atomicAdd(cursor, 1u);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot >= n_work) break;
        const uint32_t item = order[slot];
        const uint32_t cell = work[2 * (size_t)item], first = work[2 * (size_t)item + 1];
        const uint32_t cend = cell_start[cell + 1];
        const int cx = (int)(cell % nc), cy = (int)((cell / nc) % nc), cz = (int)(cell / (nc * nc));
        const uint32_t i = first + lane;
        const bool valid = i < cend;
        const uint32_t ii = valid ? i : first;
        const double4_16a xi = rel[ii];
        const double xa = pos[ii], ya = pos[n + ii], za = pos[2 * n + ii];
        const double vix = vs[ii], viy = vs[n + ii], viz = vs[2 * n + ii];
        double o[3] = {0.0, 0.0, 0.0};
        for (int nb = 0; nb < 27; ++nb) {
            const int ux = cx + nb % 3 - 1, uy = cy + (nb / 3) % 3 - 1, uz = cz + nb / 9 - 1;
            const int wx = (ux + nc) % nc, wy = (uy + nc) % nc, wz = (uz + nc) % nc;
            const uint32_t q = ((uint32_t)wz * nc + wy) * nc + wx;
            const uint32_t js = cell_start[q], je = cell_start[q + 1];
            if (js == je) continue;
            const double L = g.box;
            const double ix = ux < 0 ? -L : (ux >= nc ? L : 0.0);
            const double iy = uy < 0 ? -L : (uy >= nc ? L : 0.0);
            const double iz = uz < 0 ? -L : (uz >= nc ? L : 0.0);
            const float cxs = (float)(xa - ix), cys = (float)(ya - iy), czs = (float)(za - iz);
            double ox = 0, oy = 0, oz = 0;
            for (uint32_t b = js >> 5; b * 32u < je; ++b) {
                const float4 lo = __ldg(block_box + 2 * b), hi = __ldg(block_box + 2 * b + 1);
                const float ex = fmaxf(fmaxf(lo.x - cxs, cxs - hi.x), 0.0f);
                const float ey = fmaxf(fmaxf(lo.y - cys, cys - hi.y), 0.0f);
                const float ez = fmaxf(fmaxf(lo.z - czs, czs - hi.z), 0.0f);
                if (!__any_sync(0xffffffffu, valid && ex * ex + ey * ey + ez * ez < rcull2)) continue;
                const float fx = fmaxf(cxs - lo.x, hi.x - cxs);
                const float fy = fmaxf(cys - lo.y, hi.y - cys);
                const float fz = fmaxf(czs - lo.z, hi.z - czs);
                const bool all_in =
                    __all_sync(0xffffffffu, !valid || fx * fx + fy * fy + fz * fz < rin2);
                const uint32_t j0 = max(b * 32, js), j1 = min(b * 32 + 32, je);
                // the block's particles: one coalesced load, then broadcast lane by lane
                const uint32_t jl = min(b * 32 + lane, (uint32_t)(n - 1));
                const double4_16a ql = rel[jl];
                const double vlx = vs[jl], vly = vs[n + jl], vlz = vs[2 * n + jl];
                for (uint32_t j = j0; j < j1; ++j) {
                    const int src = (int)(j - b * 32);
                    const double dx = (__shfl_sync(0xffffffffu, ql.x, src) - xi.x) + ix;
                    const double dy = (__shfl_sync(0xffffffffu, ql.y, src) - xi.y) + iy;
                    const double dz = (__shfl_sync(0xffffffffu, ql.z, src) - xi.z) + iz;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    const bool in = valid && (all_in || r2 < rc2) && r2 > 0.0;
                    const double w0 = __shfl_sync(0xffffffffu, vlx, src) - vix;
                    const double w1 = __shfl_sync(0xffffffffu, vly, src) - viy;
                    const double w2 = __shfl_sync(0xffffffffu, vlz, src) - viz;
                    if (!all_in && !__any_sync(0xffffffffu, in)) continue;
                    double h, hr;
                    pair_jac(r2, eps2, inv_rs, h, hr);
                    const double dw = dx * w0 + dy * w1 + dz * w2;
                    const double c = in ? hr * dw : 0.0;
                    const double hh = in ? h : 0.0;
                    ox += hh * w0 + c * dx;
                    oy += hh * w1 + c * dy;
                    oz += hh * w2 + c * dz;
                }
            }
            o[0] += ox;
            o[1] += oy;
            o[2] += oz;
        }
        if (valid) {
            out[i] += g.gm * o[0];
            out[n + i] += g.gm * o[1];
            out[2 * n + i] += g.gm * o[2];
        }
    }
}

// FP32 mode: the force kernel's traversal and arithmetic style (one-warp persistent CTAs,
// bulk-copy tiles of the block-SoA coordinates and v, block culling, the all-inside fast path,
// two j particles per lane in packed f32x2, per-tile FP32 sums added in FP64), for
//   out_k += Gm sum_j [h(r) w + (h'(r)/r)(d.w) d],  w = v_j - v_k,
//   h = g s^3, h'/r = -(r e / (2 sqrt(pi) r_s^3)) s^3 - 3 h s^2,  s = (r^2 + eps^2)^-1/2,
//   e = exp(-r^2 / (4 r_s^2)),
// g from the fitted polynomial (g'(x) = -x^2 exp(-x^2/4) / (2 sqrt(pi)) in closed form).  r^2
// starts at kVjpTiny = 1e-20 like in the force kernel; r = 0 pairs are selected out (their w need
// not vanish for coincident particles).  r^2 = kVjpTiny can only occur in the work item's own
// cell (the particle itself, coincident particles), so only the own cell tests r^2 > kVjpTiny.
// Tiles of 3 blocks of coordinates and v (4.5 KB for both buffers) keep 32 CTAs per SM.
constexpr float kVjpTiny = 1e-20f;
constexpr int kVjpBlocksPerTile = 3;

// 2^x (MUFU); here x in [-7.3, 0], no denormal results
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct VjpConst2 {
    f2 c[P3M_SPLIT_DEG + 1];
    f2 c11, m1, one, eps2, tiny, ex2arg, c1, m3;
};

// h and h'/r of both halves of r2 (r2 includes kVjpTiny)
__device__ __forceinline__ void pair_jac2(f2 r2, const VjpConst2 &k, f2 &h, f2 &hr)
{
    float r2l, r2h, s2l, s2h, al, ah;
    const f2 s2 = f2_add(r2, k.eps2);
    f2_unpack(r2, r2l, r2h);
    f2_unpack(s2, s2l, s2h);
    const f2 s = f2_pack(rsqrt_approx(s2l), rsqrt_approx(s2h));
    const f2 r = f2_pack(sqrt_approx(r2l), sqrt_approx(r2h));
    const f2 tau = f2_fma(r2, k.c11, k.m1);
    f2 p = k.c[P3M_SPLIT_DEG];
#pragma unroll
    for (int q = P3M_SPLIT_DEG - 1; q >= 0; --q) p = f2_fma(p, tau, k.c[q]);
    const f2 gval = f2_fma(f2_mul(r2, r), p, k.one);
    const f2 ss = f2_mul(s, s);
    const f2 s3 = f2_mul(ss, s);
    h = f2_mul(gval, s3);
    f2_unpack(f2_mul(r2, k.ex2arg), al, ah);  // -r^2 log2(e) / (4 r_s^2)
    const f2 e = f2_pack(ex2_approx(al), ex2_approx(ah));
    const f2 res3 = f2_mul(f2_mul(r, e), s3);
    hr = f2_fma(res3, k.c1, f2_mul(f2_mul(h, ss), k.m3));  // c1 = -1/(2 sqrt(pi) r_s^3), m3 = -3
}

__global__ void __launch_bounds__(32, 32)
    k_pairs_vjp_x2(const float *__restrict__ relx, const float *__restrict__ vfx,
                   const float4 *__restrict__ rel, const double *__restrict__ pos,
                   const float4 *__restrict__ block_box, const uint32_t *__restrict__ cell_start,
                   const uint32_t *__restrict__ work, const uint32_t *__restrict__ order,
                   const uint32_t *__restrict__ n_work_ptr, P3MGeom g, GPolyA gp, float rcull2,
                   float rin2, uint32_t *__restrict__ cursor, uint32_t *__restrict__ flags,
                   double *__restrict__ out)
{
    constexpr int kBlockFloats = 96;
    __shared__ __align__(128) float sj[2][kVjpBlocksPerTile * kBlockFloats];
    __shared__ __align__(128) float sv[2][kVjpBlocksPerTile * kBlockFloats];
    __shared__ __align__(16) float4 sbox[2][2 * kVjpBlocksPerTile];  // the tile's block boxes
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ NeighbourF nbr[27];

    const int lane = threadIdx.x;
    const int64_t n = g.n;
    const uint32_t n_work = *n_work_ptr;
    const float rc2 = (float)(g.r_c * g.r_c);
    const int nc = g.n_c;
    VjpConst2 kc;
#pragma unroll
    for (int q = 0; q <= P3M_SPLIT_DEG; ++q) kc.c[q] = f2_pack(gp.c[q], gp.c[q]);
    kc.c11 = f2_pack(gp.c[11], gp.c[11]);
    kc.m1 = f2_pack(-1.0f, -1.0f);
    kc.one = f2_pack(1.0f, 1.0f);
    const float e2 = (float)(g.eps * g.eps);
    kc.eps2 = f2_pack(e2, e2);
    kc.tiny = f2_pack(kVjpTiny, kVjpTiny);
    const float xa_ = (float)(-1.4426950408889634 / (4.0 * g.r_s * g.r_s));
    kc.ex2arg = f2_pack(xa_, xa_);
    const float c1 = (float)(-0.28209479177387814347 / (g.r_s * g.r_s * g.r_s));
    kc.c1 = f2_pack(c1, c1);
    kc.m3 = f2_pack(-3.0f, -3.0f);

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
        const uint32_t item = order[slot];
        const uint32_t cell = work[2 * (size_t)item];
        const uint32_t first = work[2 * (size_t)item + 1];
        const uint32_t cend = cell_start[cell + 1];
        const int cx = (int)(cell % nc), cy = (int)((cell / nc) % nc), cz = (int)(cell / (nc * nc));
        __syncwarp();  // the previous item is done with nbr
        if (lane < 27) nbr[lane] = make_neighbour(g, cell_start, cx, cy, cz, lane);
        __syncwarp();

        const uint32_t i = first + lane;
        const bool valid = i < cend;
        const uint32_t ii = valid ? i : first;
        const float4 xi = rel[ii];
        const float xa = (float)pos[ii], ya = (float)pos[n + ii], za = (float)pos[2 * n + ii];
        const float *vi = vfx + (ii >> 5) * kBlockFloats + (ii & 31);
        const f2 vix2 = f2_pack(vi[0], vi[0]), viy2 = f2_pack(vi[32], vi[32]),
                 viz2 = f2_pack(vi[64], vi[64]);
        double sox = 0.0, soy = 0.0, soz = 0.0;

        auto next_tile = [&](int &nb, uint32_t &b) {
            while (nb < 27 && b * 32u >= nbr[nb].end) {
                ++nb;
                if (nb < 27) b = nbr[nb].start >> 5;
            }
        };
        auto issue = [&](int nb, uint32_t b, int to) {
            const uint32_t bend = min(b + kVjpBlocksPerTile, (nbr[nb].end + 31) >> 5);
            const uint32_t bytes = (bend - b) * (uint32_t)(kBlockFloats * sizeof(float));
            const uint32_t box_bytes = (bend - b) * (uint32_t)(2 * sizeof(float4));
            mbar_expect_tx(&bar[to], 2 * bytes + box_bytes);
            bulk_load(&sj[to][0], relx + (size_t)b * kBlockFloats, bytes, &bar[to]);
            bulk_load(&sv[to][0], vfx + (size_t)b * kBlockFloats, bytes, &bar[to]);
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
            const uint32_t bend = min(b_c + kVjpBlocksPerTile, (nend + 31) >> 5);
            int nb_n = nb_c;
            uint32_t b_n = bend;
            next_tile(nb_n, b_n);
            __syncwarp();  // every lane is done with the other buffer before it is refilled
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
            f2 ox = make_float2(0.0f, 0.0f), oy = ox, oz = ox;

            // pair (j, j+1) from packed coordinates (x, y, z) and v (u, v, w); lo/hi: which
            // halves take part; test: r < r_c; own: the work item's own cell (r^2 > kVjpTiny test)
            auto pair_vjp = [&](auto own, f2 xj, f2 yj, f2 zj, f2 uj, f2 vj, f2 wj, bool lo,
                                bool hi, bool test) {
                const f2 dx = f2_sub(xj, xs2), dy = f2_sub(yj, ys2), dz = f2_sub(zj, zs2);
                const f2 r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_fma(dx, dx, kc.tiny)));
                float r2l, r2h;
                f2_unpack(r2, r2l, r2h);
                const bool own_c = decltype(own)::value;
                const bool inl = lo && (!own_c || r2l > kVjpTiny) && (!test || r2l < rc2);
                const bool inh = hi && (!own_c || r2h > kVjpTiny) && (!test || r2h < rc2);
                if (test && !__any_sync(0xffffffffu, inl || inh)) return;
                f2 h, hr;
                pair_jac2(r2, kc, h, hr);
                const f2 wx = f2_sub(uj, vix2), wy = f2_sub(vj, viy2), wz = f2_sub(wj, viz2);
                const f2 dw = f2_fma(dz, wz, f2_fma(dy, wy, f2_mul(dx, wx)));
                f2 hs = h, cs = f2_mul(hr, dw);
                if (own_c || test || !(lo && hi)) {
                    float hl, hh, cl, ch;
                    f2_unpack(hs, hl, hh);
                    f2_unpack(cs, cl, ch);
                    hs = f2_pack(inl ? hl : 0.0f, inh ? hh : 0.0f);
                    cs = f2_pack(inl ? cl : 0.0f, inh ? ch : 0.0f);
                }
                ox = f2_fma(cs, dx, f2_fma(hs, wx, ox));
                oy = f2_fma(cs, dy, f2_fma(hs, wy, oy));
                oz = f2_fma(cs, dz, f2_fma(hs, wz, oz));
            };
            // the aligned pair (p, p+1) of the block at bx / bv
            auto pair_at = [&](auto own, const float *bx, const float *bv, uint32_t p, bool lo,
                               bool hi, bool test) {
                const f2 *x2 = (const f2 *)bx, *v2 = (const f2 *)bv;
                pair_vjp(own, x2[p / 2], x2[16 + p / 2], x2[32 + p / 2], v2[p / 2], v2[16 + p / 2],
                         v2[32 + p / 2], lo, hi, test);
            };

            auto blocks = [&](auto own) {
            for (uint32_t b = b_c; b < bend; ++b) {
                const float4 lo = sbox[buf][2 * (b - b_c)], hi = sbox[buf][2 * (b - b_c) + 1];
                const float ex = fmaxf(fmaxf(lo.x - cxs, cxs - hi.x), 0.0f);
                const float ey = fmaxf(fmaxf(lo.y - cys, cys - hi.y), 0.0f);
                const float ez = fmaxf(fmaxf(lo.z - czs, czs - hi.z), 0.0f);
                if (!__any_sync(0xffffffffu, valid && ex * ex + ey * ey + ez * ez < rcull2)) continue;
                const uint32_t j0 = max(b * 32, nstart) - b * 32;
                const uint32_t j1 = min(b * 32 + 32, nend) - b * 32;
                const float *bx = sj[buf] + (b - b_c) * kBlockFloats;
                const float *bv = sv[buf] + (b - b_c) * kBlockFloats;
                const float fx = fmaxf(cxs - lo.x, hi.x - cxs);
                const float fy = fmaxf(cys - lo.y, hi.y - cys);
                const float fz = fmaxf(czs - lo.z, hi.z - czs);
                const bool test =
                    !__all_sync(0xffffffffu, !valid || fx * fx + fy * fy + fz * fz < rin2);
                uint32_t p = j0 & ~1u;
                if ((j0 & 1u) && j0 < j1) {
                    pair_at(own, bx, bv, p, false, true, true);
                    p += 2;
                }
                if (test) {
                    for (; p + 1 < j1; p += 2) pair_at(own, bx, bv, p, true, true, true);
                } else {
                    if ((p & 2u) && p + 1 < j1) {
                        pair_at(own, bx, bv, p, true, true, false);
                        p += 2;
                    }
                    for (; p + 3 < j1; p += 4) {  // four j: 16-byte loads
                        const float4 X = *(const float4 *)(bx + p), Y = *(const float4 *)(bx + 32 + p),
                                     Z = *(const float4 *)(bx + 64 + p);
                        const float4 U = *(const float4 *)(bv + p), V = *(const float4 *)(bv + 32 + p),
                                     W = *(const float4 *)(bv + 64 + p);
                        pair_vjp(own, f2_pack(X.x, X.y), f2_pack(Y.x, Y.y), f2_pack(Z.x, Z.y),
                                 f2_pack(U.x, U.y), f2_pack(V.x, V.y), f2_pack(W.x, W.y), true, true,
                                 false);
                        pair_vjp(own, f2_pack(X.z, X.w), f2_pack(Y.z, Y.w), f2_pack(Z.z, Z.w),
                                 f2_pack(U.z, U.w), f2_pack(V.z, V.w), f2_pack(W.z, W.w), true, true,
                                 false);
                    }
                    for (; p + 1 < j1; p += 2) pair_at(own, bx, bv, p, true, true, false);
                }
                if (p < j1) pair_at(own, bx, bv, p, true, false, true);
            }
            };
            if (nb_c == 13)
                blocks(std::true_type{});
            else
                blocks(std::false_type{});
            float lo_, hi_;
            f2_unpack(ox, lo_, hi_);
            sox += (double)(lo_ + hi_);
            f2_unpack(oy, lo_, hi_);
            soy += (double)(lo_ + hi_);
            f2_unpack(oz, lo_, hi_);
            soz += (double)(lo_ + hi_);
            buf ^= 1;
            nb_c = nb_n;
            b_c = b_n;
        }
        if (timed_out) break;
        if (valid) {
            out[i] += g.gm * sox;
            out[n + i] += g.gm * soy;
            out[2 * n + i] += g.gm * soz;
        }
    }
    if (timed_out && lane == 0) atomicOr(flags, P3M_FLAG_TIMEOUT);
}

// ------------------------------------------------------------------ potential energy

// phi_k = G(k) rho_k (the potential spectrum of the forward pass, no gradient).
template <typename T, typename C2>
__global__ void k_kspace_potential(const C2 *__restrict__ rk, const T *__restrict__ tk,
                                   const T *__restrict__ tg, int M, T gconst, int green_only,
                                   C2 *__restrict__ out)
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
        C2 o;
        if (green_only) {  // the kernel K = IFFT(G) itself
            o.x = G;
            o.y = T(0);
        } else {
            const C2 r = rk[idx];
            o.x = G * r.x;
            o.y = G * r.y;
        }
        out[idx] = o;
    }
}

// Per particle: Phi_LR(x_k) - S_k, S_k = sum_{c,c'} w_c w_c' K(n_c - n_c') (kself: K at the
// 27 offsets {-1,0,1}^3, index (dx+1)*9 + (dy+1)*3 + (dz+1)); phi_out[k] = that + cst.
template <typename T>
__global__ void k_gather_potential(const double *__restrict__ pos, P3MGeom g,
                                   const T *__restrict__ phi_mesh, const double *__restrict__ kself,
                                   double cst, double *__restrict__ phi_out)
{
    const int M = g.mesh;
    const int64_t n = g.n;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int i3[3];
        double f3[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) stencil64(pos[d * n + k], g.inv_h, i3[d], f3[d]);
        double w[8];
        double phi = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int a = c >> 2, b = (c >> 1) & 1, e = c & 1;
            w[c] = (a ? f3[0] : 1.0 - f3[0]) * (b ? f3[1] : 1.0 - f3[1]) * (e ? f3[2] : 1.0 - f3[2]);
            const size_t node = ((size_t)wrap_index(i3[0] + a, M) * M + wrap_index(i3[1] + b, M)) * M +
                                wrap_index(i3[2] + e, M);
            phi += w[c] * (double)phi_mesh[node];
        }
        double self = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                const int dx = (c >> 2) - (d >> 2), dy = ((c >> 1) & 1) - ((d >> 1) & 1),
                          dz = (c & 1) - (d & 1);
                self += w[c] * w[d] * kself[(dx + 1) * 9 + (dy + 1) * 3 + (dz + 1)];
            }
        phi_out[k] = phi - self + cst;
    }
}

// Short-range pair potential: phi_out[k] += -Gm sum_j erfc(r/(2 r_s)) / sqrt(r^2 + eps^2),
// the pair kernel's traversal (work items, block culling, shuffled j blocks).
template <typename T>
__global__ void __launch_bounds__(32)
    k_pairs_potential(const typename V4Of<T>::type *__restrict__ rel, const double *__restrict__ pos,
                      const float4 *__restrict__ block_box, const uint32_t *__restrict__ cell_start,
                      const uint32_t *__restrict__ work, const uint32_t *__restrict__ order,
                      const uint32_t *__restrict__ n_work_ptr, P3MGeom g, float rcull2,
                      uint32_t *__restrict__ cursor, double *__restrict__ phi_out)
{
    using V4 = typename V4Of<T>::type;
    constexpr bool kAbsolute = sizeof(T) == 8;
    const int lane = threadIdx.x;
    const int64_t n = g.n;
    const uint32_t n_work = *n_work_ptr;
    const T rc2 = (T)(g.r_c * g.r_c), eps2 = (T)(g.eps * g.eps), half_inv_rs = (T)(0.5 / g.r_s);
    const int nc = g.n_c;
    for (;;) {
        uint32_t slot = 0;
        if (lane == 0) slot = atomicAdd(cursor, 1u);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot >= n_work) break;
        const uint32_t item = order[slot];
        const uint32_t cell = work[2 * (size_t)item], first = work[2 * (size_t)item + 1];
        const uint32_t cend = cell_start[cell + 1];
        const int cx = (int)(cell % nc), cy = (int)((cell / nc) % nc), cz = (int)(cell / (nc * nc));
        const uint32_t i = first + lane;
        const bool valid = i < cend;
        const uint32_t ii = valid ? i : first;
        const V4 xi = rel[ii];
        const double xa = pos[ii], ya = pos[n + ii], za = pos[2 * n + ii];
        double acc = 0.0;
        for (int nb = 0; nb < 27; ++nb) {
            const int ux = cx + nb % 3 - 1, uy = cy + (nb / 3) % 3 - 1, uz = cz + nb / 9 - 1;
            const int wx = (ux + nc) % nc, wy = (uy + nc) % nc, wz = (uz + nc) % nc;
            const uint32_t q = ((uint32_t)wz * nc + wy) * nc + wx;
            const uint32_t js = cell_start[q], je = cell_start[q + 1];
            if (js == je) continue;
            const double L = g.box, cs = g.cs;
            const double imx = ux < 0 ? -L : (ux >= nc ? L : 0.0);
            const double imy = uy < 0 ? -L : (uy >= nc ? L : 0.0);
            const double imz = uz < 0 ? -L : (uz >= nc ? L : 0.0);
            T xs, ys, zs, ix = 0, iy = 0, iz = 0;
            if (kAbsolute) {
                xs = (T)xi.x;
                ys = (T)xi.y;
                zs = (T)xi.z;
                ix = (T)imx;
                iy = (T)imy;
                iz = (T)imz;
            } else {
                xs = (T)((double)xi.x - (((double)wx * cs + imx) - (double)cx * cs));
                ys = (T)((double)xi.y - (((double)wy * cs + imy) - (double)cy * cs));
                zs = (T)((double)xi.z - (((double)wz * cs + imz) - (double)cz * cs));
            }
            const float cxs = (float)(xa - imx), cys = (float)(ya - imy), czs = (float)(za - imz);
            T s = 0;
            for (uint32_t b = js >> 5; b * 32u < je; ++b) {
                const float4 lo = __ldg(block_box + 2 * b), hi = __ldg(block_box + 2 * b + 1);
                const float ex = fmaxf(fmaxf(lo.x - cxs, cxs - hi.x), 0.0f);
                const float ey = fmaxf(fmaxf(lo.y - cys, cys - hi.y), 0.0f);
                const float ez = fmaxf(fmaxf(lo.z - czs, czs - hi.z), 0.0f);
                if (!__any_sync(0xffffffffu, valid && ex * ex + ey * ey + ez * ez < rcull2)) continue;
                const uint32_t j0 = max(b * 32, js), j1 = min(b * 32 + 32, je);
                const uint32_t jl = min(b * 32 + lane, (uint32_t)(n - 1));
                const V4 ql = rel[jl];
                for (uint32_t j = j0; j < j1; ++j) {
                    const int src = (int)(j - b * 32);
                    T dx = __shfl_sync(0xffffffffu, (T)ql.x, src) - xs;
                    T dy = __shfl_sync(0xffffffffu, (T)ql.y, src) - ys;
                    T dz = __shfl_sync(0xffffffffu, (T)ql.z, src) - zs;
                    if (kAbsolute) {
                        dx += ix;
                        dy += iy;
                        dz += iz;
                    }
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    const bool in = valid && r2 < rc2 && r2 > T(0);
                    if (!__any_sync(0xffffffffu, in)) continue;
                    const T term = erfc(sqrt(r2) * half_inv_rs) / sqrt(r2 + eps2);
                    s += in ? term : T(0);
                }
            }
            acc += (double)s;
        }
        if (valid) phi_out[i] -= g.gm * acc;
    }
}

// Sum of m/2 phi over particles, per-block partials then one block (fixed order).
__global__ void __launch_bounds__(256) k_sum_vec(const double *__restrict__ x, int64_t n, double *part)
{
    __shared__ double s[256];
    double a = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        a += x[k];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

template <typename T, typename C2>
cudaError_t potential_impl(p3m_ctx *c, double cst, double *phi_slots, double *sum_dev)
{
    const int M = c->g.mesh;
    const size_t nk = (size_t)M * M * (M / 2 + 1);
    C2 *spec = (C2 *)c->frc_k;  // free after the force evaluation; FFT(rho) stays in rho_k
    T *mesh = (T *)c->adj_u;
    const int gk = grid_for((int64_t)nk, 256, c->num_sms);
    c->launches += 2;
    if (!c->kself_ready) {  // K = IFFT(G) near the origin, once per context
        k_kspace_potential<T, C2><<<gk, 256, 0, c->stream>>>(spec, (const T *)c->tab_k,
                                                             (const T *)c->tab_g, M,
                                                             (T)c->green_const, 1, spec);
        cufftResult r = sizeof(T) == 4 ? cufftExecC2R(c->plan_c2r_one, (cufftComplex *)spec, (cufftReal *)mesh)
                                       : cufftExecZ2D(c->plan_c2r_one, (cufftDoubleComplex *)spec,
                                                      (cufftDoubleReal *)mesh);
        if (r != CUFFT_SUCCESS) return cudaErrorUnknown;
        std::vector<T> host((size_t)M * M * M);
        double k27[27];
        cudaError_t e = cudaMemcpyAsync(host.data(), mesh, sizeof(T) * host.size(), cudaMemcpyDeviceToHost,
                                        c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return e;
        for (int t = 0; t < 27; ++t) {
            const int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
            const size_t node = ((size_t)((dx + M) % M) * M + (dy + M) % M) * M + (dz + M) % M;
            k27[t] = (double)host[node];
        }
        e = cudaMemcpyAsync(c->kself, k27, sizeof(k27), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return e;
        c->kself_ready = true;
    }
    // potential mesh from the current deposit (c->rho_k holds FFT(rho) after launch_deposit + R2C)
    k_kspace_potential<T, C2><<<gk, 256, 0, c->stream>>>((const C2 *)c->rho_k, (const T *)c->tab_k,
                                                         (const T *)c->tab_g, M, (T)c->green_const, 0,
                                                         spec);
    cufftResult r = sizeof(T) == 4 ? cufftExecC2R(c->plan_c2r_one, (cufftComplex *)spec, (cufftReal *)mesh)
                                   : cufftExecZ2D(c->plan_c2r_one, (cufftDoubleComplex *)spec,
                                                  (cufftDoubleReal *)mesh);
    if (r != CUFFT_SUCCESS) return cudaErrorUnknown;
    c->launches += 1;
    k_gather_potential<T><<<grid_for(c->g.n, 256, c->num_sms), 256, 0, c->stream>>>(
        c->pos, c->g, mesh, c->kself, cst, phi_slots);
    if (c->short_range) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs_potential<T>, 32, 0);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(c->counters + 3, 0, sizeof(uint32_t), c->stream);
        if (e != cudaSuccess) return e;
        const double rcull = c->g.r_c * (1.0 + 1e-4) + c->g.box * 1e-6;
        c->launches += 1;
        k_pairs_potential<T><<<c->num_sms * (per_sm < 1 ? 1 : per_sm), 32, 0, c->stream>>>(
            (const typename V4Of<T>::type *)c->rel, c->pos, c->block_box, c->cell_start, c->work,
            c->work_order, c->work_off + c->g.n_cells, c->g, (float)(rcull * rcull), c->counters + 3,
            phi_slots);
    }
    c->launches += 2;
    k_sum_vec<<<1024, 256, 0, c->stream>>>(phi_slots, c->g.n, c->red);
    k_sum_parts<<<1, 256, 0, c->stream>>>(c->red, 1024, sum_dev);
    return cudaGetLastError();
}

template <typename T, typename C2>
cudaError_t vjp_mesh(p3m_ctx *c, const double *v_slots, double *out_slots)
{
    const int M = c->g.mesh;
    const size_t M3 = (size_t)M * M * M, nk = (size_t)M * M * (M / 2 + 1);
    T *u = (T *)c->adj_u;
    unsigned long long *maxbits = (unsigned long long *)(c->fix_exp + 2);
    cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->rho_fix, 0, 3 * M3 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    int nb = 0;
    while (nb < 63 && (c->g.n >> nb)) ++nb;
    const int gn = grid_for(c->g.n, 256, c->num_sms);
    c->launches += 6;
    k_absmax_bits<<<gn, 256, 0, c->stream>>>(v_slots, 3 * c->g.n, maxbits);
    k_fix_exponent<<<1, 1, 0, c->stream>>>(maxbits, nb, c->fix_exp);
    k_deposit_vec<<<gn, 256, 0, c->stream>>>(c->pos, v_slots, c->g, c->fix_exp, c->rho_fix);
    k_fix_to_vec<T><<<grid_for((int64_t)(3 * M3), 256, c->num_sms), 256, 0, c->stream>>>(c->rho_fix, 3 * M3,
                                                                                       c->fix_exp, u);
    C2 *uk = (C2 *)c->frc_k;
    for (int b = 0; b < 3; ++b) {
        cufftResult r = sizeof(T) == 4
                            ? cufftExecR2C(c->plan_r2c, (cufftReal *)(u + b * M3), (cufftComplex *)(uk + b * nk))
                            : cufftExecD2Z(c->plan_r2c, (cufftDoubleReal *)(u + b * M3),
                                           (cufftDoubleComplex *)(uk + b * nk));
        if (r != CUFFT_SUCCESS) return cudaErrorUnknown;
    }
    C2 *psik = (C2 *)c->rho_k;
    k_kspace_adjoint<T, C2><<<grid_for((int64_t)nk, 256, c->num_sms), 256, 0, c->stream>>>(
        uk, uk + nk, uk + 2 * nk, (const T *)c->tab_k, (const T *)c->tab_kg, (const T *)c->tab_g, M,
        (T)c->green_const, psik);
    T *psi = (T *)c->rho;
    cufftResult r = sizeof(T) == 4 ? cufftExecC2R(c->plan_c2r_one, (cufftComplex *)psik, (cufftReal *)psi)
                                   : cufftExecZ2D(c->plan_c2r_one, (cufftDoubleComplex *)psik,
                                                  (cufftDoubleReal *)psi);
    if (r != CUFFT_SUCCESS) return cudaErrorUnknown;
    k_gather_grad<T><<<grid_for(c->g.n, 256, c->num_sms), 256, 0, c->stream>>>(
        c->pos, c->g, (const T *)c->frc, v_slots, psi, 1.0, out_slots);
    return cudaGetLastError();
}

cudaError_t vjp_pairs(p3m_ctx *c, const double *v_slots, double *out_slots)
{
    int per_sm = 0;
    const bool fp32 = c->precision == P3M_PREC_MIXED;
    cudaError_t e = fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs_vjp_x2, 32, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs_vjp64, 32, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    e = cudaMemsetAsync(c->counters + 3, 0, sizeof(uint32_t), c->stream);
    if (e != cudaSuccess) return e;
    const double rcull = c->g.r_c * (1.0 + 1e-4) + c->g.box * 1e-6;
    const double rin = c->g.r_c * (1.0 - 1e-4) - c->g.box * 1e-6;
    const float rcull2 = (float)(rcull * rcull), rin2 = rin > 0.0 ? (float)(rin * rin) : 0.0f;
    c->launches += 1;
    if (fp32) {
        GPolyA gp;
        for (int k = 0; k < 12; ++k) gp.c[k] = c->gpoly[k];
        k_pairs_vjp_x2<<<c->num_sms * per_sm, 32, 0, c->stream>>>(
            c->relx, c->adj_vfx, (const float4 *)c->rel, c->pos, c->block_box, c->cell_start, c->work,
            c->work_order, c->work_off + c->g.n_cells, c->g, gp, rcull2, rin2, c->counters + 3,
            c->counters + 1, out_slots);
    } else {
        k_pairs_vjp64<<<c->num_sms * per_sm, 32, 0, c->stream>>>(
            (const double4_16a *)c->rel, c->pos, c->block_box, v_slots, c->cell_start, c->work,
            c->work_order, c->work_off + c->g.n_cells, c->g, rcull2, rin2, c->counters + 3,
            out_slots);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_to_slots(p3m_ctx *c, const double *v, double *vs)
{
    c->launches += 1;
    k_to_slots<<<grid_for(c->g.n, 256, c->num_sms), 256, 0, c->stream>>>(
        v, c->pid, c->g.n, vs, c->precision == P3M_PREC_MIXED ? c->adj_vfx : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_force_vjp(p3m_ctx *c, const double *v_slots, double *out_slots)
{
    cudaError_t e = cudaMemsetAsync(out_slots, 0, 3 * sizeof(double) * c->g.n, c->stream);
    if (e != cudaSuccess) return e;
    if (c->precision == P3M_PREC_MIXED) {
        e = vjp_mesh<float, cufftComplex>(c, v_slots, out_slots);
        if (e == cudaSuccess && c->short_range) e = vjp_pairs(c, v_slots, out_slots);
    } else {
        e = vjp_mesh<double, cufftDoubleComplex>(c, v_slots, out_slots);
        if (e == cudaSuccess && c->short_range) e = vjp_pairs(c, v_slots, out_slots);
    }
    return e;
}

cudaError_t launch_potential(p3m_ctx *c, double cst, double *phi_slots, double *sum_dev)
{
    return c->precision == P3M_PREC_MIXED ? potential_impl<float, cufftComplex>(c, cst, phi_slots, sum_dev)
                                          : potential_impl<double, cufftDoubleComplex>(c, cst, phi_slots, sum_dev);
}

cudaError_t launch_density_loss(p3m_ctx *c, const double *target, double *loss_dev, double *grad_slots)
{
    const int M = c->g.mesh;
    const size_t M3 = (size_t)M * M * M;
    const double inv_nbar = 1.0 / c->g.mean_count;
    const int nb = 1024;
    c->launches += 2;
    if (c->precision == P3M_PREC_MIXED)
        k_loss_mesh<float><<<nb, 256, 0, c->stream>>>((float *)c->rho, target, M3, inv_nbar, c->red);
    else
        k_loss_mesh<double><<<nb, 256, 0, c->stream>>>((double *)c->rho, target, M3, inv_nbar, c->red);
    k_sum_parts<<<1, 256, 0, c->stream>>>(c->red, nb, loss_dev);
    if (grad_slots) {
        cudaError_t e = cudaMemsetAsync(grad_slots, 0, 3 * sizeof(double) * c->g.n, c->stream);
        if (e != cudaSuccess) return e;
        c->launches += 1;
        if (c->precision == P3M_PREC_MIXED)
            k_gather_grad<float><<<grid_for(c->g.n, 256, c->num_sms), 256, 0, c->stream>>>(
                c->pos, c->g, nullptr, nullptr, (const float *)c->rho, 1.0, grad_slots);
        else
            k_gather_grad<double><<<grid_for(c->g.n, 256, c->num_sms), 256, 0, c->stream>>>(
                c->pos, c->g, nullptr, nullptr, (const double *)c->rho, 1.0, grad_slots);
    }
    return cudaGetLastError();
}
