// lbib_device.cuh -- device helpers shared by the library's kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lbib_internal.cuh"

namespace lbib {

// D2Q9 weights printed after Eq. 3 (rest 4/9, axis 1/9, diagonal 1/36).
// Programmatic dependent launch: pdl_wait blocks until the grids this one
// depends on have completed and their writes are visible (it returns at once
// when the launch had no programmatic dependency); pdl_trigger lets the
// dependent grid be scheduled once every block of this one has issued it or
// exited.  Every thread of a block issues both at the same point.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename R>
__device__ __forceinline__ R wq(int q)
{
    return q == 0 ? R(4) / R(9) : (q < 5 ? R(1) / R(9) : R(1) / R(36));
}

// ------------------------------------------------------------ storage types
template <typename S, typename R>
__device__ __forceinline__ R ld(const S* p)
{
    return static_cast<R>(__ldg(p));
}
template <typename S, typename R>
__device__ __forceinline__ void st(S* p, R v)
{
    *p = static_cast<S>(v);
}
// 16-bit storage of FP32 deviations: bfloat16 as is (round to nearest even);
// binary16 scaled by HALF_SCALE (exact power of two) on the way in and out
template <>
__device__ __forceinline__ float ld<__nv_bfloat16, float>(const __nv_bfloat16* p)
{
    return __bfloat162float(__ldg(p));
}
template <>
__device__ __forceinline__ void st<__nv_bfloat16, float>(__nv_bfloat16* p, float v)
{
    *p = __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ float ld<__half, float>(const __half* p)
{
    return __half2float(__ldg(p)) * (1.0f / HALF_SCALE);
}
template <>
__device__ __forceinline__ void st<__half, float>(__half* p, float v)
{
    *p = __float2half_rn(v * HALF_SCALE);
}

// The same conversions from a stored value already loaded (from shared memory)
template <typename S, typename R>
__device__ __forceinline__ R from_store(S v)
{
    return static_cast<R>(v);
}
template <>
__device__ __forceinline__ float from_store<__nv_bfloat16, float>(__nv_bfloat16 v)
{
    return __bfloat162float(v);
}
template <>
__device__ __forceinline__ float from_store<__half, float>(__half v)
{
    return __half2float(v) * (1.0f / HALF_SCALE);
}

// ------------------------------------------------------- Peskin 4-point kernel
// phi(a), a = |r|: (3 - 2a + sqrt(2 - 4 (a - 1/2)^2)) / 8 on [0, 1],
// (5 - 2a - sqrt(2 - 4 (a - 3/2)^2)) / 8 on (1, 2], zero beyond (Peskin 2002).
template <typename R>
__device__ __forceinline__ R peskin(R r)
{
    R a = fabs(r);
    if (a <= R(1)) {
        R t = a - R(0.5);
        return (R(3) - R(2) * a + sqrt(R(2) - R(4) * t * t)) * R(0.125);
    }
    if (a <= R(2)) {
        R t = a - R(1.5);
        return (R(5) - R(2) * a - sqrt(R(2) - R(4) * t * t)) * R(0.125);
    }
    return R(0);
}

// ------------------------------------------ moving-least-squares transfer
// Weight along one direction: the cubic spline of q = |r| / 2,
// 2/3 - 4 q^2 + 4 q^3 on [0, 1/2], (4/3) (1 - q)^3 on (1/2, 1], zero beyond,
// so its support is the 4 x 4 stencil of the Peskin kernel.
template <typename R>
__device__ __forceinline__ R mls_w(R r)
{
    const R q = fabs(r) * R(0.5);
    if (q <= R(0.5)) return R(2.0 / 3.0) - R(4) * q * q + R(4) * q * q * q;
    if (q < R(1)) {
        const R t = R(1) - q;
        return R(4.0 / 3.0) * t * t * t;
    }
    return R(0);
}

// Inverse of the MLS moment matrix A = sum_j W_j p_j p_j^T for the linear
// basis p = (1, dx, dy) and separable weights W = wx(dx) wy(dy) over a
// product stencil, from the 1-D moments a_k = sum wx dx^k, b_k = sum wy dy^k:
// A = [[a0 b0, a1 b0, a0 b1], [a1 b0, a2 b0, a1 b1], [a0 b1, a1 b1, a0 b2]].
// Row r of the inverse gives the shape functions W_j (inv_r . p_j) of the
// value (r = 0) and of the x- and y-derivatives (r = 1, 2).  False when A is
// singular (fewer than two weighted columns or rows).
template <typename R>
__device__ __forceinline__ bool mls_inverse(R a0, R a1, R a2, R b0, R b1, R b2, R inv[9])
{
    const R A0 = a0 * b0, A1 = a1 * b0, A2 = a0 * b1, A4 = a2 * b0, A5 = a1 * b1, A8 = a0 * b2;
    const R c00 = A4 * A8 - A5 * A5, c01 = A5 * A2 - A1 * A8, c02 = A1 * A5 - A4 * A2;
    const R det = A0 * c00 + A1 * c01 + A2 * c02;
    if (!(fabs(det) > R(1e-6) * A0 * A0 * A0)) return false;
    const R id = R(1) / det;
    inv[0] = c00 * id;
    inv[1] = inv[3] = c01 * id;
    inv[2] = inv[6] = c02 * id;
    inv[4] = (A0 * A8 - A2 * A2) * id;
    inv[5] = inv[7] = (A2 * A1 - A0 * A5) * id;
    inv[8] = (A0 * A4 - A1 * A1) * id;
    return true;
}

// d phi / d r
template <typename R>
__device__ __forceinline__ R peskin_d(R r)
{
    R a = fabs(r);
    R g;
    if (a <= R(1)) {
        R t = a - R(0.5);
        g = (R(-2) - R(4) * t / sqrt(R(2) - R(4) * t * t)) * R(0.125);
    } else if (a <= R(2)) {
        R t = a - R(1.5);
        g = (R(-2) + R(4) * t / sqrt(R(2) - R(4) * t * t)) * R(0.125);
    } else {
        g = R(0);
    }
    return r < R(0) ? -g : g;
}

// phi and d phi / d r together (one square root)
template <typename R>
__device__ __forceinline__ void peskin_both(R r, R& ph, R& dph)
{
    R a = fabs(r), g;
    if (a <= R(1)) {
        R t = a - R(0.5);
        R s = sqrt(R(2) - R(4) * t * t);
        ph = (R(3) - R(2) * a + s) * R(0.125);
        g = (R(-2) - R(4) * t / s) * R(0.125);
    } else if (a <= R(2)) {
        R t = a - R(1.5);
        R s = sqrt(R(2) - R(4) * t * t);
        ph = (R(5) - R(2) * a - s) * R(0.125);
        g = (R(-2) + R(4) * t / s) * R(0.125);
    } else {
        ph = R(0);
        g = R(0);
    }
    dph = r < R(0) ? -g : g;
}

// ------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror & Shaw (SC'11): counter-based generator, 10 rounds.
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t a = 0xD2511F53u * c.x, ah = __umulhi(0xD2511F53u, c.x);
        uint32_t b = 0xCD9E8D57u * c.z, bh = __umulhi(0xCD9E8D57u, c.z);
        c = U4{bh ^ c.y ^ k0, b, ah ^ c.w ^ k1, a};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// uniform draw of ligand site `site` at Lagrangian step `n`: 24 high bits of the
// first output word of counter (n_lo, n_hi, site, 0) under key (seed_lo, seed_hi)
__device__ __forceinline__ float bond_draw(uint64_t seed, int64_t n, uint32_t site)
{
    U4 c{(uint32_t)(uint64_t)n, (uint32_t)((uint64_t)n >> 32), site, 0u};
    U4 o = philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return (float)(o.x >> 8) * (1.0f / 16777216.0f);
}

// ------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block (deterministic tree); every thread gets the result.
// scratch: >= 32 elements of T in shared memory.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    T t = (lane < nw) ? scratch[lane] : T(0);
    t = warp_sum(t);
    return t;
}

template <typename T>
__device__ __forceinline__ T warp_min(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename T>
__device__ __forceinline__ T block_min(T v, T* scratch)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_min(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    T t = (lane < nw) ? scratch[lane] : scratch[0];
    return warp_min(t);
}
template <typename T>
__device__ __forceinline__ T block_max(T v, T* scratch)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    T t = (lane < nw) ? scratch[lane] : scratch[0];
    return warp_max(t);
}

__device__ __forceinline__ int tile_of(const Lattice& L, int i, int j)
{
    return (j / TY) * L.ntx + (i / TX);
}

}  // namespace lbib
