// lbib_lbm.cu -- lattice kernels: fused pull streaming + boundary conditions +
// moments + Guo-forced BGK collision over SoA deviation populations.
//
// One thread updates one node; a 32 x 4 block updates one tile.  The bulk
// kernel covers every tile that no membrane can reach this step and has no
// immersed-boundary force to add; the near kernel walks the compact list of
// the other tiles, gathers the spread direct-forcing force of the markers
// whose stencil touches the tile (bit mask, ascending marker order), applies
// the same node update with that force and writes rho - 1 and u for the
// Lagrangian kernel.
//
// Per node and step: Eq. 1 (streaming as a pull from x - e_i, collision),
// Eq. 2 (equilibrium), Eq. 4 (forcing), Eqs. 5-6 (moments with half force),
// halfway bounce-back on the walls y = 0, ny and Zou-He on the inlet x = 0
// (plane-Poiseuille velocity, Sec. 3.1) and outlet x = nx - 1 (density),
// x counted within the node's instance (a context may hold a batch of
// capillaries side by side; each tile column carries its instance's origin
// and width).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <type_traits>

#include "lbib_device.cuh"

namespace lbib {

__device__ __forceinline__ constexpr int cx(int q) { return (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0); }
__device__ __forceinline__ constexpr int cy(int q) { return (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0); }
__device__ __forceinline__ constexpr int op(int q) { return q == 0 ? 0 : (q <= 4 ? ((q + 1) % 4) + 1 : ((q - 3) % 4) + 5); }

template <typename R>
__device__ __forceinline__ R inlet_profile(const Lattice& L, int y)
{
    R yy = R(y) + R(0.5), H = R(L.ny);
    return R(4) * lat_param<R>(L.umax, L.umax_f) * yy * (H - yy) / (H * H);
}

// Zou-He on deviations g_i = f_i - w_i (the rest weights cancel pairwise).
template <typename R>
__device__ __forceinline__ void zou_he_inlet(R g[9], R u)
{
    R s = g[0] + g[2] + g[4] + R(2) * (g[3] + g[6] + g[7]);
    R rho = (R(1) + s) / (R(1) - u);
    R ru = rho * u;
    R h = R(0.5) * (g[2] - g[4]);
    g[1] = g[3] + R(2) / R(3) * ru;
    g[5] = g[7] - h + ru / R(6);
    g[8] = g[6] + h + ru / R(6);
}

template <typename R>
__device__ __forceinline__ void zou_he_outlet(R g[9], R rho_out)
{
    R s = g[0] + g[2] + g[4] + R(2) * (g[1] + g[5] + g[8]);
    R u = (s + (R(1) - rho_out)) / rho_out;
    R ru = rho_out * u;
    R h = R(0.5) * (g[2] - g[4]);
    g[3] = g[1] - R(2) / R(3) * ru;
    g[7] = g[5] + h - ru / R(6);
    g[6] = g[8] - h - ru / R(6);
}

// Pull the nine post-collision deviations that stream into node (x, y); xl is
// x within its instance of width nxi (global column x - xl is the origin).
template <typename S, typename R>
__device__ __forceinline__ void pull(const Lattice& L, const S* __restrict__ fin, int x, int y, int xl, int nxi,
                                     R g[9])
{
    const int qs = L.qstride, nxp = L.nxp;
    if (xl > 0 && xl < nxi - 1 && y > 0 && y < L.ny - 1) {
#pragma unroll
        for (int q = 0; q < 9; ++q)
            g[q] = ld<S, R>(fin + LBIB_IDX(q * qs + (y - cy(q)) * nxp + (x - cx(q)), 9LL * qs, L.chk_status));
        return;
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        int xs = xl - cx(q), ys = y - cy(q);
        if (ys < 0 || ys >= L.ny) {
            g[q] = ld<S, R>(fin + LBIB_IDX(op(q) * qs + y * nxp + x, 9LL * qs, L.chk_status));  // halfway bounce-back
        } else if (xs < 0 || xs >= nxi) {
            if (L.bc == LBIB_BC_PERIODIC_FORCE) {
                xs = xs < 0 ? xs + nxi : xs - nxi;
                g[q] = ld<S, R>(fin + LBIB_IDX(q * qs + ys * nxp + (x - xl) + xs, 9LL * qs, L.chk_status));
            } else {
                g[q] = R(0);  // unknown, set by Zou-He
            }
        } else {
            g[q] = ld<S, R>(fin + LBIB_IDX(q * qs + ys * nxp + (x - cx(q)), 9LL * qs, L.chk_status));
        }
    }
    if (L.bc == LBIB_BC_INLET_OUTLET) {
        if (xl == 0) zou_he_inlet<R>(g, inlet_profile<R>(L, y));
        else if (xl == nxi - 1) zou_he_outlet<R>(g, lat_param<R>(L.rho_out, L.rho_out_f));
    }
}

// Moments with the half-force shift and the Guo-forced BGK collision.
// Opposite directions q, o (e_o = -e_q) share the even part of the
// equilibrium, A = w (drho + rho (9/2 (e.u)^2 - 3/2 u.u)), and differ in the
// sign of the odd part, B = 3 w rho e_q.u (Eq. 2); likewise the forcing term
// of Eq. 4.  The relaxation is g' = (1 - omega) g + omega f_eq with omega
// folded into the equilibrium terms.  FORCED = false is the same update for
// F = 0 (it gives the same values as FORCED = true with F = 0, without the
// source arithmetic).
//
// Every operation is explicitly rounded (fused multiply-adds where written,
// nothing else fused or reordered): the lattice kernels inline these pieces
// in different orders (a node at a time, or the moments of several nodes
// first and then one population pair of all of them), and left to the
// compiler's contraction the same expressions were fused differently in
// different kernels.  Written out, every kernel gives every node the same
// bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// 1 / rho.  FP32: the hardware's approximate reciprocal refined by one
// Newton-Raphson step, x' = x + x (1 - rho x), which leaves it within an ulp
// of the quotient for the densities a stable run has (rho is 1 to within a few
// per cent; the step needs rho away from zero, infinity and subnormals, where
// the divergence check has already stopped the run), without the division's
// special-case branch.  FP64: the correctly rounded quotient.
__device__ __forceinline__ float recip(float rho)
{
    float x;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x) : "f"(rho));
    return fma_rn(x, fma_rn(-rho, x, 1.0f), x);
}
__device__ __forceinline__ double recip(double rho) { return 1.0 / rho; }

// relaxation constants of one omega (the same in every thread)
template <typename R>
struct Relax {
    R omega, keep, cf;
    __device__ __forceinline__ explicit Relax(R om)
        : omega(om), keep(sub_rn(R(1), om)), cf(fma_rn(R(-0.5), om, R(1)))
    {
    }
    __device__ __forceinline__ R ow(int q) const { return mul_rn(omega, wq<R>(q)); }
    __device__ __forceinline__ R ow3(int q) const { return mul_rn(R(3), mul_rn(omega, wq<R>(q))); }
    __device__ __forceinline__ R cfw(int q) const { return mul_rn(cf, wq<R>(q)); }
};

template <typename R>
struct Mom {
    R drho, rho, ux, uy, u2, uF;
};

// Eqs. 5-6: rho - 1, rho and u with the half-force shift
template <typename R, bool FORCED>
__device__ __forceinline__ Mom<R> moments(const R g[9], R Fx, R Fy)
{
    Mom<R> m;
    // the x-moving populations' sums serve both the density and jx
    const R east = add_rn(add_rn(g[1], g[5]), g[8]), west = add_rn(add_rn(g[3], g[6]), g[7]);
    m.drho = add_rn(add_rn(add_rn(g[0], g[2]), g[4]), add_rn(east, west));
    m.rho = add_rn(R(1), m.drho);
    R jx = sub_rn(east, west);
    R jy = sub_rn(add_rn(add_rn(g[2], g[5]), g[6]), add_rn(add_rn(g[4], g[7]), g[8]));
    if (FORCED) {
        jx = fma_rn(R(0.5), Fx, jx);
        jy = fma_rn(R(0.5), Fy, jy);
    }
    const R inv = recip(m.rho);
    m.ux = mul_rn(jx, inv);
    m.uy = mul_rn(jy, inv);
    m.u2 = mul_rn(R(1.5), fma_rn(m.ux, m.ux, mul_rn(m.uy, m.uy)));
    m.uF = FORCED ? fma_rn(m.ux, Fx, mul_rn(m.uy, Fy)) : R(0);
    return m;
}

// rest population after collision
template <typename R, bool FORCED>
__device__ __forceinline__ R relax_rest(const Relax<R>& X, R g0, const Mom<R>& m)
{
    R r = fma_rn(X.keep, g0, mul_rn(X.ow(0), fma_rn(-m.rho, m.u2, m.drho)));
    if (FORCED) r = add_rn(r, mul_rn(X.cfw(0), mul_rn(R(-3), m.uF)));
    return r;
}

// pair k = 0..3: q = 1, 2, 5, 6 and its opposite o = 3, 4, 7, 8
__device__ __forceinline__ constexpr int pair_q(int k) { return (k < 2) ? 1 + k : 3 + k; }

template <typename R, bool FORCED>
__device__ __forceinline__ void relax_pair(const Relax<R>& X, int k, R& gq, R& go, const Mom<R>& m, R Fx, R Fy)
{
    const int q = pair_q(k);
    // e_q . u and e_q . F for e_1 = (1, 0), e_2 = (0, 1), e_5 = (1, 1), e_6 = (-1, 1)
    const R eu = q == 1 ? m.ux : (q == 2 ? m.uy : (q == 5 ? add_rn(m.ux, m.uy) : sub_rn(m.uy, m.ux)));
    const R t = fma_rn(mul_rn(R(4.5), eu), eu, -m.u2);
    const R oA = mul_rn(X.ow(q), fma_rn(m.rho, t, m.drho));
    const R oB = mul_rn(mul_rn(X.ow3(q), m.rho), eu);
    R a = fma_rn(X.keep, gq, add_rn(oA, oB));
    R b = fma_rn(X.keep, go, sub_rn(oA, oB));
    if (FORCED) {
        const R eF = q == 1 ? Fx : (q == 2 ? Fy : (q == 5 ? add_rn(Fx, Fy) : sub_rn(Fy, Fx)));
        const R even = mul_rn(X.cfw(q), fma_rn(mul_rn(R(9), eu), eF, mul_rn(R(-3), m.uF)));
        const R odd = mul_rn(X.cfw(q), mul_rn(R(3), eF));
        a = add_rn(a, add_rn(even, odd));
        b = add_rn(b, sub_rn(even, odd));
    }
    gq = a;
    go = b;
}

template <typename R, bool FORCED>
__device__ __forceinline__ void collide_t(R g[9], R Fx, R Fy, R omega, R& drho, R& ux, R& uy)
{
    const Relax<R> X(omega);
    const Mom<R> m = moments<R, FORCED>(g, Fx, Fy);
    drho = m.drho;
    ux = m.ux;
    uy = m.uy;
    g[0] = relax_rest<R, FORCED>(X, g[0], m);
#pragma unroll
    for (int k = 0; k < 4; ++k) relax_pair<R, FORCED>(X, k, g[pair_q(k)], g[op(pair_q(k))], m, Fx, Fy);
}

template <typename R>
__device__ __forceinline__ void collide(R g[9], R Fx, R Fy, R omega, R& drho, R& ux, R& uy)
{
    collide_t<R, true>(g, Fx, Fy, omega, drho, ux, uy);
}

// One block covers RT tiles stacked in y (a TX x RT TY node box) with
// TX x (RT TY / NPT) threads; a thread updates NPT nodes of one column, NPT
// rows apart, issuing all their loads before the first collision (more bytes
// in flight per thread when fewer threads are resident).  The block reads its
// tiles' near flags once (a tile the near kernel owns is skipped) and decides
// once whether its box touches a wall or an instance's first or last column:
// an interior box pulls every node with one base offset plus the nine
// per-plane offsets, which are the same for every thread, and needs no
// per-node boundary test; a boundary box takes the general pull.
// at most 40 registers a thread (48 resident warps): the lean address arithmetic let the
// compiler take 48 at two nodes a thread, which cost a fifth of the resident
// warps and, inside the step graph, more time than the instructions saved
template <typename S, typename R, int RT, int NPT, bool FORCED>
__global__ void __launch_bounds__(TX* TY* RT / NPT, 1536 / (TX * TY * RT / NPT)) k_bulk(Dev d, int p, int slot)
{
    const Lattice& L = d.L;
    constexpr int ROWS = TY * RT, STEP = ROWS / NPT;
    const int4 ci = d.colinfo[blockIdx.x];
    uint32_t own = 0u;  // bit r: the bulk update owns tile row blockIdx.y RT + r
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const int t = blockIdx.y * RT + r;
        if (t < L.nty && !d.nearflag[slot][t * L.ntx + blockIdx.x]) own |= 1u << r;
    }
    if (!own) return;  // the whole block
    const int x = blockIdx.x * TX + threadIdx.x;
    const int xl = x - ci.x;
    const int yb = blockIdx.y * ROWS;
    const int xt = blockIdx.x * TX - ci.x;  // the tile column's first column within its instance
    const bool interior = yb > 0 && yb + ROWS < L.ny && xt > 0 && xt + TX < ci.y;
    const S* __restrict__ fin = static_cast<const S*>(d.f[p]);
    S* __restrict__ fout = static_cast<S*>(d.f[p ^ 1]);
    R g[NPT][9];
    bool act[NPT];
    if (interior) {
        const int base = (yb + threadIdx.y) * L.nxp + x;
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            act[j] = (own >> ((threadIdx.y + j * STEP) / TY)) & 1u;
            if (act[j])
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    g[j][q] = ld<S, R>(fin + LBIB_IDX(base + j * STEP * L.nxp + (q * L.qstride - cy(q) * L.nxp - cx(q)),
                                                      9LL * L.qstride, L.chk_status));
        }
    } else {
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const int y = yb + threadIdx.y + j * STEP;
            act[j] = y < L.ny && xl < ci.y && ((own >> ((threadIdx.y + j * STEP) / TY)) & 1u);
            if (act[j]) pull<S, R>(L, fin, x, y, xl, ci.y, g[j]);
        }
    }
    bool bad = false;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        if (!act[j]) continue;
        R drho, ux, uy;
        collide_t<R, FORCED>(g[j], lat_param<R>(L.gx, L.gx_f), lat_param<R>(L.gy, L.gy_f),
                             lat_param<R>(L.omega, L.omega_f), drho, ux, uy);
        if (!(drho > R(-1) && fabs(ux + uy) < R(INFINITY))) bad = true;
        const int base = (yb + threadIdx.y + j * STEP) * L.nxp + x;
#pragma unroll
        for (int q = 0; q < 9; ++q)
            st<S, R>(fout + LBIB_IDX(q * L.qstride + base, 9LL * L.qstride, L.chk_status), g[j][q]);
    }
    if (bad) atomicOr(d.status, ST_DIVERGED);
}

// Vectorised bulk update.  A thread updates BV consecutive nodes of a row
// (BV = 16 bytes of FP32 or FP64 storage, 8 bytes of 16-bit storage) and
// walks the four rows of its tile row; a warp spans 32 BV node columns and
// each warp of a block takes one tile row.  The pull reads every population
// plane as one aligned vector per thread at the row the plane streams from
// (y - e_y, or the node's own row for a population bounced at a wall), so
// no node needs its own load or address.  The plus-or-minus-one x shift of
// the pull becomes a warp shuffle of the vector's end element: a lane takes
// its left (right) neighbour's last (first) element, and a lane whose
// neighbour did not load, or that sits at the warp's end, loads that one
// value itself.  Zou-He then overrides the unknowns of inlet and outlet
// nodes.  In the periodic mode the lanes holding an instance's first or last
// column load the populations that wrap around to the other end.  The node update is k_bulk's
// (same pulled values, same collide_t), so every node gets the same bits.
template <typename S, typename R, int V>
struct VecIO;
template <>
struct VecIO<float, float, 4> {
    static __device__ __forceinline__ void ld_shared(const float* p, float o[4])
    {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
    static __device__ __forceinline__ void ld(const float* p, float o[4])
    {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
    static __device__ __forceinline__ void st(float* p, const float o[4])
    {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <>
struct VecIO<double, double, 2> {
    static __device__ __forceinline__ void ld_shared(const double* p, double o[2])
    {
        const double2 v = *reinterpret_cast<const double2*>(p);
        o[0] = v.x;
        o[1] = v.y;
    }
    static __device__ __forceinline__ void ld(const double* p, double o[2])
    {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = v.x;
        o[1] = v.y;
    }
    static __device__ __forceinline__ void st(double* p, const double o[2])
    {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    }
};
// bfloat16: element k of a 32-bit word pair sits in bits 16 (k & 1) .. of word
// k / 2; widening is a shift, narrowing rounds to nearest even (as st<>)
template <>
struct VecIO<__nv_bfloat16, float, 4> {
    static __device__ __forceinline__ void ld_shared(const __nv_bfloat16* p, float o[4])
    {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        o[0] = __uint_as_float(v.x << 16);
        o[1] = __uint_as_float(v.x & 0xffff0000u);
        o[2] = __uint_as_float(v.y << 16);
        o[3] = __uint_as_float(v.y & 0xffff0000u);
    }
    static __device__ __forceinline__ void ld(const __nv_bfloat16* p, float o[4])
    {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
        o[0] = __uint_as_float(v.x << 16);
        o[1] = __uint_as_float(v.x & 0xffff0000u);
        o[2] = __uint_as_float(v.y << 16);
        o[3] = __uint_as_float(v.y & 0xffff0000u);
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, const float o[4])
    {
        const __nv_bfloat162 a = __floats2bfloat162_rn(o[0], o[1]), b = __floats2bfloat162_rn(o[2], o[3]);
        uint2 v;
        v.x = *reinterpret_cast<const uint32_t*>(&a);
        v.y = *reinterpret_cast<const uint32_t*>(&b);
        *reinterpret_cast<uint2*>(p) = v;
    }
};
// binary16 scaled by HALF_SCALE, as ld<> / st<>
template <>
struct VecIO<__half, float, 4> {
    static __device__ __forceinline__ void ld_shared(const __half* p, float o[4])
    {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
        o[0] = a.x * (1.0f / HALF_SCALE);
        o[1] = a.y * (1.0f / HALF_SCALE);
        o[2] = b.x * (1.0f / HALF_SCALE);
        o[3] = b.y * (1.0f / HALF_SCALE);
    }
    static __device__ __forceinline__ void ld(const __half* p, float o[4])
    {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
        o[0] = a.x * (1.0f / HALF_SCALE);
        o[1] = a.y * (1.0f / HALF_SCALE);
        o[2] = b.x * (1.0f / HALF_SCALE);
        o[3] = b.y * (1.0f / HALF_SCALE);
    }
    static __device__ __forceinline__ void st(__half* p, const float o[4])
    {
        const __half2 a = __floats2half2_rn(o[0] * HALF_SCALE, o[1] * HALF_SCALE);
        const __half2 b = __floats2half2_rn(o[2] * HALF_SCALE, o[3] * HALF_SCALE);
        uint2 v;
        v.x = *reinterpret_cast<const uint32_t*>(&a);
        v.y = *reinterpret_cast<const uint32_t*>(&b);
        *reinterpret_cast<uint2*>(p) = v;
    }
};

#ifndef LBIB_VEC_NODES
#define LBIB_VEC_NODES 4
#endif
#ifndef LBIB_VEC_MIN_BLOCKS
#define LBIB_VEC_MIN_BLOCKS 3
#endif
constexpr int VEC_MIN_BLOCKS = LBIB_VEC_MIN_BLOCKS;
template <>
struct VecIO<float, float, 2> {
    static __device__ __forceinline__ void ld(const float* p, float o[2])
    {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        o[0] = v.x;
        o[1] = v.y;
    }
    static __device__ __forceinline__ void st(float* p, const float o[2])
    {
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    }
};
template <>
struct VecIO<__nv_bfloat16, float, 2> {
    static __device__ __forceinline__ void ld(const __nv_bfloat16* p, float o[2])
    {
        const uint32_t v = __ldg(reinterpret_cast<const unsigned int*>(p));
        o[0] = __uint_as_float(v << 16);
        o[1] = __uint_as_float(v & 0xffff0000u);
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, const float o[2])
    {
        const __nv_bfloat162 a = __floats2bfloat162_rn(o[0], o[1]);
        *reinterpret_cast<uint32_t*>(p) = *reinterpret_cast<const uint32_t*>(&a);
    }
};
template <>
struct VecIO<__half, float, 2> {
    static __device__ __forceinline__ void ld(const __half* p, float o[2])
    {
        const uint32_t v = __ldg(reinterpret_cast<const unsigned int*>(p));
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v));
        o[0] = a.x * (1.0f / HALF_SCALE);
        o[1] = a.y * (1.0f / HALF_SCALE);
    }
    static __device__ __forceinline__ void st(__half* p, const float o[2])
    {
        const __half2 a = __floats2half2_rn(o[0] * HALF_SCALE, o[1] * HALF_SCALE);
        *reinterpret_cast<uint32_t*>(p) = *reinterpret_cast<const uint32_t*>(&a);
    }
};

template <typename S>
__host__ __device__ constexpr int vec_width() { return sizeof(S) == 8 ? 2 : LBIB_VEC_NODES; }

// One row of a vectorised bulk thread.  WALL: 0 interior row, 1 the row at
// y = 0, 2 the row at y = ny - 1 (populations arriving through that wall are
// bounced from the node's own opposite population: no shift at all).  The
// moments of the V nodes come first; then each population pair is relaxed
// for all V nodes and stored as two vectors, so that no node's whole output
// waits in registers for the others.
template <typename S, typename R, int V, int WALL, bool FORCED>
__device__ __forceinline__ bool vec_row(const Lattice& L, const S* __restrict__ fin, S* __restrict__ fout, int x0,
                                        int xs, int xl0, int nxi, int y, bool act, bool need_l, bool need_r,
                                        bool bnd)
{
    R v[9][V];
    constexpr bool bb[9] = {false,
                            false,
                            WALL == 1,
                            false,
                            WALL == 2,
                            WALL == 1,
                            WALL == 1,
                            WALL == 2,
                            WALL == 2};
    const int row = y * L.nxp + x0;
    // every lane loads (a lane that updates nothing reads the first updating
    // lane's vectors: the requests merge, and the values go unused); loads
    // under a lane predicate cost the kernel 40 more registers
    const int rs = y * L.nxp + xs;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int src = bb[q] ? op(q) * L.qstride + rs : q * L.qstride + rs - cy(q) * L.nxp;
        VecIO<S, R, V>::ld(fin + LBIB_IDX(src, 9LL * L.qstride - (V - 1), L.chk_status), v[q]);
    }
    // the value each shifted plane brings in at the lane's left or right end
    R in[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        if (bb[q] || cx(q) == 0) continue;
        const int src = q * L.qstride + row - cy(q) * L.nxp;
        if (cx(q) == 1) {
            in[q] = __shfl_up_sync(0xffffffffu, v[q][V - 1], 1);
            if (need_l) in[q] = xl0 > 0 ? ld<S, R>(fin + LBIB_IDX(src - 1, 9LL * L.qstride, L.chk_status)) : R(0);
        } else {
            in[q] = __shfl_down_sync(0xffffffffu, v[q][0], 1);
            if (need_r)
                in[q] = xl0 + V < nxi ? ld<S, R>(fin + LBIB_IDX(src + V, 9LL * L.qstride, L.chk_status)) : R(0);
        }
    }
    if (!act) return false;
    R g[V][9];
#pragma unroll
    for (int i = 0; i < V; ++i) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            if (bb[q] || cx(q) == 0) g[i][q] = v[q][i];
            else if (cx(q) == 1) g[i][q] = i > 0 ? v[q][i - 1] : in[q];
            else g[i][q] = i < V - 1 ? v[q][i + 1] : in[q];
        }
    }
    if (bnd) {
        // lanes holding an instance's first or last column: the populations
        // entering through the inlet or outlet are Zou-He's unknowns, or, in
        // the periodic mode, come from the instance's other end
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const int xl = xl0 + i;
            if (L.bc == LBIB_BC_PERIODIC_FORCE) {
                if (xl == 0) {
#pragma unroll
                    for (int q = 0; q < 9; ++q)
                        if (!bb[q] && cx(q) == 1)
                            g[i][q] = ld<S, R>(fin + LBIB_IDX(q * L.qstride + row - cy(q) * L.nxp + i + nxi - 1,
                                                              9LL * L.qstride, L.chk_status));
                }
                if (xl == nxi - 1) {
#pragma unroll
                    for (int q = 0; q < 9; ++q)
                        if (!bb[q] && cx(q) == -1)
                            g[i][q] = ld<S, R>(fin + LBIB_IDX(q * L.qstride + row - cy(q) * L.nxp + i - (nxi - 1),
                                                              9LL * L.qstride, L.chk_status));
                }
            } else if (xl == 0) {
                zou_he_inlet<R>(g[i], inlet_profile<R>(L, y));
            } else if (xl == nxi - 1) {
                zou_he_outlet<R>(g[i], lat_param<R>(L.rho_out, L.rho_out_f));
            }
        }
    }
    const R Fx = lat_param<R>(L.gx, L.gx_f), Fy = lat_param<R>(L.gy, L.gy_f);
    const Relax<R> X(lat_param<R>(L.omega, L.omega_f));
    Mom<R> m[V];
    bool bad = false;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        m[i] = moments<R, FORCED>(g[i], Fx, Fy);
        if (xl0 + i < nxi && !(m[i].drho > R(-1) && fabs(m[i].ux + m[i].uy) < R(INFINITY))) bad = true;
    }
    const bool full = xl0 + V <= nxi;
    auto store = [&](int q, const R o[V]) {
        if (full) {
            VecIO<S, R, V>::st(fout + LBIB_IDX(q * L.qstride + row, 9LL * L.qstride - (V - 1), L.chk_status), o);
        } else {
            // the instance ends inside the vector: only its own columns are written
#pragma unroll
            for (int i = 0; i < V; ++i)
                if (xl0 + i < nxi)
                    st<S, R>(fout + LBIB_IDX(q * L.qstride + row + i, 9LL * L.qstride, L.chk_status), o[i]);
        }
    };
    {
        R o[V];
#pragma unroll
        for (int i = 0; i < V; ++i) o[i] = relax_rest<R, FORCED>(X, g[i][0], m[i]);
        store(0, o);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int q = pair_q(k), o = op(q);
        R a[V], b[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            a[i] = g[i][q];
            b[i] = g[i][o];
            relax_pair<R, FORCED>(X, k, a[i], b[i], m[i], Fx, Fy);
        }
        store(q, a);
        store(o, b);
    }
    return bad;
}

template <typename S, typename R, int V, bool FORCED>
__global__ void __launch_bounds__(256, VEC_MIN_BLOCKS) k_bulk_vec(Dev d, int p, int slot)
{
    const Lattice& L = d.L;
    const int lane = threadIdx.x;
    const int x0 = (blockIdx.x * 32 + lane) * V;
    const int ty = blockIdx.y * blockDim.y + threadIdx.y;  // the warp's tile row
    if (ty >= L.nty) return;                                // whole warps
    const int tx = x0 / TX;
    bool act = false;
    int xl0 = 0, nxi = 0;
    if (x0 < L.nxp) {
        const int4 ci = d.colinfo[tx];
        xl0 = x0 - ci.x;
        nxi = ci.y;
        act = xl0 < nxi && !d.nearflag[slot][ty * L.ntx + tx];
    }
    const uint32_t am = __ballot_sync(0xffffffffu, act);
    if (am == 0u) return;
    const bool need_l = act && (lane == 0 || !((am >> (lane - 1)) & 1u));
    const bool need_r = act && (lane == 31 || !((am >> (lane + 1)) & 1u));
    const bool bnd = act && (xl0 == 0 || xl0 + V >= nxi);
    const int xs = act ? x0 : (blockIdx.x * 32 + __ffs(am) - 1) * V;  // where this lane's vectors come from
    const S* __restrict__ fin = static_cast<const S*>(d.f[p]);
    S* __restrict__ fout = static_cast<S*>(d.f[p ^ 1]);
    bool bad = false;
    // interior rows first, then the wall rows (each in a code region of its
    // own: one loop over the three row kinds needed twice the registers)
    const int y0 = ty * TY, y1 = min(y0 + TY, L.ny);
#pragma unroll 1
    for (int y = max(y0, 1); y < min(y1, L.ny - 1); ++y)
        bad |= vec_row<S, R, V, 0, FORCED>(L, fin, fout, x0, xs, xl0, nxi, y, act, need_l, need_r, bnd);
    if (y0 == 0) bad |= vec_row<S, R, V, 1, FORCED>(L, fin, fout, x0, xs, xl0, nxi, 0, act, need_l, need_r, bnd);
    if (y1 == L.ny)
        bad |= vec_row<S, R, V, 2, FORCED>(L, fin, fout, x0, xs, xl0, nxi, L.ny - 1, act, need_l, need_r, bnd);
    if (bad) atomicOr(d.status, ST_DIVERGED);
}

// TMA-staged bulk update.  A job is a 32 x 8 node box (two tiles of one tile
// column); one 3-D tensor copy brings its nine population planes with a halo
// of one row above and below and 16 bytes of columns on either side (the
// copy's x must sit on a 16-byte boundary; rows outside the lattice arrive as
// zeros) into one of TB_STAGES shared-memory stages, signalled on an mbarrier.
// A block of 32 x 8 threads takes TB_JOBS consecutive jobs (neighbouring tile
// columns): one warp first lists those with a tile the bulk update owns, with
// their near flags and column records, in shared memory (so issuing a copy
// needs no global read), and the copies run TB_STAGES jobs ahead of the
// update.  Interior nodes read their nine pulls from the stage at
// fixed offsets; wall, inlet and outlet nodes take the global path (pull).
// Jobs whose two tiles are both near-membrane are skipped without a copy.
// The node update is k_bulk's (same pull values, same collide_t), so every
// node gets the same bits either way.  A launch option: on the 64-capillary
// sweep it is slower than k_bulk (FP32 126 vs 106 us alone): the halo sectors
// of the copies raise the DRAM reads from 367 to 445 MB per launch, and the
// instructions per node do not fall (about 235 either way: the collision and
// the stores, not the load addressing, make up most of them).
constexpr int TB_ROWS = 8;
constexpr int TB_STAGES = 3;
constexpr int TB_JOBS = 8;  // at most 32 (one warp lists them)
constexpr uint32_t TB_WAIT_LIMIT = 1u << 24;  // mbarrier polls before a block gives up
template <typename S>
__host__ __device__ constexpr int tb_hx() { return 16 / (int)sizeof(S); }
template <typename S>
__host__ __device__ constexpr int tb_w() { return TX + 2 * tb_hx<S>(); }
template <typename S>
__host__ __device__ constexpr uint32_t tb_copy_bytes() { return 9u * (TB_ROWS + 2) * tb_w<S>() * (uint32_t)sizeof(S); }
template <typename S>
__host__ __device__ constexpr uint32_t tb_stage_bytes() { return (tb_copy_bytes<S>() + 127u) & ~127u; }

__device__ __forceinline__ uint32_t tb_smem(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ bool tb_wait(uint64_t* bar, uint32_t parity)
{
    for (uint32_t it = 0; it < TB_WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(tb_smem(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// job = row pair * ntx + tile column: the jobs of a block are neighbouring
// tile columns, so their halo columns are each other's (ordering the jobs down
// a column instead raised the DRAM reads from 445 to 486 MB per launch)
__device__ __forceinline__ void tb_issue(const CUtensorMap* tm, uint64_t* bar, void* dst, int job, int ntx, int hx,
                                         uint32_t bytes)
{
    const int x = (job % ntx) * TX - hx, y = (job / ntx) * TB_ROWS - 1, z = 0;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tb_smem(bar)), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(tb_smem(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(tb_smem(bar))
        : "memory");
}

template <typename S, typename R, bool FORCED>
__global__ void __launch_bounds__(TX* TB_ROWS) k_bulk_tma(const __grid_constant__ CUtensorMap tm, Dev d, int p, int slot)
{
    extern __shared__ __align__(128) unsigned char tb_raw[];
    __shared__ __align__(8) uint64_t full[TB_STAGES];
    __shared__ int s_list[TB_JOBS];         // the block's jobs with a tile the bulk update owns
    __shared__ uint32_t s_near[TB_JOBS][2]; // near flags of each listed job's two tiles
    __shared__ int4 s_ci[TB_JOBS];          // column record of each listed job
    __shared__ int s_n, s_abort;
    const Lattice& L = d.L;
    constexpr int HX = tb_hx<S>(), W = tb_w<S>(), H = TB_ROWS + 2;
    constexpr uint32_t SB = tb_stage_bytes<S>(), CB = tb_copy_bytes<S>();
    const int tid = threadIdx.y * TX + threadIdx.x;
    // stages on a 128-byte boundary of the shared window (tensor-copy destinations)
    unsigned char* tb_stage = tb_raw + ((128u - (tb_smem(tb_raw) & 127u)) & 127u);
    const int jy = (L.nty + 1) / 2;
    const int njobs = L.ntx * jy;
    const int first = blockIdx.x * TB_JOBS;
    const S* __restrict__ fin = static_cast<const S*>(d.f[p]);
    S* __restrict__ fout = static_cast<S*>(d.f[p ^ 1]);
    // the block's jobs, their near flags and column records, read once (one warp)
    if (threadIdx.y == 0) {
        const int j = first + threadIdx.x;
        uint32_t n0 = 1u, n1 = 1u;
        int4 ci = make_int4(0, 0, 0, 0);
        if (threadIdx.x < TB_JOBS && j < njobs) {
            const int tx = j % L.ntx, t0 = (j / L.ntx) * 2;
            n0 = d.nearflag[slot][t0 * L.ntx + tx];
            n1 = (t0 + 1 < L.nty) ? d.nearflag[slot][(t0 + 1) * L.ntx + tx] : 1u;
            ci = d.colinfo[tx];
        }
        const bool live = threadIdx.x < TB_JOBS && j < njobs && (!n0 || !n1);
        const uint32_t m = __ballot_sync(0xffffffffu, live);
        if (live) {
            const int k = __popc(m & ((1u << threadIdx.x) - 1u));
            s_list[k] = j;
            s_near[k][0] = n0;
            s_near[k][1] = n1;
            s_ci[k] = ci;
        }
        if (threadIdx.x == 0) {
            s_n = __popc(m);
            s_abort = 0;
            for (int i = 0; i < TB_STAGES; ++i)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tb_smem(&full[i])), "r"(1));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncwarp();
        if (threadIdx.x == 0)
            for (int k = 0; k < TB_STAGES && k < __popc(m); ++k)
                tb_issue(&tm, &full[k], tb_stage + k * SB, s_list[k], L.ntx, HX, CB);
    }
    __syncthreads();
    const int n = s_n;
    // this thread's node within a job, and its place in a stage
    const int cx0 = threadIdx.x + HX, cy0 = threadIdx.y + 1;
    int k = 0;
    for (; k < n; ++k) {
        const int sg = k % TB_STAGES;
        if (!tb_wait(&full[sg], (uint32_t)(k / TB_STAGES) & 1u)) s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        const int job = s_list[k];
        const int tx = job % L.ntx;
        const int x = tx * TX + threadIdx.x, y = (job / L.ntx) * TB_ROWS + threadIdx.y;
        const int4 ci = s_ci[k];
        const int xl = x - ci.x;
        if (y < L.ny && xl < ci.y && !s_near[k][threadIdx.y / TY]) {
            R g[9];
            if (xl > 0 && xl < ci.y - 1 && y > 0 && y < L.ny - 1) {
                const S* sp = reinterpret_cast<const S*>(tb_stage + sg * SB);
#pragma unroll
                for (int q = 0; q < 9; ++q) g[q] = from_store<S, R>(sp[(q * H + cy0 - cy(q)) * W + cx0 - cx(q)]);
            } else {
                pull<S, R>(L, fin, x, y, xl, ci.y, g);
            }
            R drho, ux, uy;
            collide_t<R, FORCED>(g, lat_param<R>(L.gx, L.gx_f), lat_param<R>(L.gy, L.gy_f),
                                 lat_param<R>(L.omega, L.omega_f), drho, ux, uy);
            if (!(drho > R(-1)) || !isfinite(ux + uy)) atomicOr(d.status, ST_DIVERGED);
            const int base = (int)LBIB_IDX(y * L.nxp + x, L.qstride, L.chk_status);
#pragma unroll
            for (int q = 0; q < 9; ++q) st<S, R>(fout + q * L.qstride + base, g[q]);
        }
        __syncthreads();  // every thread is done with stage sg
        if (tid == 0 && k + TB_STAGES < n) tb_issue(&tm, &full[sg], tb_stage + sg * SB, s_list[k + TB_STAGES], L.ntx, HX, CB);
    }
    if (s_abort && tid == 0) {
        atomicOr(d.status, ST_TMA_TIMEOUT);
        // the copies still in flight land before the block's shared memory is released
        for (int k2 = k; k2 < n && k2 < k + TB_STAGES; ++k2)
            (void)tb_wait(&full[k2 % TB_STAGES], (uint32_t)(k2 / TB_STAGES) & 1u);
    }
}

constexpr int NEAR_WARPS = 4;     // warps per near-kernel block; each warp updates one tile at a time
constexpr int NEAR_STAGE = 64;    // markers a warp stages per pass

// Near-membrane update, in two launches.  k_spread: each warp walks its share
// of the near-tile list and forms the force density of a whole 32 x 4 tile,
// lane l owning column l.  The tile's bit mask is read 32 words per round (one
// word per lane); the set bits are ranked across the warp (ascending marker
// order) and staged in passes of NEAR_STAGE markers with their stencil
// weights; each node then adds the forces of the staged markers whose 4 x 4
// stencil holds it, in that order, to the uniform body force, and the sums go
// to fx / fy.  Warp-local throughout: no block barrier.  k_near_lbm then
// updates the tiles' nodes with that force, a thread per node: the latency-
// bound gather and the bandwidth-bound lattice update no longer share one
// warp's registers, and the update runs at the bulk kernel's efficiency.
template <typename R, bool MLS>
__global__ void __launch_bounds__(32 * NEAR_WARPS) k_spread(Dev d, int p)
{
    pdl_wait();  // step counter, list and markers come from the membrane update
    const Lattice& L = d.L;
    const int64_t m = *d.step;  // lattice step (the Lagrangian counter has reached it)
    const int c = (int)(m % 3);
    const int cnt = min(d.count[c], d.list_cap);
    const int nm = d.nmark;  // marker arrays span the whole batch
    const int32_t* __restrict__ mki = d.mki[p];
    const R* __restrict__ mkf = static_cast<const R*>(d.mkf[p]);
    uint32_t* mask = d.mask[p];
    R* fx_o = static_cast<R*>(d.fx);
    R* fy_o = static_cast<R*>(d.fy);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // per warp: stencil origin, the four x and y weights phi(1 - a + frac),
    // a = 0..3, over the marker's columns / rows, and F ds
    __shared__ int s_ix[NEAR_WARPS][NEAR_STAGE], s_iy[NEAR_WARPS][NEAR_STAGE];
    __shared__ R s_wx[NEAR_WARPS][NEAR_STAGE][4], s_wy[NEAR_WARPS][NEAR_STAGE][4];
    // MLS only: node weight = s_wx[a] s_wy[b] + s_ax[a] s_cy[b]
    __shared__ R s_ax[NEAR_WARPS][MLS ? NEAR_STAGE : 1][4], s_cy[NEAR_WARPS][MLS ? NEAR_STAGE : 1][4];
    __shared__ R s_Fx[NEAR_WARPS][NEAR_STAGE], s_Fy[NEAR_WARPS][NEAR_STAGE];
    const R gx = lat_param<R>(L.gx, L.gx_f), gy = lat_param<R>(L.gy, L.gy_f);
    const int k0 = blockIdx.x * NEAR_WARPS + wid, kstep = gridDim.x * NEAR_WARPS;
    for (int k = k0; k < cnt; k += kstep) {
        const int t = d.list[c][k];
        const int tx = t % L.ntx, ty = t / L.ntx;
        const int4 ci = d.colinfo[tx];
        const int x = tx * TX + lane, y0 = ty * TY;
        const int xl = x - ci.x;
        bool live[TY];
#pragma unroll
        for (int r = 0; r < TY; ++r) live[r] = (xl < ci.y && y0 + r < L.ny);
        R Fx[TY], Fy[TY];
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            Fx[r] = gx;
            Fy[r] = gy;
        }
        for (int w0 = 0; w0 < d.mw; w0 += 32) {
            const bool has = w0 + lane < d.mw;
            const uint32_t wd = has ? mask[(size_t)t * d.mw + w0 + lane] : 0u;
            // exclusive prefix of the set-bit counts across the lanes
            const int cw = __popc(wd);
            int incl = cw;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int off = incl - cw;
            const int n = __shfl_sync(0xffffffffu, incl, 31);
            if (has && wd) mask[(size_t)t * d.mw + w0 + lane] = 0u;  // consumed
            for (int base = 0; base < n; base += NEAR_STAGE) {
                // stage the markers of rank [base, base + NEAR_STAGE): lane l takes
                // ranks base + l, base + l + 32, ...; the word holding rank r is the
                // last lane whose exclusive prefix is <= r (binary search by shuffles)
                const int ns = min(NEAR_STAGE, n - base);
                for (int pos = lane; pos < 32 * ((ns + 31) / 32); pos += 32) {
                    const int r = base + pos;
                    int src = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int cand = src + step;
                        const int co = __shfl_sync(0xffffffffu, off, cand & 31);
                        if (cand < 32 && co <= r) src = cand;
                    }
                    const uint32_t sw = __shfl_sync(0xffffffffu, wd, src);
                    const int so = __shfl_sync(0xffffffffu, off, src);
                    if (pos < ns) {
                        const int bit = (int)__fns(sw, 0u, r - so + 1);  // (r - so + 1)-th set bit
                        const int id = ci.z + (w0 + src) * 32 + bit;     // instance-local bit -> batch marker
                        s_ix[wid][pos] = mki[id];
                        s_iy[wid][pos] = mki[nm + id];
                        const R fx = mkf[id], fy = mkf[nm + id];
                        if constexpr (MLS) {
                            // MLS shape function of node (a, b) at the marker:
                            // wx_a wy_b (c0 + c1 dx_a + c2 dy_b), the fit over the
                            // whole stencil (the share of wall nodes stays with
                            // the wall: those nodes are never updated here)
                            R wxv[4], wyv[4], a0 = R(0), a1 = R(0), a2 = R(0), b0 = R(0), b1 = R(0), b2 = R(0);
#pragma unroll
                            for (int a = 0; a < 4; ++a) {
                                const R dx = R(a - 1) - fx, dy = R(a - 1) - fy;
                                wxv[a] = mls_w<R>(dx);
                                wyv[a] = mls_w<R>(dy);
                                a0 += wxv[a];
                                a1 += wxv[a] * dx;
                                a2 += wxv[a] * dx * dx;
                                b0 += wyv[a];
                                b1 += wyv[a] * dy;
                                b2 += wyv[a] * dy * dy;
                            }
                            R inv[9];
                            const bool ok = mls_inverse<R>(a0, a1, a2, b0, b1, b2, inv);
                            const R c0 = ok ? inv[0] : R(0), c1 = ok ? inv[1] : R(0), c2 = ok ? inv[2] : R(0);
#pragma unroll
                            for (int a = 0; a < 4; ++a) {
                                s_wx[wid][pos][a] = wxv[a] * (c0 + c1 * (R(a - 1) - fx));
                                s_ax[wid][pos][a] = wxv[a];
                                s_wy[wid][pos][a] = wyv[a];
                                s_cy[wid][pos][a] = wyv[a] * c2 * (R(a - 1) - fy);
                            }
                        } else {
#pragma unroll
                            for (int a = 0; a < 4; ++a) {
                                // X - (ix - 1 + a) = 1 - a + frac, as the node-side difference below
                                s_wx[wid][pos][a] = peskin<R>(R(1 - a) + fx);
                                s_wy[wid][pos][a] = peskin<R>(R(1 - a) + fy);
                            }
                        }
                        s_Fx[wid][pos] = mkf[2 * nm + id];
                        s_Fy[wid][pos] = mkf[3 * nm + id];
                    }
                }
                __syncwarp();
                if constexpr (MLS) {
                    for (int q = 0; q < ns; ++q) {
                        const int a = x - s_ix[wid][q] + 1;
                        if ((unsigned)a >= 4u) continue;
                        const R wxa = s_wx[wid][q][a], axa = s_ax[wid][q][a], Fq = s_Fx[wid][q], Gq = s_Fy[wid][q];
                        const int b0 = y0 - s_iy[wid][q] + 1;
#pragma unroll
                        for (int r = 0; r < TY; ++r) {
                            const int b = b0 + r;
                            if ((unsigned)b < 4u) {
                                const R wt = wxa * s_wy[wid][q][b] + axa * s_cy[wid][q][b];
                                Fx[r] += wt * Fq;
                                Fy[r] += wt * Gq;
                            }
                        }
                    }
                } else {
                    for (int q = 0; q < ns; ++q) {
                        // node (x, y) in the marker's 4 x 4 stencil [ix - 1, ix + 2] x [iy - 1, iy + 2]
                        const int a = x - s_ix[wid][q] + 1;
                        if ((unsigned)a >= 4u) continue;
                        const R wxa = s_wx[wid][q][a], Fq = s_Fx[wid][q], Gq = s_Fy[wid][q];
                        const int b0 = y0 - s_iy[wid][q] + 1;
#pragma unroll
                        for (int r = 0; r < TY; ++r) {
                            const int b = b0 + r;
                            if ((unsigned)b < 4u) {
                                const R wt = wxa * s_wy[wid][q][b];
                                Fx[r] += wt * Fq;
                                Fy[r] += wt * Gq;
                            }
                        }
                    }
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            if (!live[r]) continue;
            const int base = (int)LBIB_IDX((y0 + r) * L.nxp + x, L.qstride, L.chk_status);
            fx_o[base] = Fx[r];
            fy_o[base] = Fy[r];
        }
    }
    pdl_trigger();
}

// Forced lattice update of the near tiles of step m: one block of TX x TY
// threads per tile (a thread per node; blocks stride over the list), with the
// force density k_spread left in fx / fy; writes the populations, rho - 1 and
// u for the membrane update, and marks the tile as holding step m.
template <typename S, typename R>
__global__ void __launch_bounds__(TX* TY, (std::is_same<R, float>::value ? 12 : 1)) k_near_lbm(Dev d, int p)
{
    pdl_wait();  // the force density comes from k_spread
    const Lattice& L = d.L;
    const int64_t m = *d.step;
    const int c = (int)(m % 3);
    const int cnt = min(d.count[c], d.list_cap);
    const S* __restrict__ fin = static_cast<const S*>(d.f[p]);
    S* __restrict__ fout = static_cast<S*>(d.f[p ^ 1]);
    const R* __restrict__ fx_i = static_cast<const R*>(d.fx);
    const R* __restrict__ fy_i = static_cast<const R*>(d.fy);
    R* drho_o = static_cast<R*>(d.drho);
    R* ux_o = static_cast<R*>(d.ux);
    R* uy_o = static_cast<R*>(d.uy);
    const R omega = lat_param<R>(L.omega, L.omega_f);
    for (int k = blockIdx.x; k < cnt; k += gridDim.x) {
        const int t = d.list[c][k];
        const int tx = t % L.ntx, ty = t / L.ntx;
        const int4 ci = d.colinfo[tx];
        const int x = tx * TX + threadIdx.x, y = ty * TY + threadIdx.y;
        const int xl = x - ci.x;
        if (xl < ci.y && y < L.ny) {
            R g[9];
            pull<S, R>(L, fin, x, y, xl, ci.y, g);
            const int base = (int)LBIB_IDX(y * L.nxp + x, L.qstride, L.chk_status);
            R drho, ux, uy;
            collide<R>(g, fx_i[base], fy_i[base], omega, drho, ux, uy);
            if (!(drho > R(-1)) || !isfinite(ux + uy)) atomicOr(d.status, ST_DIVERGED);
#pragma unroll
            for (int q = 0; q < 9; ++q) st<S, R>(fout + q * L.qstride + base, g[q]);
            drho_o[base] = drho;
            ux_o[base] = ux;
            uy_o[base] = uy;
        }
        if (threadIdx.x == 0 && threadIdx.y == 0) d.fresh[t] = (int32_t)m;  // cleared by the next membrane update
    }
    pdl_trigger();
}

// Initial post-collision populations: equilibrium at rho = 1 with the inlet
// profile (or at rest); the columns past an instance's end (row padding) get
// zeros, so the whole buffer is written and needs no fill beforehand.
template <typename S, typename R>
__global__ void k_init_populations(Dev d, int buf)
{
    const Lattice& L = d.L;
    int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    if (y >= L.ny) return;
    S* f = static_cast<S*>(d.f[buf]);
    if (x - d.colinfo[blockIdx.x].x >= d.colinfo[blockIdx.x].y) {
#pragma unroll
        for (int q = 0; q < 9; ++q)
            st<S, R>(f + LBIB_IDX(q * L.qstride + y * L.nxp + x, 9LL * L.qstride, L.chk_status), R(0));
        return;
    }
    R u = (L.bc == LBIB_BC_INLET_OUTLET) ? inlet_profile<R>(L, y) : R(0);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        R eu = R(cx(q)) * u;
        st<S, R>(f + LBIB_IDX(q * L.qstride + y * L.nxp + x, 9LL * L.qstride, L.chk_status),
                 wq<R>(q) * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * u * u));
    }
}

// Density and velocity of lattice step m from the post-collision populations:
// sum f* = rho, sum f* e = rho u + F / 2 with F the force density of the step
// (the near kernel's on tiles it updated at step m, else the uniform body
// force).  One formula for every tile, so a read does not depend on which
// tiles were scheduled near.
template <typename S, typename R, typename O>
__global__ void k_macro(Dev d, int buf, int64_t m, int x0, int inx, O* rho_o, O* ux_o, O* uy_o, int add_one)
{
    const Lattice& L = d.L;
    const int xl = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    if (xl >= inx || y >= L.ny) return;
    const int x = x0 + xl;
    int t = blockIdx.y * L.ntx + x / TX;
    int base = (int)LBIB_IDX(y * L.nxp + x, L.qstride, L.chk_status), ob = y * inx + xl;
    R Fx = lat_param<R>(L.gx, L.gx_f), Fy = lat_param<R>(L.gy, L.gy_f);
    if (d.fresh[t] == (int32_t)m) {
        Fx = static_cast<const R*>(d.fx)[base];
        Fy = static_cast<const R*>(d.fy)[base];
    }
    const S* f = static_cast<const S*>(d.f[buf]);
    R g[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) g[q] = ld<S, R>(f + q * L.qstride + base);
    const R drho = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8];
    const R jx = (g[1] + g[5] + g[8]) - (g[3] + g[6] + g[7]) - R(0.5) * Fx;
    const R jy = (g[2] + g[5] + g[6]) - (g[4] + g[7] + g[8]) - R(0.5) * Fy;
    const R ux = jx / (R(1) + drho);
    const R uy = jy / (R(1) + drho);
    if (rho_o) rho_o[ob] = add_one ? O(1) + O(drho) : O(drho);
    if (ux_o) ux_o[ob] = O(ux);
    if (uy_o) uy_o[ob] = O(uy);
}

// Marks as near, for lattice steps m (which & 1) and m + 1 (which & 2), every
// tile within an element's reach of its centroid of X^m (initial activation
// and after a restore).
template <typename R>
__global__ void k_activate(Dev d, int64_t m, int which)
{
    const Lattice& L = d.L;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.nmark) return;
    int b = 0;
    while (b + 1 < d.nbodies && d.body[b + 1].off <= k) ++b;
    const BodyConst& B = d.body[b];
    int l = k - B.off, w = B.off + (l + 1) % B.nv;
    const double* P = d.pos[m & 1];
    double X = 0.5 * (P[k] + P[w]), Y = 0.5 * (P[d.nmark + k] + P[d.nmark + w]);
    // positions are in instance coordinates; the box is clipped to the instance
    // half-width: vertex / probe offset plus the stencil (max(l / 2, 1.2) + 2)
    // and a quarter node of motion, as the membrane update's activation
    const double ex_ = P[w] - P[k], ey_ = P[d.nmark + w] - P[d.nmark + k];
    const double ra = fmax(0.5 * sqrt(ex_ * ex_ + ey_ * ey_), 1.2) + 2.25;
    int i0 = B.x0 + max(0, (int)floor(X - ra)), i1 = B.x0 + min(B.nxi - 1, (int)floor(X + ra) + 1);
    int j0 = max(0, (int)floor(Y - 0.5 - ra)), j1 = min(L.ny - 1, (int)floor(Y - 0.5 + ra) + 1);
    if (i0 > i1 || j0 > j1) return;
    for (int s = 0; s < 2; ++s) {
        if (!(which & (1 << s))) continue;
        int64_t step = m + s;
        uint32_t* flag = d.nearflag[step % 3];
        int c = (int)(step % 3);
        for (int ty = j0 / TY; ty <= j1 / TY; ++ty)
            for (int tx = i0 / TX; tx <= i1 / TX; ++tx) {
                int t = ty * L.ntx + tx;
                if (flag[t] == 0u && atomicExch(&flag[t], 1u) == 0u) {
                    int pos = atomicAdd(&d.count[c], 1);
                    if (pos < d.list_cap) d.list[c][pos] = t;
                    else atomicOr(d.status, ST_LIST_OVERFLOW);
                }
            }
    }
}

// Sets the spreading bit masks of the markers of lattice step m (after a restore).
template <typename R>
__global__ void k_rebuild_mask(Dev d, int parity, int slot)
{
    const Lattice& L = d.L;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.nmark) return;
    const R* mkf = static_cast<const R*>(d.mkf[parity]);
    const int32_t* mki = d.mki[parity];
    int nm = d.nmark;
    if (mkf[2 * nm + k] == R(0) && mkf[3 * nm + k] == R(0)) return;
    int b = 0;
    while (b + 1 < d.nbodies && d.body[b + 1].off <= k) ++b;
    const BodyConst& B = d.body[b];
    const int kl = k - B.moff;  // instance-local marker id
    int i0 = max(B.x0, mki[k] - 1), i1 = min(B.x0 + B.nxi - 1, mki[k] + 2);
    int j0 = max(0, mki[nm + k] - 1), j1 = min(L.ny - 1, mki[nm + k] + 2);
    if (i0 > i1 || j0 > j1) return;
    for (int ty = j0 / TY; ty <= j1 / TY; ++ty)
        for (int tx = i0 / TX; tx <= i1 / TX; ++tx) {
            int t = ty * L.ntx + tx;
            if (!d.nearflag[slot][t]) atomicOr(d.status, ST_SPREAD_MISS);
            atomicOr(&d.mask[parity][(size_t)t * d.mw + (kl >> 5)], 1u << (kl & 31));
        }
}

// ------------------------------------------------------------------ launchers

// Calls fn(S*, R*) with null pointers of the storage and compute types of the
// context's populations (the lattice kernels are templates on both).
template <typename F>
static void by_store(int store, F&& fn)
{
    switch (store) {
    case STORE_F64: fn((double*)nullptr, (double*)nullptr); break;
    case STORE_BF16: fn((__nv_bfloat16*)nullptr, (float*)nullptr); break;
    case STORE_F16: fn((__half*)nullptr, (float*)nullptr); break;
    default: fn((float*)nullptr, (float*)nullptr); break;
    }
}

#define LBIB_TYPES(sp, rp)                                  \
    using S = typename std::remove_pointer<decltype(sp)>::type; \
    using R = typename std::remove_pointer<decltype(rp)>::type

template <int RT, int NPT>
static void launch_bulk_rt(const Dev& d, int parity, int slot, cudaStream_t s)
{
    dim3 grid(d.L.ntx, (d.L.nty + RT - 1) / RT), block(TX, TY * RT / NPT);
    const bool forced = d.L.gx != 0.0 || d.L.gy != 0.0;  // uniform body force (PERIODIC_FORCE mode)
    by_store(d.store, [&](auto sp, auto rp) {
        LBIB_TYPES(sp, rp);
        if (forced) k_bulk<S, R, RT, NPT, true><<<grid, block, 0, s>>>(d, parity, slot);
        else k_bulk<S, R, RT, NPT, false><<<grid, block, 0, s>>>(d, parity, slot);
    });
}

template <typename S>
static CUtensorMapDataType tb_dtype()
{
    if (std::is_same<S, double>::value) return CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    if (std::is_same<S, float>::value) return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    if (std::is_same<S, __nv_bfloat16>::value) return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
}

cudaError_t make_population_maps(const Dev& d, void* out)
{
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (!fn || q != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    CUtensorMap* maps = static_cast<CUtensorMap*>(out);
    CUresult r = CUDA_SUCCESS;
    by_store(d.store, [&](auto sp, auto rp) {
        LBIB_TYPES(sp, rp);
        (void)sizeof(R);
        const cuuint64_t es = sizeof(S);
        // x (row pitch nxp), y (ny rows), plane q (stride ny nxp)
        const cuuint64_t dims[3] = {(cuuint64_t)d.L.nxp, (cuuint64_t)d.L.ny, 9};
        const cuuint64_t strides[2] = {(cuuint64_t)d.L.nxp * es, (cuuint64_t)d.L.qstride * es};
        const cuuint32_t box[3] = {(cuuint32_t)tb_w<S>(), (cuuint32_t)(TB_ROWS + 2), 9};
        const cuuint32_t estr[3] = {1, 1, 1};
        for (int b = 0; b < 2 && r == CUDA_SUCCESS; ++b)
            r = encode(&maps[b], tb_dtype<S>(), 3, d.f[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    });
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t configure_bulk_tma(int store)
{
    cudaError_t e = cudaSuccess;
    by_store(store, [&](auto sp, auto rp) {
        LBIB_TYPES(sp, rp);
        const int bytes = (int)(TB_STAGES * tb_stage_bytes<S>() + 128);
        e = cudaFuncSetAttribute(k_bulk_tma<S, R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_bulk_tma<S, R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    });
    return e;
}

static void launch_bulk_tma(const Dev& d, int parity, int slot, cudaStream_t s)
{
    const int njobs = d.L.ntx * ((d.L.nty + 1) / 2);
    const int grid = std::max(1, (njobs + TB_JOBS - 1) / TB_JOBS);
    const bool forced = d.L.gx != 0.0 || d.L.gy != 0.0;
    const CUtensorMap& tm = static_cast<const CUtensorMap*>(d.fmaps)[parity];
    by_store(d.store, [&](auto sp, auto rp) {
        LBIB_TYPES(sp, rp);
        const size_t bytes = TB_STAGES * tb_stage_bytes<S>() + 128;
        if (forced) k_bulk_tma<S, R, true><<<grid, dim3(TX, TB_ROWS), bytes, s>>>(tm, d, parity, slot);
        else k_bulk_tma<S, R, false><<<grid, dim3(TX, TB_ROWS), bytes, s>>>(tm, d, parity, slot);
    });
}

static void launch_bulk_vec(const Dev& d, int parity, int slot, cudaStream_t s)
{
    const int rt = (d.bulk_tiles_y == 2 || d.bulk_tiles_y == 4) ? d.bulk_tiles_y : 1;
    const dim3 block(32, 2 * rt);  // a warp per tile row
    const bool forced = d.L.gx != 0.0 || d.L.gy != 0.0;
    by_store(d.store, [&](auto sp, auto rp) {
        LBIB_TYPES(sp, rp);
        constexpr int V = vec_width<S>();
        const dim3 grid((d.L.nxp + 32 * V - 1) / (32 * V), (d.L.nty + block.y - 1) / block.y);
        if (forced) k_bulk_vec<S, R, V, true><<<grid, block, 0, s>>>(d, parity, slot);
        else k_bulk_vec<S, R, V, false><<<grid, block, 0, s>>>(d, parity, slot);
    });
}

cudaError_t launch_lbm_bulk(const Dev& d, int prec, int parity, int slot, cudaStream_t s)
{
    (void)prec;  // the storage type fixes the compute type
    if (d.bulk_tma && d.fmaps) {
        launch_bulk_tma(d, parity, slot, s);
        return cudaGetLastError();
    }
    if (d.bulk_nodes_per_thread == 4) {
        launch_bulk_vec(d, parity, slot, s);
        return cudaGetLastError();
    }
    const int v = 10 * (d.bulk_tiles_y == 2 || d.bulk_tiles_y == 4 ? d.bulk_tiles_y : 1) +
                  (d.bulk_nodes_per_thread == 2 ? 2 : 1);
    switch (v) {
    case 12: launch_bulk_rt<1, 2>(d, parity, slot, s); break;
    case 21: launch_bulk_rt<2, 1>(d, parity, slot, s); break;
    case 22: launch_bulk_rt<2, 2>(d, parity, slot, s); break;
    case 41: launch_bulk_rt<4, 1>(d, parity, slot, s); break;
    case 42: launch_bulk_rt<4, 2>(d, parity, slot, s); break;
    default: launch_bulk_rt<1, 1>(d, parity, slot, s); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_lbm_near(const Dev& d, int prec, int parity, int grid, int update_grid, cudaStream_t s, bool pdl)
{
    (void)prec;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * NEAR_WARPS);
    cfg.stream = s;
    int na = 0;
    if (d.chain_priority) {
        attr[na].id = cudaLaunchAttributePriority;
        attr[na++].val.priority = d.chain_priority;
    }
    if (pdl) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na++].val.programmaticStreamSerializationAllowed = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    cudaError_t e = cudaSuccess;
    by_store(d.store, [&](auto sp, auto rp) {
        LBIB_TYPES(sp, rp);
        if (d.L.transfer == LBIB_TRANSFER_MLS) e = cudaLaunchKernelEx(&cfg, k_spread<R, true>, d, parity);
        else e = cudaLaunchKernelEx(&cfg, k_spread<R, false>, d, parity);
        if (e != cudaSuccess) return;
        // one tile per block at a time, striding over the list
        cfg.gridDim = dim3((unsigned)std::max(1, std::min(d.list_cap, update_grid)));
        cfg.blockDim = dim3(TX, TY);
        e = cudaLaunchKernelEx(&cfg, k_near_lbm<S, R>, d, parity);
    });
    return e;
}

cudaError_t launch_init_populations(const Dev& d, int prec, int buf, cudaStream_t s)
{
    (void)prec;
    dim3 grid(d.L.ntx, d.L.nty), block(TX, TY);
    by_store(d.store, [&](auto sp, auto rp) {
        LBIB_TYPES(sp, rp);
        k_init_populations<S, R><<<grid, block, 0, s>>>(d, buf);
    });
    return cudaGetLastError();
}

cudaError_t launch_macro(const Dev& d, int prec, int buf, int64_t m, int x0, int inx, double* rho, double* ux,
                         double* uy, cudaStream_t s)
{
    (void)prec;
    dim3 grid((inx + TX - 1) / TX, d.L.nty), block(TX, TY);
    by_store(d.store, [&](auto sp, auto rp) {
        LBIB_TYPES(sp, rp);
        k_macro<S, R, double><<<grid, block, 0, s>>>(d, buf, m, x0, inx, rho, ux, uy, 1);
    });
    return cudaGetLastError();
}

cudaError_t launch_macro_typed(const Dev& d, int prec, int buf, int64_t m, int x0, int inx, void* ux, void* uy,
                               int dtype, cudaStream_t s)
{
    (void)prec;
    dim3 grid((inx + TX - 1) / TX, d.L.nty), block(TX, TY);
    by_store(d.store, [&](auto sp, auto rp) {
        LBIB_TYPES(sp, rp);
        if (dtype == 1)
            k_macro<S, R, double><<<grid, block, 0, s>>>(d, buf, m, x0, inx, nullptr, (double*)ux, (double*)uy, 1);
        else
            k_macro<S, R, float><<<grid, block, 0, s>>>(d, buf, m, x0, inx, nullptr, (float*)ux, (float*)uy, 1);
    });
    return cudaGetLastError();
}

#undef LBIB_TYPES

cudaError_t launch_activate(const Dev& d, int prec, int64_t m, int which, cudaStream_t s)
{
    if (d.nmark == 0) return cudaSuccess;
    int th = 128, bl = (d.nmark + th - 1) / th;
    if (prec == PREC_F64) k_activate<double><<<bl, th, 0, s>>>(d, m, which);
    else k_activate<float><<<bl, th, 0, s>>>(d, m, which);
    return cudaGetLastError();
}

cudaError_t launch_rebuild_mask(const Dev& d, int prec, int64_t m, cudaStream_t s)
{
    if (d.nmark == 0) return cudaSuccess;
    int th = 128, bl = (d.nmark + th - 1) / th;
    const int parity = (int)(m & 1), slot = (int)(m % 3);
    if (prec == PREC_F64) k_rebuild_mask<double><<<bl, th, 0, s>>>(d, parity, slot);
    else k_rebuild_mask<float><<<bl, th, 0, s>>>(d, parity, slot);
    return cudaGetLastError();
}

}  // namespace lbib
