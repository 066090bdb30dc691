// lbib_lag_kernel.cuh -- the Lagrangian update: one thread block per membrane
// (kernel template; instantiated for the Peskin transfer in lbib_lag.cu and
// for the MLS transfer in lbib_lag_mls.cu, compiled in parallel).
//
// Lagrangian step n (after the lattice step n has written rho^n - 1 and u^n on
// its near tiles), for the block's body, in this order:
//   1. chain geometry at X^n: edges, lengths, outward element normals, vertex
//      normals and signed turning angles; shoelace area in FP64;
//   2. fluid velocity at the vertices (Sec. 2.8) with the truncated Peskin
//      stencil; pressure and velocity gradient at a probe 1.2 dx along each
//      element normal, stopped at a wall it would cross (Sec. 2.6);
//   3. ligand-receptor kinetics from Philox4x32-10 draws keyed on (seed;
//      step, site), then Eq. 13 per element (Sec. 2.5);
//   4. Eq. 8, Eq. 10, Eq. 11 (deformable bodies), Eq. 12 against the vertices
//      of every other body, Eqs. 14-15; element forces split half to each of
//      the element's vertices; the total of Eq. 16;
//   5. Verlet (Eq. 17) and BDF2 velocity (Eq. 18), or rigid BDF2 (Eq. 19), or
//      nothing for a body fixed to the wall;
//   6. direct forcing rho (U_struct - U*) at the new element centroids,
//      written as markers for lattice step n + 1 together with the bit masks of
//      the tiles their stencils touch (the tiles around the new centroids are
//      scheduled as near for lattice step n + 2 by k_activate_next, which runs
//      after this kernel off the membrane -> near chain);
//   7. area, perimeter change, centroid and extent of X^{n+1} (per body, for
//      k_observables, which writes the record of step n + 1 right after); the
//      last block to finish advances n.
//
// The kernel is latency-bound (a few hundred markers per block).  Positions
// are carried as float-float pairs (value = hi + lo) so that differences,
// stencil origins and fractional offsets, probe and centroid positions and
// the Verlet update are exact to ~1e-12 dx in FP32 arithmetic; FP64 appears
// only in the conversions at load and store and in the area and centroid
// reductions, never in a long dependent chain.  Each interpolation point is
// sampled by a group of K = 4, 2 or 1 lanes (as many as keep the largest
// body in one pass over the block), each lane summing 4 / K stencil rows.
#pragma once
#include <cuda_runtime.h>

#include "lbib_device.cuh"

namespace lbib {

// ---------------------------------------------------- float-float positions
template <typename R>
struct P2 {
    R h, l;
};

template <typename R>
__device__ __forceinline__ P2<R> p2_of(double X)
{
    const R h = (R)X;
    return P2<R>{h, (R)(X - (double)h)};
}

template <typename R>
__device__ __forceinline__ double p2_double(P2<R> p)
{
    return (double)p.h + (double)p.l;
}

// a - b as a single compute-precision value
template <typename R>
__device__ __forceinline__ R p2_sub(P2<R> a, P2<R> b)
{
    return (a.h - b.h) + (a.l - b.l);
}

// a + d, renormalised (Knuth TwoSum on the high part)
template <typename R>
__device__ __forceinline__ P2<R> p2_add(P2<R> a, R d)
{
    const R s = a.h + d;
    const R bb = s - a.h;
    const R err = (a.h - (s - bb)) + (d - bb);
    const R lo = a.l + err;
    const R h2 = s + lo;
    return P2<R>{h2, lo - (h2 - s)};
}

// integer floor of a - shift and the fractional remainder in [0, 1)
template <typename R>
__device__ __forceinline__ void p2_floor(P2<R> a, R shift, int& i, R& frac)
{
    const R h = a.h - shift;
    R f = floor(h);
    R r = (h - f) + a.l;
    if (r < R(0)) {
        f -= R(1);
        r += R(1);
    } else if (r >= R(1)) {
        f += R(1);
        r -= R(1);
    }
    i = (int)f;
    frac = r;
}

// ---------------------------------------------------------------- sampling
template <typename R>
struct Sample {
    R u, v, ux, uy, vx, vy, drho, W;  // drho: renormalised rho - 1
};

template <typename R>
struct Spot {
    int ix, jy;  // floor(X), floor(Y - 1/2)
    R ax, ay;    // X - ix, Y - 1/2 - jy
};

template <typename R>
__device__ __forceinline__ Spot<R> spot_of(P2<R> X, P2<R> Y)
{
    Spot<R> s;
    p2_floor<R>(X, R(0), s.ix, s.ax);
    p2_floor<R>(Y, R(0.5), s.jy, s.ay);
    return s;
}

// Products and fused multiply-adds with rounding stated explicitly, so that a
// sum is evaluated the same way whatever the surrounding code.
template <typename R>
__device__ __forceinline__ R mul_rn(R a, R b);
template <>
__device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <>
__device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }

template <typename R, bool GRAD>
struct RowSums {
    R W, u, v, r, ux, uy, vx, vy;
    __device__ __forceinline__ void add(const RowSums& o)
    {
        W += o.W;
        u += o.u;
        v += o.v;
        r += o.r;
        if (GRAD) {
            ux += o.ux;
            uy += o.uy;
            vx += o.vx;
            vy += o.vy;
        }
    }
    __device__ __forceinline__ RowSums xor_partner(int o) const
    {
        RowSums t;
        t.W = __shfl_xor_sync(0xffffffffu, W, o);
        t.u = __shfl_xor_sync(0xffffffffu, u, o);
        t.v = __shfl_xor_sync(0xffffffffu, v, o);
        t.r = __shfl_xor_sync(0xffffffffu, r, o);
        if (GRAD) {
            t.ux = __shfl_xor_sync(0xffffffffu, ux, o);
            t.uy = __shfl_xor_sync(0xffffffffu, uy, o);
            t.vx = __shfl_xor_sync(0xffffffffu, vx, o);
            t.vy = __shfl_xor_sync(0xffffffffu, vy, o);
        }
        return t;
    }
};

// Truncated-stencil velocity (and optionally its gradient) and renormalised
// density deviation at a point from the near-tile output of lattice step m,
// computed by a group of K lanes (K = 1, 2, 4): lane r takes the stencil rows
// jy - 1 + r, jy - 1 + r + K, ...  Each row is summed over its four nodes in
// order and the four row sums are combined as (row0 + row1) + (row2 + row3)
// for every K (by shuffles across the group), so the result does not depend
// on K; every lane of the group gets it.  The point is in the coordinates of
// its instance (node columns [x0, x0 + nxi) of the lattice).  Indices are
// clamped into the instance and the weights of nodes outside it zeroed, so a
// lane's loads are independent and issued together.  All 32 lanes of the warp
// must call this together.  With the MLS transfer the node weights are the
// fit's shape functions (value and gradient) over the whole stencil, wall
// nodes included with zero velocity, as for the Peskin weights.
template <typename R, bool GRAD, int K, bool MLS>
__device__ __forceinline__ void sample_group(const Dev& d, const Spot<R>& sp, int32_t m, int r, int x0, int nxi,
                                             Sample<R>& o, uint32_t& miss)
{
    const Lattice& L = d.L;
    const R* __restrict__ ux = static_cast<const R*>(d.ux);
    const R* __restrict__ uy = static_cast<const R*>(d.uy);
    const R* __restrict__ dr = static_cast<const R*>(d.drho);
    constexpr int NR = 4 / K;  // rows per lane
    const int i0 = sp.ix - 1;
    int ic[4];
    R px[4], dpx[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = i0 + a;
        const bool vi = (i >= 0 && i < nxi);
        ic[a] = x0 + min(max(i, 0), nxi - 1);
        const R rx = sp.ax + R(1 - a);  // X - i
        dpx[a] = R(0);
        if constexpr (MLS) {
            px[a] = mls_w<R>(rx);  // wall nodes are zeroed once the moments are formed
        } else {
            if (GRAD) peskin_both<R>(rx, px[a], dpx[a]);
            else px[a] = peskin<R>(rx);
            if (!vi) px[a] = dpx[a] = R(0);
        }
    }
    // MLS: the fit's inverse moment matrix over the whole 4 x 4 stencil (nodes
    // beyond a wall or an instance end are wall nodes); every lane forms it
    // from the same terms in the same order, whatever K
    R inv[9];
    if constexpr (MLS) {
        R a0 = R(0), a1 = R(0), a2 = R(0), b0 = R(0), b1 = R(0), b2 = R(0);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const R dx = R(a - 1) - sp.ax;  // x_i - X
            a0 += px[a];
            a1 += px[a] * dx;
            a2 += px[a] * dx * dx;
        }
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const R dy = R(rr - 1) - sp.ay;  // y_j - Y
            const R w = mls_w<R>(dy);
            b0 += w;
            b1 += w * dy;
            b2 += w * dy * dy;
        }
        if (!mls_inverse<R>(a0, a1, a2, b0, b1, b2, inv)) {
#pragma unroll
            for (int q = 0; q < 9; ++q) inv[q] = R(0);  // not reached: the full stencil is regular
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
            if (!(i0 + a >= 0 && i0 + a < nxi)) px[a] = R(0);  // wall nodes: zero velocity
    }
    int jc[NR];
    R py[NR], dpy[NR];
    int32_t fr[2 * NR];
    R a_u[4 * NR], a_v[4 * NR], a_r[4 * NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int rr = r + K * k;
        const int j = sp.jy - 1 + rr;
        const bool vj = (j >= 0 && j < L.ny);
        jc[k] = min(max(j, 0), L.ny - 1);
        const R ry = sp.ay + R(1 - rr);  // Y - (j + 1/2)
        dpy[k] = R(0);
        if constexpr (MLS) py[k] = mls_w<R>(ry);
        else if (GRAD) peskin_both<R>(ry, py[k], dpy[k]);
        else py[k] = peskin<R>(ry);
        if (!vj) py[k] = dpy[k] = R(0);
        // the row's nodes lie in at most two tiles: both must hold step m
        fr[2 * k] = d.fresh[LBIB_IDX(tile_of(L, ic[0], jc[k]), L.ntiles, L.chk_status)];
        fr[2 * k + 1] = d.fresh[LBIB_IDX(tile_of(L, ic[3], jc[k]), L.ntiles, L.chk_status)];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int idx = (int)LBIB_IDX(jc[k] * L.nxp + ic[a], L.qstride, L.chk_status);
            a_u[4 * k + a] = ux[idx];
            a_v[4 * k + a] = uy[idx];
            a_r[4 * k + a] = dr[idx];
        }
    }
#pragma unroll
    for (int k = 0; k < 2 * NR; ++k)
        if (fr[k] != m) miss = 1u;
    RowSums<R, GRAD> rs[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        RowSums<R, GRAD>& s = rs[k];
        s.W = s.u = s.v = s.r = s.ux = s.uy = s.vx = s.vy = R(0);
        const R dy = R(r + K * k - 1) - sp.ay;  // y_j - Y (MLS)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            R w, wx = R(0), wy = R(0);
            if constexpr (MLS) {
                // shape functions W_j (inv_r . (1, dx, dy)) of the value and the gradient
                const R base = mul_rn<R>(px[a], py[k]), dx = R(a - 1) - sp.ax;
                w = base * (inv[0] + inv[1] * dx + inv[2] * dy);
                if (GRAD) {
                    wx = base * (inv[3] + inv[4] * dx + inv[5] * dy);
                    wy = base * (inv[6] + inv[7] * dx + inv[8] * dy);
                }
            } else {
                w = mul_rn<R>(px[a], py[k]);
                if (GRAD) {
                    wx = mul_rn<R>(dpx[a], py[k]);
                    wy = mul_rn<R>(px[a], dpy[k]);
                }
            }
            const int q = 4 * k + a;
            s.W += w;
            s.u = fma(a_u[q], w, s.u);
            s.v = fma(a_v[q], w, s.v);
            s.r = fma(a_r[q], w, s.r);
            if (GRAD) {
                s.ux = fma(a_u[q], wx, s.ux);
                s.uy = fma(a_u[q], wy, s.uy);
                s.vx = fma(a_v[q], wx, s.vx);
                s.vy = fma(a_v[q], wy, s.vy);
            }
        }
    }
    // (row0 + row1) + (row2 + row3); IEEE addition is commutative, so both
    // lanes of a pair form the same partial sum
    RowSums<R, GRAD> t;
    if (K == 1) {
        t = rs[0];
        t.add(rs[1]);
        RowSums<R, GRAD> t2 = rs[NR > 2 ? 2 : 0];
        t2.add(rs[NR > 3 ? 3 : 0]);
        t.add(t2);
    } else if (K == 2) {  // lane r holds rows r and r + 2
        t = rs[0];
        t.add(rs[0].xor_partner(1));
        RowSums<R, GRAD> t2 = rs[NR > 1 ? 1 : 0];
        t2.add(rs[NR > 1 ? 1 : 0].xor_partner(1));
        t.add(t2);
    } else {  // K == 4: lane r holds row r
        t = rs[0];
        t.add(t.xor_partner(1));
        t.add(t.xor_partner(2));
    }
    o.W = t.W;
    o.u = t.u;
    o.v = t.v;
    if (GRAD) {
        o.ux = t.ux;
        o.uy = t.uy;
        o.vx = t.vx;
        o.vy = t.vy;
    } else {
        o.ux = o.uy = o.vx = o.vy = R(0);
    }
    // density: no wall value, weights renormalised over the fluid nodes
    o.drho = (t.W > R(0)) ? t.r / t.W : R(0);
}

// Tiles overlapping the node box [i0, i1] x [j0, j1]: enumerates at most 8 of
// them per call into t[], starting after `start` tiles; returns the count.
__device__ __forceinline__ int box_tiles(const Lattice& L, int i0, int i1, int j0, int j1, int start, int t[8])
{
    int n = 0, k = 0;
    for (int ty = j0 / TY; ty <= j1 / TY; ++ty)
        for (int tx = i0 / TX; tx <= i1 / TX; ++tx) {
            if (k++ < start) continue;
            if (n < 8) t[n++] = ty * L.ntx + tx;
        }
    return n;
}

// Sums of per-vertex terms are laid out over VLANES virtual lanes (vertex v
// in lane v % VLANES, each lane summing its vertices in ascending order) and
// combined by one fixed shuffle tree, whatever the block size T: a thread of
// a T-thread block holds VL = VLANES / T lanes.  So T changes no result.
constexpr int VLANES = 512;

template <typename V, int VL>
__device__ __forceinline__ V vlane_sum(V (&acc)[VL], V* scratch)  // scratch: >= VLANES / 32 elements
{
    constexpr int W = VLANES / VL / 32;  // warps of the block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < VL; ++j) acc[j] = warp_sum(acc[j]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < VL; ++j) scratch[j * W + wid] = acc[j];
    __syncthreads();
    const V t = (lane < VLANES / 32) ? scratch[lane] : V(0);
    return warp_sum(t);
}

template <typename R, int K, int T, bool MLS>
__global__ void __launch_bounds__(T) k_lagrangian(Dev d, int p)
{
    static_assert(VLANES % T == 0 && T % 32 == 0, "block size divides the virtual lanes");
    constexpr int VL = VLANES / T;
    const Lattice& L = d.L;
    const int bi = blockIdx.x;
    const BodyConst& B = d.body[bi];
    const int nv = B.nv, off = B.off, NM = d.nmark, tid = threadIdx.x;
    const int64_t n = *d.step;
    const int32_t mf = (int32_t)n;  // lattice step whose rho/u the interpolation reads
    const double* __restrict__ Pn = d.pos[n & 1];
    double* Pw = d.pos[(n + 1) & 1];  // X^{n-1} on entry, X^{n+1} on exit
    const R* __restrict__ Fn = static_cast<const R*>(d.posf[n & 1]);
    R* Fw = static_cast<R*>(d.posf[(n + 1) & 1]);
    R* diag = static_cast<R*>(d.diag);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* xh = reinterpret_cast<R*>(smem_raw);  // X^n
    R* xl = xh + nv;
    R* yh = xl + nv;
    R* yl = yh + nv;
    R* qxh = yl + nv;  // X^{n+1}
    R* qxl = qxh + nv;
    R* qyh = qxl + nv;
    R* qyl = qyh + nv;
    R* ddx = qyl + nv;  // X^n - X^{n-1}
    R* ddy = ddx + nv;
    R* ex = ddy + nv;
    R* ey = ex + nv;
    R* len = ey + nv;
    R* nlx = len + nv;
    R* nly = nlx + nv;
    R* vnx = nly + nv;
    R* vny = vnx + nv;
    R* th = vny + nv;
    R* uvx = th + nv;
    R* uvy = uvx + nv;
    R* ewx = uvy + nv;
    R* ewy = ewx + nv;
    R* ehx = ewy + nv;
    R* ehy = ehx + nv;
    R* fpx = ehy + nv;
    R* fpy = fpx + nv;
    R* ftx = fpy + nv;
    R* fty = ftx + nv;
    R* svx = fty + nv;
    R* svy = svx + nv;
    R* sl0 = svy + nv;
    R* sth0 = sl0 + nv;
    R* ilen = sth0 + nv;
    __shared__ double dscr[8][32];
    __shared__ R rscr[8][32];
    __shared__ double rig[RG_N];
    __shared__ double rot[2];
    __shared__ R ext[MAX_BODIES][4];
    uint32_t miss = 0u, bad = 0u;
    const int lane4 = tid % K, Q = T / K;  // K lanes per interpolation point
    const int nvq = ((nv + Q - 1) / Q) * Q;

    // the near update of lattice step n is done: its tiles' flags (slot n % 3)
    // are cleared here, spread over the blocks; the last block then empties
    // the list (the slot is set again for step n + 3 by the next update)
    {
        const int c0 = (int)(n % 3);
        const int cnt = min(d.count[c0], d.list_cap);
        uint32_t* f0 = d.nearflag[c0];
        const int32_t* l0 = d.list[c0];
        for (int k = blockIdx.x * T + tid; k < cnt; k += gridDim.x * T) f0[LBIB_IDX(l0[k], L.ntiles, L.chk_status)] = 0u;
    }

    // 0. one round of global loads; positions to float-float pairs; the FP64
    //    shoelace terms of X^n (Eq. 11's area) directly from the loaded values
    double a2[VL];
#pragma unroll
    for (int j = 0; j < VL; ++j) a2[j] = 0.0;
    {
        const R* l0 = static_cast<const R*>(d.l0) + off;
        const R* th0 = static_cast<const R*>(d.th0) + off;
        for (int v0 = tid; v0 < nv; v0 += VLANES)
#pragma unroll
        for (int j = 0; j < VL; ++j) {
            const int v = v0 + j * T;  // virtual lane tid + j T
            if (v >= nv) break;
            const int w = (v + 1 == nv) ? 0 : v + 1;
            const double X = Pn[off + v], Y = Pn[NM + off + v];
            const double Xw = Pn[off + w], Yw = Pn[NM + off + w];
            const double Xp = Pw[off + v], Yp = Pw[NM + off + v];
            const P2<R> px = p2_of<R>(X), py = p2_of<R>(Y);
            xh[v] = px.h;
            xl[v] = px.l;
            yh[v] = py.h;
            yl[v] = py.l;
            ddx[v] = (R)(X - Xp);
            ddy[v] = (R)(Y - Yp);
            sl0[v] = l0[v];
            sth0[v] = th0[v];
            a2[j] += X * Yw - Xw * Y;
        }
        if (tid < RG_N) rig[tid] = d.rigid[bi * RG_N + tid];
        const double* eo = d.body_obs[n & 1] + (size_t)B.b0 * BO_N;  // the instance's bodies
        for (int k = tid; k < 4 * B.nbi; k += T) ext[k >> 2][k & 3] = (R)eo[(k >> 2) * BO_N + BO_XMIN + (k & 3)];
    }
    const double area = 0.5 * vlane_sum<double, VL>(a2, dscr[0]);  // FP64 area reduction (Eq. 11)

    // 1. geometry at X^n (the reduction above synchronised the block)
    for (int l = tid; l < nv; l += T) {
        const int w = (l + 1 == nv) ? 0 : l + 1;
        const R dx = p2_sub<R>(P2<R>{xh[w], xl[w]}, P2<R>{xh[l], xl[l]});
        const R dy = p2_sub<R>(P2<R>{yh[w], yl[w]}, P2<R>{yh[l], yl[l]});
        const R ll = sqrt(dx * dx + dy * dy);
        const R il = R(1) / ll;
        ex[l] = dx;
        ey[l] = dy;
        len[l] = ll;
        ilen[l] = il;
        nlx[l] = dy * il;
        nly[l] = -dx * il;
    }
    __syncthreads();
    for (int v = tid; v < nv; v += T) {
        const int lm = (v == 0) ? nv - 1 : v - 1;
        th[v] = atan2(ex[lm] * ey[v] - ey[lm] * ex[v], ex[lm] * ex[v] + ey[lm] * ey[v]);
        const R sxn = nlx[lm] + nlx[v], syn = nly[lm] + nly[v];
        const R s = sqrt(sxn * sxn + syn * syn);
        vnx[v] = sxn / s;
        vny[v] = syn / s;
    }

    // 2. fluid velocity at each vertex and traction of each element (Eqs. 14-15);
    //    K lanes per vertex/element
    const R nu = (R)L.nu;
    for (int v0 = tid / K; v0 < nvq; v0 += Q) {
        const bool valid = v0 < nv;
        const int l = valid ? v0 : nv - 1;
        const P2<R> X = P2<R>{xh[l], xl[l]}, Y = P2<R>{yh[l], yl[l]};
        // probe: element centroid + 1.2 dx along the outward normal, stopped at a wall
        const P2<R> PX = p2_add<R>(X, R(0.5) * ex[l] + (R)d.probe * nlx[l]);
        P2<R> PY = p2_add<R>(Y, R(0.5) * ey[l] + (R)d.probe * nly[l]);
        if (PY.h + PY.l < R(0)) PY = P2<R>{R(0), R(0)};
        if (PY.h + PY.l > R(L.ny)) PY = P2<R>{R(L.ny), R(0)};
        Sample<R> o, q;
        sample_group<R, false, K, MLS>(d, spot_of<R>(X, Y), mf, lane4, B.x0, B.nxi, o, miss);
        sample_group<R, true, K, MLS>(d, spot_of<R>(PX, PY), mf, lane4, B.x0, B.nxi, q, miss);
        if (valid && lane4 == 0) {
            uvx[l] = o.u;
            uvy[l] = o.v;
            R fx = 0, fy = 0;
            if (q.W > R(0)) {
                const R pr = q.drho / R(3);  // c_s^2 rho - p_ref
                const R mu = (R(1) + q.drho) * nu;
                const R txx = R(2) * mu * q.ux, txy = mu * (q.uy + q.vx), tyy = R(2) * mu * q.vy;
                fx = (-pr * nlx[l] + txx * nlx[l] + txy * nly[l]) * len[l];
                fy = (-pr * nly[l] + txy * nlx[l] + tyy * nly[l]) * len[l];
            }
            ehx[l] = fx;
            ehy[l] = fy;
            ewx[l] = 0;
            ewy[l] = 0;
        }
    }
    __syncthreads();

    // 3. ligand-receptor kinetics (one draw per site and step) and Eq. 13
    if (B.adhesive) {
        const R* lt = static_cast<const R*>(d.lig_t);
        R* mg = static_cast<R*>(d.margin);
        const R Pf = (R)B.Pf, ycr = (R)B.ycr, yeq = (R)B.yeq, H = (R)L.ny;
        const uint64_t seed = d.inst[B.inst].seed;  // sites are numbered within the instance
        if (B.motion != LBIB_FIXED) {
            for (int k = B.lig_off + tid; k < B.lig_off + B.nlig; k += T) {
                const int l = d.lig_el[k] - off;
                const R t = lt[k];
                const int bd = d.bound[k];
                const P2<R> SX = p2_add<R>(P2<R>{xh[l], xl[l]}, t * ex[l]);
                const P2<R> SY = p2_add<R>(P2<R>{yh[l], yl[l]}, t * ey[l]);
                const R u = (R)bond_draw(seed, n, (uint32_t)(k - B.lig0));
                if (bd) {
                    const R dxa = p2_sub<R>(SX, p2_of<R>(d.anchor[k]));
                    const R dya = p2_sub<R>(SY, p2_of<R>(d.anchor[d.nlig + k]));
                    const R ylen = sqrt(dxa * dxa + dya * dya);
                    const R dy = ylen - yeq;
                    const R Pr = R(1) - exp(-(R)B.kr0_dt * exp((R)B.xi * dy * dy));
                    mg[k] = fabs(u - Pr);
                    if (u < Pr) d.bound[k] = 0;
                } else {
                    // gap to the nearest wall below y_cr, decided on the float-float value
                    const bool lower = (SY.h - H * R(0.5)) + SY.l < R(0);
                    const R gap_m_ycr = lower ? (SY.h - ycr) + SY.l : ((H - SY.h) - ycr) - SY.l;
                    if (gap_m_ycr < R(0)) {
                        mg[k] = fabs(u - Pf);
                        if (u < Pf) {
                            d.bound[k] = 1;
                            d.anchor[k] = p2_double<R>(SX);
                            d.anchor[d.nlig + k] = lower ? 0.0 : (double)L.ny;
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (!B.sigma_inf) {
            // Eq. 13 as a linear spring: sigma (y_l - y_eq) along the unit vector
            // from the site to its receptor (the element normal for a site on its anchor)
            const R sig = (R)B.sigma;
            for (int l = tid; l < nv; l += T) {
                R fx = 0, fy = 0;
                for (int k = d.site_off[off + l]; k < d.site_off[off + l + 1]; ++k) {
                    if (!d.bound[k]) continue;
                    const R t = lt[k];
                    const P2<R> SX = p2_add<R>(P2<R>{xh[l], xl[l]}, t * ex[l]);
                    const P2<R> SY = p2_add<R>(P2<R>{yh[l], yl[l]}, t * ey[l]);
                    const R dxa = p2_sub<R>(p2_of<R>(d.anchor[k]), SX);
                    const R dya = p2_sub<R>(p2_of<R>(d.anchor[d.nlig + k]), SY);
                    const R ylen = sqrt(dxa * dxa + dya * dya);
                    const R F = sig * (ylen - yeq);
                    const bool on = ylen > R(0);
                    fx += F * (on ? dxa / ylen : nlx[l]);
                    fy += F * (on ? dya / ylen : nly[l]);
                }
                ewx[l] = fx;
                ewy[l] = fy;
            }
        }
    }

    // repulsion (Eq. 12) from the vertices of every other body of the instance within the cut-off
    const R c0 = R(1e-4) / (R(8) * sqrt(R(2)));
    const R dcut = (R)d.dcut;
    for (int v = tid; v < nv; v += T) {
        R ax = 0, ay = 0;
        const P2<R> X = P2<R>{xh[v], xl[v]}, Y = P2<R>{yh[v], yl[v]};
        const R xa = X.h + X.l, ya = Y.h + Y.l;
        for (int ol = 0; ol < B.nbi; ++ol) {
            const int o = B.b0 + ol;
            if (o == bi) continue;
            if (xa < ext[ol][0] - dcut || xa > ext[ol][1] + dcut || ya < ext[ol][2] - dcut || ya > ext[ol][3] + dcut)
                continue;
            const BodyConst& C = d.body[o];
            for (int w = 0; w < C.nv; ++w) {
                const int g = C.off + w;
                const R ddx_ = p2_sub<R>(X, P2<R>{Fn[g], Fn[NM + g]});
                const R ddy_ = p2_sub<R>(Y, P2<R>{Fn[2 * NM + g], Fn[3 * NM + g]});
                const R dd = sqrt(ddx_ * ddx_ + ddy_ * ddy_);
                if (dd < dcut) {
                    const R mag = c0 * sqrt(R(1) / (dd * dd * dd * dd * dd));
                    ax += mag * (-vnx[v]);
                    ay += mag * (-vny[v]);
                }
            }
        }
        fpx[v] = ax;
        fpy[v] = ay;
    }
    __syncthreads();

    // 4. vertex forces (Eq. 16)
    const bool deform = (B.motion == LBIB_DEFORMABLE);
    const R ks = (R)B.ks, kb = (R)B.kb;
    // Eq. 11: -k_a (1 - A / A_0) p_ref n^- l with n^- = -n
    const R fa_c = deform ? (R)(B.ka * ((B.A0 - area) * B.inv_A0) / 3.0) : R(0);
    for (int v = tid; v < nv; v += T) {
        const int lm = (v == 0) ? nv - 1 : v - 1, w = (v + 1 == nv) ? 0 : v + 1;
        R fsx = 0, fsy = 0, fbx = 0, fby = 0;
        if (deform) {
            // Eq. 8: element lm pulls v along e_lm, element v along -e_v
            const R cl = -ks * (len[lm] - sl0[lm]) * ilen[lm];
            const R cr = -ks * (len[v] - sl0[v]) * ilen[v];
            fsx = cl * ex[lm] - cr * ex[v];
            fsy = cl * ey[lm] - cr * ey[v];
            // Eq. 10: triples centred at lm (v on its right), v, and w (v on its
            // left).  Sec. 2.3 names l_right the length of the edge on the left
            // of the centre and l_left that of the edge on its right, so an end
            // vertex takes the share of the edge on the far side of the centre
            // (the three forces then have no net torque).
            const int lmm = (lm == 0) ? nv - 1 : lm - 1;
            const R kl = kb * (th[lm] - sth0[lm]);
            const R kc = kb * (th[v] - sth0[v]);
            const R kr = kb * (th[w] - sth0[w]);
            const R cR = kl * len[lmm] / (len[lmm] + len[lm]);
            const R cL = kr * len[w] / (len[v] + len[w]);
            fbx = cR * vnx[lm] - kc * vnx[v] + cL * vnx[w];
            fby = cR * vny[lm] - kc * vny[v] + cL * vny[w];
        }
        const R fax = R(0.5) * fa_c * (len[lm] * nlx[lm] + len[v] * nlx[v]);
        const R fay = R(0.5) * fa_c * (len[lm] * nly[lm] + len[v] * nly[v]);
        const R fwx = R(0.5) * (ewx[lm] + ewx[v]), fwy = R(0.5) * (ewy[lm] + ewy[v]);
        const R fhx = R(0.5) * (ehx[lm] + ehx[v]), fhy = R(0.5) * (ehy[lm] + ehy[v]);
        const R tx = fsx + fbx + fax + fpx[v] + fwx + fhx;
        const R ty = fsy + fby + fay + fpy[v] + fwy + fhy;
        ftx[v] = tx;
        fty[v] = ty;
        const int g = off + v;
        diag[LBIB_FIELD_UVX * NM + g] = uvx[v];
        diag[LBIB_FIELD_UVY * NM + g] = uvy[v];
        diag[LBIB_FIELD_FSX * NM + g] = fsx;
        diag[LBIB_FIELD_FSY * NM + g] = fsy;
        diag[LBIB_FIELD_FBX * NM + g] = fbx;
        diag[LBIB_FIELD_FBY * NM + g] = fby;
        diag[LBIB_FIELD_FAX * NM + g] = fax;
        diag[LBIB_FIELD_FAY * NM + g] = fay;
        diag[LBIB_FIELD_FPX * NM + g] = fpx[v];
        diag[LBIB_FIELD_FPY * NM + g] = fpy[v];
        diag[LBIB_FIELD_FWX * NM + g] = fwx;
        diag[LBIB_FIELD_FWY * NM + g] = fwy;
        diag[LBIB_FIELD_FHX * NM + g] = fhx;
        diag[LBIB_FIELD_FHY * NM + g] = fhy;
        diag[LBIB_FIELD_FTX * NM + g] = tx;
        diag[LBIB_FIELD_FTY * NM + g] = ty;
    }
    __syncthreads();

    // 5. integration
    if (deform) {
        const R mv = (R)B.mv;
        for (int v = tid; v < nv; v += T) {
            // Eq. 17 (dt = 1); Eq. 18 as 3/2 (X^{n+1} - X^n) - 1/2 (X^n - X^{n-1})
            const R dxn = uvx[v] + R(0.5) * ftx[v] / mv, dyn = uvy[v] + R(0.5) * fty[v] / mv;
            const P2<R> nx_ = p2_add<R>(P2<R>{xh[v], xl[v]}, dxn);
            const P2<R> ny_ = p2_add<R>(P2<R>{yh[v], yl[v]}, dyn);
            qxh[v] = nx_.h;
            qxl[v] = nx_.l;
            qyh[v] = ny_.h;
            qyl[v] = ny_.l;
            svx[v] = R(1.5) * dxn - R(0.5) * ddx[v];
            svy[v] = R(1.5) * dyn - R(0.5) * ddy[v];
        }
    } else if (B.motion == LBIB_RIGID) {
        const double xc = rig[RG_XC], yc = rig[RG_YC];
        const P2<R> XC = p2_of<R>(xc), YC = p2_of<R>(yc);
        R sfx_[VL], sfy_[VL], smz_[VL];
#pragma unroll
        for (int j = 0; j < VL; ++j) sfx_[j] = sfy_[j] = smz_[j] = R(0);
        for (int v0 = tid; v0 < nv; v0 += VLANES)
#pragma unroll
        for (int j = 0; j < VL; ++j) {
            const int v = v0 + j * T;
            if (v >= nv) break;
            sfx_[j] += ftx[v];
            sfy_[j] += fty[v];
            const R rx = p2_sub<R>(P2<R>{xh[v], xl[v]}, XC), ry = p2_sub<R>(P2<R>{yh[v], yl[v]}, YC);
            smz_[j] += rx * fty[v] - ry * ftx[v];
        }
        const R sfx = vlane_sum<R, VL>(sfx_, rscr[0]);
        const R sfy = vlane_sum<R, VL>(sfy_, rscr[1]);
        const R smz = vlane_sum<R, VL>(smz_, rscr[2]);
        __syncthreads();
        if (tid == 0) {
            // Eq. 19: u = 2/3 (2 u(t - dt) - 1/2 u(t - 2 dt) + du/dt dt), likewise omega
            const double ux = (2.0 / 3.0) * (2.0 * rig[RG_U1X] - 0.5 * rig[RG_U2X] + (double)sfx / B.mass);
            const double uy = (2.0 / 3.0) * (2.0 * rig[RG_U1Y] - 0.5 * rig[RG_U2Y] + (double)sfy / B.mass);
            const double om = (2.0 / 3.0) * (2.0 * rig[RG_W1] - 0.5 * rig[RG_W2] + (double)smz / B.inertia);
            rig[RG_U2X] = rig[RG_U1X];
            rig[RG_U1X] = ux;
            rig[RG_U2Y] = rig[RG_U1Y];
            rig[RG_U1Y] = uy;
            rig[RG_W2] = rig[RG_W1];
            rig[RG_W1] = om;
            rig[RG_XC] = xc + ux;
            rig[RG_YC] = yc + uy;
            rig[RG_ANG] += om;
            double* rs = d.rigid + bi * RG_N;
            for (int k = 0; k < RG_N; ++k) rs[k] = rig[k];
            rot[0] = cos(rig[RG_ANG]);
            rot[1] = sin(rig[RG_ANG]);
        }
        __syncthreads();
        const R ux = (R)rig[RG_U1X], uy = (R)rig[RG_U1Y], om = (R)rig[RG_W1];
        const R cs = (R)rot[0], sn = (R)rot[1];
        const P2<R> NCX = p2_of<R>(rig[RG_XC]), NCY = p2_of<R>(rig[RG_YC]);
        for (int v = tid; v < nv; v += T) {
            const R a = (R)d.rref[off + v], b = (R)d.rref[NM + off + v];
            const R rx = cs * a - sn * b, ry = sn * a + cs * b;
            const P2<R> nx_ = p2_add<R>(NCX, rx), ny_ = p2_add<R>(NCY, ry);
            qxh[v] = nx_.h;
            qxl[v] = nx_.l;
            qyh[v] = ny_.h;
            qyl[v] = ny_.l;
            svx[v] = ux - om * ry;
            svy[v] = uy + om * rx;
        }
    } else {
        for (int v = tid; v < nv; v += T) {
            qxh[v] = xh[v];
            qxl[v] = xl[v];
            qyh[v] = yh[v];
            qyl[v] = yl[v];
            svx[v] = 0;
            svy[v] = 0;
        }
    }
    __syncthreads();

    // 6. direct forcing at the new element centroids, spreading masks (the
    //    near tiles of lattice step n + 2 are set by k_activate_next, off the
    //    membrane -> near chain, from the X^{n+1} this kernel stores)
    int32_t* mki = d.mki[p];
    R* mkf = static_cast<R*>(d.mkf[p]);
    const uint32_t* flag1 = d.nearflag[(n + 1) % 3];  // near tiles of lattice step n + 1
    for (int l0 = tid / K; l0 < nvq; l0 += Q) {
        const bool valid = l0 < nv;
        const int l = valid ? l0 : nv - 1;
        const int w = (l + 1 == nv) ? 0 : l + 1;
        const R dxn = p2_sub<R>(P2<R>{qxh[w], qxl[w]}, P2<R>{qxh[l], qxl[l]});
        const R dyn = p2_sub<R>(P2<R>{qyh[w], qyl[w]}, P2<R>{qyh[l], qyl[l]});
        const P2<R> CX = p2_add<R>(P2<R>{qxh[l], qxl[l]}, R(0.5) * dxn);
        const P2<R> CY = p2_add<R>(P2<R>{qyh[l], qyl[l]}, R(0.5) * dyn);
        const Spot<R> sc = spot_of<R>(CX, CY);
        Sample<R> o;
        sample_group<R, false, K, MLS>(d, sc, mf, lane4, B.x0, B.nxi, o, miss);
        if (!valid) continue;
        const R ds = sqrt(dxn * dxn + dyn * dyn);
        const R usx = R(0.5) * (svx[l] + svx[w]), usy = R(0.5) * (svy[l] + svy[w]);
        // centroid below the first or above the last row of fluid nodes: held by the wall
        const bool held = (sc.jy < 0) || (sc.jy > L.ny - 1) || (sc.jy == L.ny - 1 && sc.ay > R(0));
        R Fx = 0, Fy = 0;
        if (o.W > R(0) && !held) {
            const R rho = R(1) + o.drho;
            Fx = rho * (usx - o.u);
            Fy = rho * (usy - o.v);
        }
        const int g = (int)LBIB_IDX(off + l, NM, L.chk_status);
        if (lane4 == 0) {
            mki[g] = B.x0 + sc.ix;  // lattice column of the stencil origin
            mki[NM + g] = sc.jy;
            mkf[g] = sc.ax;
            mkf[NM + g] = sc.ay;
            mkf[2 * NM + g] = Fx * ds;
            mkf[3 * NM + g] = Fy * ds;
            diag[LBIB_FIELD_VX * NM + g] = svx[l];
            diag[LBIB_FIELD_VY * NM + g] = svy[l];
            diag[LBIB_FIELD_MX * NM + g] = CX.h + CX.l;
            diag[LBIB_FIELD_MY * NM + g] = CY.h + CY.l;
            diag[LBIB_FIELD_MFX * NM + g] = Fx;
            diag[LBIB_FIELD_MFY * NM + g] = Fy;
            diag[LBIB_FIELD_MDS * NM + g] = ds;
            len[l] = ds;  // X^n lengths are no longer needed
        }
        int tl[8];
        if (Fx != R(0) || Fy != R(0)) {
            // stencil nodes [ix - 1, ix + 2] x [jy - 1, jy + 2]: at most 2 x 2 tiles, one per lane
            const int i0 = max(0, sc.ix - 1), i1 = min(B.nxi - 1, sc.ix + 2);
            const int j0 = max(0, sc.jy - 1), j1 = min(L.ny - 1, sc.jy + 2);
            const int gl = g - B.moff;  // bit of the marker within its instance
            if (i0 <= i1 && j0 <= j1) {
                const int nt = box_tiles(L, B.x0 + i0, B.x0 + i1, j0, j1, 0, tl);
                for (int e = lane4; e < nt; e += K) {
                    const int t = tl[e];
                    if (!flag1[t]) miss |= 2u;
                    atomicOr(&d.mask[p][(size_t)t * d.mw + (gl >> 5)], 1u << (gl & 31));
                }
            }
        }
    }

    // 7. measures of X^{n+1}: FP64 shoelace area and centroid sums, FP32
    //    perimeter change (from the element lengths of step 6) and extent;
    //    store X^{n+1}
    __syncthreads();
    double a2n_[VL], cxs_[VL], cys_[VL];
    R dper_[VL];
#pragma unroll
    for (int j = 0; j < VL; ++j) {
        a2n_[j] = cxs_[j] = cys_[j] = 0.0;
        dper_[j] = R(0);
    }
    R xmin = R(3e38), xmax = R(-3e38), ymin = R(3e38), ymax = R(-3e38);
    for (int v0 = tid; v0 < nv; v0 += VLANES)
#pragma unroll
    for (int j = 0; j < VL; ++j) {
        const int v = v0 + j * T;
        if (v >= nv) break;
        dper_[j] += len[v] - sl0[v];  // perimeter change for delta p (Sec. 3.1)
        const int w = (v + 1 == nv) ? 0 : v + 1;
        const P2<R> X = P2<R>{qxh[v], qxl[v]}, Y = P2<R>{qyh[v], qyl[v]};
        const double Xd = p2_double<R>(X), Yd = p2_double<R>(Y);
        const double Xw = p2_double<R>(P2<R>{qxh[w], qxl[w]}), Yw = p2_double<R>(P2<R>{qyh[w], qyl[w]});
        const double cr = Xd * Yw - Xw * Yd;
        a2n_[j] += cr;
        cxs_[j] += (Xd + Xw) * cr;
        cys_[j] += (Yd + Yw) * cr;
        const R xa = X.h + X.l, ya = Y.h + Y.l;
        xmin = fmin(xmin, xa);
        xmax = fmax(xmax, xa);
        ymin = fmin(ymin, ya);
        ymax = fmax(ymax, ya);
        if (!isfinite(xa) || !isfinite(ya)) bad |= ST_DIVERGED;
        Pw[off + v] = Xd;
        Pw[NM + off + v] = Yd;
        Fw[off + v] = X.h;
        Fw[NM + off + v] = X.l;
        Fw[2 * NM + off + v] = Y.h;
        Fw[3 * NM + off + v] = Y.l;
    }
    int nb = 0;
    if (B.adhesive)
        for (int k = B.lig_off + tid; k < B.lig_off + B.nlig; k += T) nb += d.bound[k];
    // fused block reductions: sums over the virtual lanes, extent and bond
    // count (exact in any order) over the real warps
    double a2n, cxs, cys;
    R dper;
    {
        constexpr int W = T / 32;
        const int lane = tid & 31, wid = tid >> 5;
        R rv[5] = {(R)nb, xmin, ymin, -xmax, -ymax};
        rv[0] = warp_sum(rv[0]);
#pragma unroll
        for (int k = 1; k < 5; ++k) rv[k] = warp_min(rv[k]);
        double sv[VL][3];
        R pv[VL];
#pragma unroll
        for (int j = 0; j < VL; ++j) {
            sv[j][0] = warp_sum(a2n_[j]);
            sv[j][1] = warp_sum(cxs_[j]);
            sv[j][2] = warp_sum(cys_[j]);
            pv[j] = warp_sum(dper_[j]);
        }
        __syncthreads();
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < VL; ++j) {
#pragma unroll
                for (int k = 0; k < 3; ++k) dscr[k][j * W + wid] = sv[j][k];
                rscr[0][j * W + wid] = pv[j];
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) rscr[1 + k][wid] = rv[k];
        }
        __syncthreads();
        double tv[3] = {0.0, 0.0, 0.0};
        R tp = R(0);
        if (wid == 0) {
            constexpr int VW = VLANES / 32;
#pragma unroll
            for (int k = 0; k < 3; ++k) tv[k] = warp_sum(lane < VW ? dscr[k][lane] : 0.0);
            tp = warp_sum(lane < VW ? rscr[0][lane] : R(0));
            rv[0] = warp_sum(lane < W ? rscr[1][lane] : R(0));
#pragma unroll
            for (int k = 1; k < 5; ++k) rv[k] = warp_min(lane < W ? rscr[1 + k][lane] : R(3e38));
        }
        a2n = tv[0];
        cxs = tv[1];
        cys = tv[2];
        dper = tp;
        nb = (int)rv[0];
        xmin = rv[1];
        ymin = rv[2];
        xmax = -rv[3];
        ymax = -rv[4];
    }
    pdl_trigger();  // the force gather may be scheduled; it waits for this grid to complete
    if (miss & 1u) bad |= ST_READ_MISS;
    if (miss & 2u) bad |= ST_SPREAD_MISS;
    if (bad) atomicOr(d.status, bad);
    if (tid == 0) {
        double* bo = d.body_obs[(n + 1) & 1] + bi * BO_N;
        const double A = 0.5 * a2n;
        bo[BO_AREA] = A;
        bo[BO_DPERIM] = (double)dper;
        // 1 / (6 A): FP32 reciprocal refined by one FP64 Newton step (no FP64 division)
        const double s6 = 6.0 * A;
        double inv = (double)(1.0f / (float)s6);
        inv = inv * (2.0 - s6 * inv);
        bo[BO_CX] = cxs * inv;
        bo[BO_CY] = cys * inv;
        bo[BO_NBOUND] = nb;
        bo[BO_XMIN] = xmin;
        bo[BO_XMAX] = xmax;
        bo[BO_YMIN] = ymin;
        bo[BO_YMAX] = ymax;
        // the last block to finish empties the consumed list and advances the
        // step counter (every block has read both by now); the observables
        // record of the step is written by k_observables, off the membrane ->
        // near chain
        const uint32_t ticket = atomicAdd(d.ticket, 1u);
        if (ticket == (uint32_t)d.nbodies - 1u) {
            __threadfence();
            d.count[n % 3] = 0;  // list of lattice step n is consumed
            *d.ticket = 0u;
            *d.step = n + 1;
            __threadfence();
        }
    }
}

// lanes per interpolation point: as many as keep every body in one pass of
// a T-thread block
inline int lanes_for(int nv_max, int T)
{
    if (nv_max * 4 <= T) return 4;
    if (nv_max * 2 <= T) return 2;
    return 1;
}

template <typename R, int T, bool MLS>
cudaError_t configure_threads(int bytes)
{
    cudaError_t e =
        cudaFuncSetAttribute(k_lagrangian<R, 1, T, MLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_lagrangian<R, 2, T, MLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_lagrangian<R, 4, T, MLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

// every instantiation of one transfer kernel for the smem the bodies need
template <bool MLS>
cudaError_t configure_transfer(int prec, int bytes)
{
    if (prec == PREC_F64) {
        cudaError_t e = configure_threads<double, 256, MLS>(bytes);
        return (e == cudaSuccess) ? configure_threads<double, 512, MLS>(bytes) : e;
    }
    cudaError_t e = configure_threads<float, 256, MLS>(bytes);
    return (e == cudaSuccess) ? configure_threads<float, 512, MLS>(bytes) : e;
}

template <typename R, int T, bool MLS>
cudaError_t launch_threads(const Dev& d, int parity, size_t bytes, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(d.nbodies);
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = d.chain_priority;
    cfg.attrs = attr;
    cfg.numAttrs = d.chain_priority ? 1 : 0;
    switch (lanes_for(d.nv_max, T)) {
    case 4: return cudaLaunchKernelEx(&cfg, k_lagrangian<R, 4, T, MLS>, d, parity);
    case 2: return cudaLaunchKernelEx(&cfg, k_lagrangian<R, 2, T, MLS>, d, parity);
    default: return cudaLaunchKernelEx(&cfg, k_lagrangian<R, 1, T, MLS>, d, parity);
    }
}

// the launch of one transfer kernel in the context's shape
template <bool MLS>
cudaError_t launch_transfer(const Dev& d, int prec, int parity, size_t bytes, cudaStream_t s)
{
    if (d.lag_threads == 256)
        return (prec == PREC_F64) ? launch_threads<double, 256, MLS>(d, parity, bytes, s)
                                  : launch_threads<float, 256, MLS>(d, parity, bytes, s);
    return (prec == PREC_F64) ? launch_threads<double, 512, MLS>(d, parity, bytes, s)
                              : launch_threads<float, 512, MLS>(d, parity, bytes, s);
}

// MLS instantiations (lbib_lag_mls.cu)
cudaError_t configure_kernels_mls(int prec, int bytes);
cudaError_t launch_lagrangian_mls(const Dev& d, int prec, int parity, size_t bytes, cudaStream_t s);

}  // namespace lbib
