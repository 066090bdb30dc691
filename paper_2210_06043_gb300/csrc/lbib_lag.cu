// lbib_lag.cu -- the Lagrangian update: one thread block per membrane.
//
// Lagrangian step n (after the lattice step n has written rho^n - 1 and u^n on
// its near tiles), for the block's body, in this order:
//   1. chain geometry at X^n: edges, lengths, outward element normals, vertex
//      normals and signed turning angles; shoelace area in FP64;
//   2. fluid velocity at the vertices (Sec. 2.9) with the truncated Peskin
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
//      the tiles their stencils touch; tiles within r_act of the new
//      centroids are scheduled as near for lattice step n + 2;
//   7. area, perimeter, centroid and extent of X^{n+1}; the last block to
//      finish writes the observables record of step n + 1 and advances n.
#include <cuda_runtime.h>

#include "lbib_device.cuh"

namespace lbib {

template <typename R>
struct Sample {
    R u, v, ux, uy, vx, vy, rho, W;
};

// Truncated-stencil velocity (and optionally its gradient) and renormalised
// density at (X, Y) from the near-tile output of lattice step m.
template <typename R>
__device__ __forceinline__ void sample(const Dev& d, double X, double Y, int32_t m, bool grad, Sample<R>& o,
                                       uint32_t& miss)
{
    const Lattice& L = d.L;
    const R* ux = static_cast<const R*>(d.ux);
    const R* uy = static_cast<const R*>(d.uy);
    const R* dr = static_cast<const R*>(d.drho);
    int i0 = (int)floor(X) - 1, j0 = (int)floor(Y - 0.5) - 1;
    R W = 0, Nu = 0, Nv = 0, Nr = 0, Nux = 0, Nuy = 0, Nvx = 0, Nvy = 0;
    for (int jj = 0; jj < 4; ++jj) {
        int j = j0 + jj;
        if (j < 0 || j >= L.ny) continue;
        R ry = (R)(Y - (j + 0.5));
        R py = peskin<R>(ry), dpy = grad ? peskin_d<R>(ry) : R(0);
        for (int ii = 0; ii < 4; ++ii) {
            int i = i0 + ii;
            if (i < 0 || i >= L.nx) continue;
            R rx = (R)(X - i);
            R px = peskin<R>(rx);
            if (d.fresh[tile_of(L, i, j)] != m) miss = 1u;
            int idx = j * L.nxp + i;
            R a = ux[idx], b = uy[idx];
            R w = px * py;
            W += w;
            Nu += a * w;
            Nv += b * w;
            Nr += dr[idx] * w;
            if (grad) {
                R dpx = peskin_d<R>(rx);
                Nux += a * dpx * py;
                Nuy += a * px * dpy;
                Nvx += b * dpx * py;
                Nvy += b * px * dpy;
            }
        }
    }
    o.u = Nu;
    o.v = Nv;
    o.ux = Nux;
    o.uy = Nuy;
    o.vx = Nvx;
    o.vy = Nvy;
    o.W = W;
    o.rho = (W > R(0)) ? R(1) + Nr / W : R(1);
}

template <typename R>
__global__ void __launch_bounds__(LAG_THREADS) k_lagrangian(Dev d, int p)
{
    const Lattice& L = d.L;
    const int bi = blockIdx.x;
    const BodyConst& B = d.body[bi];
    const int nv = B.nv, off = B.off, NM = d.nmark, tid = threadIdx.x, T = blockDim.x;
    const int64_t n = *d.step;
    const int32_t mf = (int32_t)n;  // lattice step whose rho/u the interpolation reads
    const double* __restrict__ Pn = d.pos[n & 1];
    double* Pw = d.pos[(n + 1) & 1];  // X^{n-1} on entry, X^{n+1} on exit
    const R* l0 = static_cast<const R*>(d.l0) + off;
    const R* th0 = static_cast<const R*>(d.th0) + off;
    R* diag = static_cast<R*>(d.diag);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sx = reinterpret_cast<double*>(smem_raw);
    double* sy = sx + nv;
    double* qx = sy + nv;  // X^{n+1}
    double* qy = qx + nv;
    R* ex = reinterpret_cast<R*>(qy + nv);
    R* ey = ex + nv;
    R* len = ey + nv;
    R* nlx = len + nv;
    R* nly = nlx + nv;
    R* vnx = nly + nv;
    R* vny = vnx + nv;
    R* th = vny + nv;
    R* uvx = th + nv;
    R* uvy = uvx + nv;
    R* eax = uvy + nv;
    R* eay = eax + nv;
    R* ewx = eay + nv;
    R* ewy = ewx + nv;
    R* ehx = ewy + nv;
    R* ehy = ehx + nv;
    R* fpx = ehy + nv;
    R* fpy = fpx + nv;
    R* ftx = fpy + nv;
    R* fty = ftx + nv;
    R* svx = fty + nv;
    R* svy = svx + nv;
    __shared__ double dscr[32];
    __shared__ R rscr[32];
    __shared__ double rig[4];
    uint32_t miss = 0u, bad = 0u;

    // 1. geometry at X^n
    for (int v = tid; v < nv; v += T) {
        sx[v] = Pn[off + v];
        sy[v] = Pn[NM + off + v];
    }
    __syncthreads();
    double a2 = 0.0;
    for (int l = tid; l < nv; l += T) {
        int w = (l + 1 == nv) ? 0 : l + 1;
        R dx = (R)(sx[w] - sx[l]), dy = (R)(sy[w] - sy[l]);
        R ll = sqrt(dx * dx + dy * dy);
        ex[l] = dx;
        ey[l] = dy;
        len[l] = ll;
        nlx[l] = dy / ll;
        nly[l] = -dx / ll;
        a2 += sx[l] * sy[w] - sx[w] * sy[l];
    }
    const double area = 0.5 * block_sum<double>(a2, dscr);  // FP64 area reduction (Eq. 11)
    for (int v = tid; v < nv; v += T) {
        int lm = (v == 0) ? nv - 1 : v - 1;
        th[v] = atan2(ex[lm] * ey[v] - ey[lm] * ex[v], ex[lm] * ex[v] + ey[lm] * ey[v]);
        R sxn = nlx[lm] + nlx[v], syn = nly[lm] + nly[v];
        R s = sqrt(sxn * sxn + syn * syn);
        vnx[v] = sxn / s;
        vny[v] = syn / s;
    }
    __syncthreads();

    // 2. fluid velocity at the vertices; tractions from the probes (Eqs. 14-15)
    for (int v = tid; v < nv; v += T) {
        Sample<R> o;
        sample<R>(d, sx[v], sy[v], mf, false, o, miss);
        uvx[v] = o.u;
        uvy[v] = o.v;
    }
    const R nu = (R)L.nu;
    for (int l = tid; l < nv; l += T) {
        int w = (l + 1 == nv) ? 0 : l + 1;
        double px = 0.5 * (sx[l] + sx[w]) + d.probe * (double)nlx[l];
        double py = 0.5 * (sy[l] + sy[w]) + d.probe * (double)nly[l];
        py = fmin(fmax(py, 0.0), (double)L.ny);
        Sample<R> o;
        sample<R>(d, px, py, mf, true, o, miss);
        R fx = 0, fy = 0;
        if (o.W > R(0)) {
            R pr = (o.rho - R(1)) / R(3);
            R mu = o.rho * nu;
            R txx = R(2) * mu * o.ux, txy = mu * (o.uy + o.vx), tyy = R(2) * mu * o.vy;
            fx = (-pr * nlx[l] + txx * nlx[l] + txy * nly[l]) * len[l];
            fy = (-pr * nly[l] + txy * nlx[l] + tyy * nly[l]) * len[l];
        }
        ehx[l] = fx;
        ehy[l] = fy;
        // Eq. 11: -k_a (1 - A / A_0) p_ref n^- l with n^- = -n
        R fa = (B.motion == LBIB_DEFORMABLE) ? (R)(B.ka * (1.0 - area / B.A0) / 3.0) * len[l] : R(0);
        eax[l] = fa * nlx[l];
        eay[l] = fa * nly[l];
        ewx[l] = 0;
        ewy[l] = 0;
    }
    __syncthreads();

    // 3. ligand-receptor kinetics (one draw per site and step) and Eq. 13
    if (B.adhesive) {
        const R* lt = static_cast<const R*>(d.lig_t);
        R* mg = static_cast<R*>(d.margin);
        const R Pf = (R)B.Pf;
        for (int k = B.lig_off + tid; k < B.lig_off + B.nlig; k += T) {
            if (B.motion == LBIB_FIXED) break;
            int l = d.lig_el[k] - off, w = (l + 1 == nv) ? 0 : l + 1;
            double t = (double)lt[k];
            double px = sx[l] + t * (sx[w] - sx[l]), py = sy[l] + t * (sy[w] - sy[l]);
            R u = (R)bond_draw(d.seed, n, (uint32_t)k);
            if (d.bound[k]) {
                double ddx = px - d.anchor[k], ddy = py - d.anchor[d.nlig + k];
                R yl = (R)sqrt(ddx * ddx + ddy * ddy);
                R dy = yl - (R)B.yeq;
                R Pr = R(1) - exp(-(R)B.kr0_dt * exp((R)B.xi * dy * dy));
                mg[k] = fabs(u - Pr);
                if (u < Pr) d.bound[k] = 0;
            } else {
                double gap = fmin(py, (double)L.ny - py);
                if (gap < B.ycr) {
                    mg[k] = fabs(u - Pf);
                    if (u < Pf) {
                        d.bound[k] = 1;
                        d.anchor[k] = px;
                        d.anchor[d.nlig + k] = (py < (double)L.ny - py) ? 0.0 : (double)L.ny;
                    }
                }
            }
        }
        __syncthreads();
        if (!B.sigma_inf) {
            const R sig = (R)B.sigma;
            for (int l = tid; l < nv; l += T) {
                int w = (l + 1 == nv) ? 0 : l + 1;
                R s = 0;
                for (int k = d.site_off[off + l]; k < d.site_off[off + l + 1]; ++k) {
                    if (!d.bound[k]) continue;
                    double t = (double)lt[k];
                    double px = sx[l] + t * (sx[w] - sx[l]), py = sy[l] + t * (sy[w] - sy[l]);
                    double ddx = px - d.anchor[k], ddy = py - d.anchor[d.nlig + k];
                    R yl = (R)sqrt(ddx * ddx + ddy * ddy);
                    s += sig * (yl - (R)B.yeq);
                }
                ewx[l] = s * nlx[l];
                ewy[l] = s * nly[l];
            }
        }
    }

    // repulsion (Eq. 12) from the vertices of every other body within the cut-off
    const double* ext = d.body_obs[n & 1];
    const R c0 = R(1e-4) / (R(8) * sqrt(R(2)));
    for (int v = tid; v < nv; v += T) {
        R ax = 0, ay = 0;
        for (int o = 0; o < d.nbodies; ++o) {
            if (o == bi) continue;
            const double* eo = ext + o * BO_N;
            if (sx[v] < eo[BO_XMIN] - d.dcut || sx[v] > eo[BO_XMAX] + d.dcut || sy[v] < eo[BO_YMIN] - d.dcut ||
                sy[v] > eo[BO_YMAX] + d.dcut)
                continue;
            const BodyConst& C = d.body[o];
            for (int w = 0; w < C.nv; ++w) {
                R ddx = (R)(sx[v] - Pn[C.off + w]), ddy = (R)(sy[v] - Pn[NM + C.off + w]);
                R dd = sqrt(ddx * ddx + ddy * ddy);
                if (dd < (R)d.dcut) {
                    R mag = c0 * sqrt(R(1) / (dd * dd * dd * dd * dd));
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
    for (int v = tid; v < nv; v += T) {
        int lm = (v == 0) ? nv - 1 : v - 1, w = (v + 1 == nv) ? 0 : v + 1;
        R fsx = 0, fsy = 0, fbx = 0, fby = 0;
        if (deform) {
            // Eq. 8: element lm pulls v along e_lm, element v along -e_v
            R cl = -ks * (len[lm] - l0[lm]) / len[lm];
            R cr = -ks * (len[v] - l0[v]) / len[v];
            fsx = cl * ex[lm] - cr * ex[v];
            fsy = cl * ey[lm] - cr * ey[v];
            // Eq. 10: triples centred at lm (v on its right), v, and w (v on its left)
            int lmm = (lm == 0) ? nv - 1 : lm - 1;
            R kl = kb * (th[lm] - th0[lm]);
            R kc = kb * (th[v] - th0[v]);
            R kr = kb * (th[w] - th0[w]);
            R cR = kl * len[lm] / (len[lmm] + len[lm]);
            R cL = kr * len[v] / (len[v] + len[w]);
            fbx = cR * vnx[lm] - kc * vnx[v] + cL * vnx[w];
            fby = cR * vny[lm] - kc * vny[v] + cL * vny[w];
        }
        R fax = R(0.5) * (eax[lm] + eax[v]), fay = R(0.5) * (eay[lm] + eay[v]);
        R fwx = R(0.5) * (ewx[lm] + ewx[v]), fwy = R(0.5) * (ewy[lm] + ewy[v]);
        R fhx = R(0.5) * (ehx[lm] + ehx[v]), fhy = R(0.5) * (ehy[lm] + ehy[v]);
        R tx = fsx + fbx + fax + fpx[v] + fwx + fhx;
        R ty = fsy + fby + fay + fpy[v] + fwy + fhy;
        ftx[v] = tx;
        fty[v] = ty;
        int g = off + v;
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
            double xn = sx[v] + (double)uvx[v] + (double)(R(0.5) * ftx[v] / mv);
            double yn = sy[v] + (double)uvy[v] + (double)(R(0.5) * fty[v] / mv);
            double xp = Pw[off + v], yp = Pw[NM + off + v];  // X^{n-1}
            svx[v] = (R)(1.5 * xn - 2.0 * sx[v] + 0.5 * xp);
            svy[v] = (R)(1.5 * yn - 2.0 * sy[v] + 0.5 * yp);
            qx[v] = xn;
            qy[v] = yn;
        }
    } else if (B.motion == LBIB_RIGID) {
        double* rs = d.rigid + bi * RG_N;
        const double xc = rs[RG_XC], yc = rs[RG_YC];
        R sfx = 0, sfy = 0, smz = 0;
        for (int v = tid; v < nv; v += T) {
            sfx += ftx[v];
            sfy += fty[v];
            smz += (R)(sx[v] - xc) * fty[v] - (R)(sy[v] - yc) * ftx[v];
        }
        sfx = block_sum<R>(sfx, rscr);
        sfy = block_sum<R>(sfy, rscr);
        smz = block_sum<R>(smz, rscr);
        if (tid == 0) {
            // Eq. 19: u = 2/3 (2 u(t - dt) - 1/2 u(t - 2 dt) + du/dt dt), likewise omega
            double ux = (2.0 / 3.0) * (2.0 * rs[RG_U1X] - 0.5 * rs[RG_U2X] + (double)sfx / B.mass);
            double uy = (2.0 / 3.0) * (2.0 * rs[RG_U1Y] - 0.5 * rs[RG_U2Y] + (double)sfy / B.mass);
            double om = (2.0 / 3.0) * (2.0 * rs[RG_W1] - 0.5 * rs[RG_W2] + (double)smz / B.inertia);
            rs[RG_U2X] = rs[RG_U1X];
            rs[RG_U1X] = ux;
            rs[RG_U2Y] = rs[RG_U1Y];
            rs[RG_U1Y] = uy;
            rs[RG_W2] = rs[RG_W1];
            rs[RG_W1] = om;
            rs[RG_XC] = xc + ux;
            rs[RG_YC] = yc + uy;
            rs[RG_ANG] += om;
            rig[0] = ux;
            rig[1] = uy;
            rig[2] = om;
            rig[3] = rs[RG_ANG];
        }
        __syncthreads();
        const double ux = rig[0], uy = rig[1], om = rig[2], cs = cos(rig[3]), sn = sin(rig[3]);
        const double ncx = rs[RG_XC], ncy = rs[RG_YC];
        for (int v = tid; v < nv; v += T) {
            double rx = cs * d.rref[off + v] - sn * d.rref[NM + off + v];
            double ry = sn * d.rref[off + v] + cs * d.rref[NM + off + v];
            qx[v] = ncx + rx;
            qy[v] = ncy + ry;
            svx[v] = (R)(ux - om * ry);
            svy[v] = (R)(uy + om * rx);
        }
    } else {
        for (int v = tid; v < nv; v += T) {
            qx[v] = sx[v];
            qy[v] = sy[v];
            svx[v] = 0;
            svy[v] = 0;
        }
    }
    __syncthreads();

    // 6. direct forcing at the new element centroids, spreading masks, activation
    R* mk = static_cast<R*>(d.mk[p]);
    const int64_t n2 = n + 2;
    uint32_t* flag2 = d.nearflag[n2 & 1];
    const int c2 = (int)(n2 % 3);
    double per = 0.0, cxs = 0.0, cys = 0.0, a2n = 0.0;
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int l = tid; l < nv; l += T) {
        int w = (l + 1 == nv) ? 0 : l + 1;
        double cx = 0.5 * (qx[l] + qx[w]), cy = 0.5 * (qy[l] + qy[w]);
        double dxn = qx[w] - qx[l], dyn = qy[w] - qy[l];
        double ds = sqrt(dxn * dxn + dyn * dyn);
        R usx = R(0.5) * (svx[l] + svx[w]), usy = R(0.5) * (svy[l] + svy[w]);
        Sample<R> o;
        sample<R>(d, cx, cy, mf, false, o, miss);
        bool held = (cy < 0.5) || (cy > (double)L.ny - 0.5);
        R Fx = 0, Fy = 0;
        if (o.W > R(0) && !held) {
            Fx = o.rho * (usx - o.u);
            Fy = o.rho * (usy - o.v);
        }
        const int g = off + l;
        mk[g] = (R)cx;
        mk[NM + g] = (R)cy;
        mk[2 * NM + g] = Fx * (R)ds;
        mk[3 * NM + g] = Fy * (R)ds;
        diag[LBIB_FIELD_VX * NM + g] = svx[l];
        diag[LBIB_FIELD_VY * NM + g] = svy[l];
        diag[LBIB_FIELD_MX * NM + g] = (R)cx;
        diag[LBIB_FIELD_MY * NM + g] = (R)cy;
        diag[LBIB_FIELD_MFX * NM + g] = Fx;
        diag[LBIB_FIELD_MFY * NM + g] = Fy;
        diag[LBIB_FIELD_MDS * NM + g] = (R)ds;
        if (Fx != R(0) || Fy != R(0)) {
            int i0 = max(0, (int)floor(cx) - 1), i1 = min(L.nx - 1, (int)floor(cx) + 2);
            int j0 = max(0, (int)floor(cy - 0.5) - 1), j1 = min(L.ny - 1, (int)floor(cy - 0.5) + 2);
            for (int ty = j0 / TY; ty <= j1 / TY && i0 <= i1; ++ty)
                for (int tx = i0 / TX; tx <= i1 / TX; ++tx) {
                    int t = ty * L.ntx + tx;
                    if (!d.nearflag[p][t]) miss |= 2u;
                    atomicOr(&d.mask[p][(size_t)t * d.mw + (g >> 5)], 1u << (g & 31));
                }
        }
        {
            int i0 = max(0, (int)floor(cx - d.r_act)), i1 = min(L.nx - 1, (int)floor(cx + d.r_act) + 1);
            int j0 = max(0, (int)floor(cy - 0.5 - d.r_act)), j1 = min(L.ny - 1, (int)floor(cy - 0.5 + d.r_act) + 1);
            for (int ty = j0 / TY; ty <= j1 / TY && i0 <= i1; ++ty)
                for (int tx = i0 / TX; tx <= i1 / TX; ++tx) {
                    int t = ty * L.ntx + tx;
                    if (flag2[t] == 0u && atomicExch(&flag2[t], 1u) == 0u) {
                        int pos = atomicAdd(&d.count[c2], 1);
                        if (pos < d.list_cap) d.list[c2][pos] = t;
                        else bad |= ST_LIST_OVERFLOW;
                    }
                }
        }
        // 7. measures of X^{n+1}
        double cr = qx[l] * qy[w] - qx[w] * qy[l];
        a2n += cr;
        per += ds;
        cxs += (qx[l] + qx[w]) * cr;
        cys += (qy[l] + qy[w]) * cr;
        if (!isfinite(qx[l]) || !isfinite(qy[l])) bad |= ST_DIVERGED;
    }
    for (int v = tid; v < nv; v += T) {
        xmin = fmin(xmin, qx[v]);
        xmax = fmax(xmax, qx[v]);
        ymin = fmin(ymin, qy[v]);
        ymax = fmax(ymax, qy[v]);
        Pw[off + v] = qx[v];
        Pw[NM + off + v] = qy[v];
    }
    int nb = 0;
    if (B.adhesive)
        for (int k = B.lig_off + tid; k < B.lig_off + B.nlig; k += T) nb += d.bound[k];
    a2n = block_sum<double>(a2n, dscr);
    per = block_sum<double>(per, dscr);
    cxs = block_sum<double>(cxs, dscr);
    cys = block_sum<double>(cys, dscr);
    double nbd = block_sum<double>((double)nb, dscr);
    xmin = block_min<double>(xmin, dscr);
    xmax = block_max<double>(xmax, dscr);
    ymin = block_min<double>(ymin, dscr);
    ymax = block_max<double>(ymax, dscr);
    if (miss & 1u) bad |= ST_READ_MISS;
    if (miss & 2u) bad |= ST_SPREAD_MISS;
    if (bad) atomicOr(d.status, bad);
    if (tid == 0) {
        double* bo = d.body_obs[(n + 1) & 1] + bi * BO_N;
        double A = 0.5 * a2n;
        bo[BO_AREA] = A;
        bo[BO_PERIM] = per;
        bo[BO_CX] = cxs / (6.0 * A);
        bo[BO_CY] = cys / (6.0 * A);
        bo[BO_NBOUND] = nbd;
        bo[BO_XMIN] = xmin;
        bo[BO_XMAX] = xmax;
        bo[BO_YMIN] = ymin;
        bo[BO_YMAX] = ymax;
        __threadfence();
        uint32_t ticket = atomicAdd(d.ticket, 1u);
        if (ticket == (uint32_t)d.nbodies - 1u) {
            // last block: observables of step n + 1 (Sec. 3.1), then advance n
            __threadfence();
            const double* all = d.body_obs[(n + 1) & 1];
            lbib_obs r;
            r.step = n + 1;
            r.t_star = (double)(n + 1) * d.uscale;
            double nan = __longlong_as_double(0x7ff8000000000000ULL);
            r.delta_p = nan;
            r.r = nan;
            r.n_l = nan;
            if (d.first_cell >= 0) {
                const BodyConst& Cc = d.body[d.first_cell];
                r.delta_p = (all[d.first_cell * BO_N + BO_PERIM] - Cc.P0) / Cc.P0;
            }
            if (d.first_cell >= 0 && d.first_particle >= 0) {
                double dx = all[d.first_cell * BO_N + BO_CX] - all[d.first_particle * BO_N + BO_CX];
                double dy = all[d.first_cell * BO_N + BO_CY] - all[d.first_particle * BO_N + BO_CY];
                r.r = sqrt(dx * dx + dy * dy);
            }
            int nbt = 0, nl0 = 0;
            for (int b = 0; b < d.nbodies; ++b)
                if (d.body[b].adhesive) {
                    nbt += (int)all[b * BO_N + BO_NBOUND];
                    nl0 += d.body[b].nl0;
                }
            if (nl0 > 0) r.n_l = (double)nbt / (double)nl0;
            r.n_bound = nbt;
            r.status = (int32_t)atomicOr(d.status, 0u);
            d.ring[(n + 1) % d.ring_cap] = r;
            d.count[n % 3] = 0;  // list of lattice step n is consumed
            *d.ticket = 0u;
            *d.step = n + 1;
            __threadfence();
        }
    }
}

size_t lagrangian_smem_bytes(int prec, int nv_max)
{
    size_t r = (prec == PREC_F64) ? sizeof(double) : sizeof(float);
    return (size_t)nv_max * (4 * sizeof(double) + 22 * r);
}

cudaError_t configure_kernels(int prec, int nv_max)
{
    size_t bytes = lagrangian_smem_bytes(prec, nv_max);
    if (prec == PREC_F64)
        return cudaFuncSetAttribute(k_lagrangian<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaFuncSetAttribute(k_lagrangian<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_lagrangian(const Dev& d, int prec, int parity, cudaStream_t s)
{
    size_t bytes = lagrangian_smem_bytes(prec, d.nv_max);
    if (prec == PREC_F64) k_lagrangian<double><<<d.nbodies, LAG_THREADS, bytes, s>>>(d, parity);
    else k_lagrangian<float><<<d.nbodies, LAG_THREADS, bytes, s>>>(d, parity);
    return cudaGetLastError();
}

}  // namespace lbib
