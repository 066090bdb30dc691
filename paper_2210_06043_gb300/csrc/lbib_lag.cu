// lbib_lag.cu -- host side of the Lagrangian update and the instantiations
// of its kernel (lbib_lag_kernel.cuh) for the Peskin transfer.
#include "lbib_lag_kernel.cuh"

namespace lbib {

// Observables record of the step the membrane update has just completed
// (Sec. 3.1): for every instance with membranes, delta p of its first cell,
// the distance r between the area centroids of its first cell and first
// particle, and N_L = bonds engaged / bonds engaged at t = 0, from the per-body
// measures the membrane kernel left in body_obs.  One block; launched after
// the membrane kernel on a branch of its own, so the lattice update of the
// next step does not wait for it.  The record's status is the status word
// when the record is written.
__global__ void k_observables(Dev d)
{
    pdl_wait();
    const int64_t n1 = *d.step;  // advanced by the membrane kernel
    const double* all = d.body_obs[n1 & 1];
    const double nan = __longlong_as_double(0x7ff8000000000000ULL);
    for (int i = threadIdx.x; i < d.ninst; i += blockDim.x) {
        const InstConst& I = d.inst[i];
        if (I.nbodies == 0) continue;
        lbib_obs r;
        r.step = n1;
        r.t_star = (double)n1 * d.uscale;
        r.delta_p = nan;
        r.r = nan;
        r.n_l = nan;
        const int fc = I.first_cell, fp = I.first_particle;
        if (fc >= 0) r.delta_p = all[fc * BO_N + BO_DPERIM] * d.body[fc].inv_P0;
        if (fc >= 0 && fp >= 0) {
            const double dx = all[fc * BO_N + BO_CX] - all[fp * BO_N + BO_CX];
            const double dy = all[fc * BO_N + BO_CY] - all[fp * BO_N + BO_CY];
            const double r2 = dx * dx + dy * dy;
            // FP32 square root refined by one FP64 Newton correction
            const float sq = sqrtf((float)r2);
            r.r = (sq > 0.f) ? (double)sq + (r2 - (double)sq * (double)sq) * (0.5 / (double)sq) : 0.0;
        }
        int nbt = 0, nl0 = 0;
        for (int b = I.body0; b < I.body0 + I.nbodies; ++b)
            if (d.body[b].adhesive) {
                nbt += (int)all[b * BO_N + BO_NBOUND];
                nl0 += d.body[b].nl0;
            }
        if (nl0 > 0) r.n_l = (double)nbt / (double)nl0;
        r.n_bound = nbt;
        r.status = (int32_t)atomicOr(d.status, 0u);
        d.ring[(size_t)i * d.ring_cap + n1 % d.ring_cap] = r;
    }
}

cudaError_t launch_observables(const Dev& d, cudaStream_t s, bool urgent, bool pdl)
{
    // urgent: at the chain's priority (on the chain, queued behind the bulk
    // lattice blocks it would finish after them and hold up the end of the step)
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(128);
    cfg.stream = s;
    int na = 0;
    if (urgent && d.chain_priority) {
        attr[na].id = cudaLaunchAttributePriority;
        attr[na++].val.priority = d.chain_priority;
    }
    if (pdl) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na++].val.programmaticStreamSerializationAllowed = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, k_observables, d);
}

// Near tiles of lattice step m + 1, m = *d.step the step the membrane update
// has just reached, from the X^m it stored: every stencil the membrane update
// of step m + 1 reads (vertices, probes, the new element centroids) and the
// spreading of step m + 1 writes lies, per element e, within the box of
// half-width reach_e = max(l_e / 2, 1.2) + 2 around its centroid (vertex /
// probe offset plus the stencil), widened by a quarter node for two steps of
// motion (a stable lattice flow moves a marker by less than 0.1 dx per step;
// a larger move shows up as a read or spread miss).  Every act_stride-th
// element covers itself and the following ones up to the next activating
// element, at their current distances; the box is taken around the stencil
// origin (floor(x), floor(y - 1/2)), one node more.  One block per membrane,
// a thread per activating element; unflagged tiles are claimed with an
// exchange and appended to the list.  It runs on a branch of its own after
// the membrane kernel: the tiles are first needed by the next step's graph.
__global__ void __launch_bounds__(256) k_activate_next(Dev d)
{
    const Lattice& L = d.L;
    const int64_t m = *d.step;
    const int64_t s2 = m + 1;
    uint32_t* flag = d.nearflag[s2 % 3];
    const int c = (int)(s2 % 3);
    const BodyConst& B = d.body[blockIdx.x];
    const double* PX = d.pos[m & 1] + B.off;
    const double* PY = d.pos[m & 1] + d.nmark + B.off;
    const int nv = B.nv, stride = d.act_stride;
    for (int l = threadIdx.x; l < nv; l += blockDim.x) {
        if (l % stride != 0 && l != nv - 1) continue;
        const int cover = (l % stride == 0) ? min(stride, nv - l) : 1;
        const int w = (l + 1 == nv) ? 0 : l + 1;
        const double cx = PX[l] + 0.5 * (PX[w] - PX[l]), cy = PY[l] + 0.5 * (PY[w] - PY[l]);
        double reach = 0.0;
        for (int j = 0; j < cover; ++j) {
            const int e = l + j, e1 = (e + 1 == nv) ? 0 : e + 1;
            const double ex = PX[e1] - PX[e], ey = PY[e1] - PY[e];
            const double cxe = PX[e] + 0.5 * ex, cye = PY[e] + 0.5 * ey;
            const double own = fmax(0.5 * sqrt(ex * ex + ey * ey), 1.2) + 2.0;
            reach = fmax(reach, fmax(fabs(cxe - cx), fabs(cye - cy)) + own);
        }
        const int ra = (int)ceil(reach + 0.25) + 1;
        const int ix = (int)floor(cx), jy = (int)floor(cy - 0.5);
        const int i0 = B.x0 + max(0, ix - ra), i1 = B.x0 + min(B.nxi - 1, ix + ra);
        const int j0 = max(0, jy - ra), j1 = min(L.ny - 1, jy + ra);
        if (i0 > i1 || j0 > j1) continue;
        for (int ty = j0 / TY; ty <= j1 / TY; ++ty)
            for (int tx = i0 / TX; tx <= i1 / TX; ++tx) {
                const int t = (int)LBIB_IDX(ty * L.ntx + tx, L.ntiles, L.chk_status);
                if (flag[t] == 0u && atomicExch(&flag[t], 1u) == 0u) {
                    const int pos = atomicAdd(&d.count[c], 1);
                    if (pos < d.list_cap) d.list[c][pos] = t;
                    else atomicOr(d.status, ST_LIST_OVERFLOW);
                }
            }
    }
}

cudaError_t launch_activate_next(const Dev& d, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(d.nbodies);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = d.chain_priority;
    cfg.attrs = attr;
    cfg.numAttrs = d.chain_priority ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_activate_next, d);
}

size_t lagrangian_smem_bytes(int prec, int nv_max)
{
    size_t r = (prec == PREC_F64) ? sizeof(double) : sizeof(float);
    return (size_t)nv_max * 33 * r;
}

cudaError_t configure_kernels(int prec, int nv_max)
{
    const int bytes = (int)lagrangian_smem_bytes(prec, nv_max);
    cudaError_t e = configure_transfer<false>(prec, bytes);
    return (e == cudaSuccess) ? configure_kernels_mls(prec, bytes) : e;
}

cudaError_t launch_lagrangian(const Dev& d, int prec, int parity, cudaStream_t s)
{
    const size_t bytes = lagrangian_smem_bytes(prec, d.nv_max);
    if (d.L.transfer == LBIB_TRANSFER_MLS) return launch_lagrangian_mls(d, prec, parity, bytes, s);
    return launch_transfer<false>(d, prec, parity, bytes, s);
}

}  // namespace lbib
