// lbib_internal.cuh -- device data layout and device helpers of the capillary
// solver (internal to the library; the public boundary is include/lbib.h).
//
// Layout in HBM
//   populations  Store f[2][9][ny][nxp], stored as deviations f_i - w_i from the
//                rest weights (w_i rho_ref, rho_ref = 1), double-buffered; the
//                lattice step m reads f[m & 1] and writes f[(m + 1) & 1].
//   tiles        32 x 4 nodes; one thread block of the lattice kernels updates
//                one tile.  Tiles within R_act of a membrane are "near": their
//                update adds the spread immersed-boundary force and writes
//                rho - 1 and u for the Lagrangian kernel; all others are "bulk".
//   markers      element centroids with their direct force times ds,
//                double-buffered by the parity of the lattice step that
//                consumes them, each stored as the integer origin of its 4 x 4
//                stencil plus an exact fractional offset (so FP32 kernel
//                weights do not lose the ~1e-5 dx that FP32 coordinates near
//                x ~ 1000 would); per near tile a bit mask of the markers whose
//                stencil touches it (ascending marker order = the order in
//                which the forces are summed).
//   bodies       vertex positions in FP64 in global memory (per-step
//                displacements at Re = 1e-2 are ~1e-5 dx, below FP32
//                resolution at channel coordinates), carried inside the
//                Lagrangian kernel as float-float pairs (hi + lo, ~48 bits)
//                so that no FP64 operation sits on its dependency chains
//                (FP64 latency on this part is ~10^2 cycles per dependent
//                operation); forces in the compute precision; the area and
//                centroid reductions in FP64.
#pragma once

#include <cstdint>

#include "../../include/lbib.h"

namespace lbib {

constexpr int TX = 32;            // tile width (nodes along x) = one warp
constexpr int TY = 4;             // tile height
constexpr int MAX_BODIES = 16;
constexpr int MAX_NV = 1024;      // vertices per body
constexpr int LAG_THREADS = 512;  // default threads of the Lagrangian kernel's blocks (256 or 512)
constexpr int ACT_STRIDE = 4;     // default: near-tile activation from every 4th element centroid
constexpr int NDIAG = LBIB_FIELD_COUNT;

// device status bits (host maps them to lbib_status)
enum : uint32_t {
    ST_DIVERGED = 1u,       // non-finite or non-positive density/velocity/positions
    ST_READ_MISS = 2u,      // an interpolation stencil reached a tile not updated as near
    ST_SPREAD_MISS = 4u,    // a spreading stencil reached a tile not scheduled as near
    ST_LIST_OVERFLOW = 8u,  // near-tile list capacity exceeded
    ST_TMA_TIMEOUT = 16u,   // a bulk-update block gave up waiting for a tensor copy
    ST_BOUNDS = 32u,        // bounds-checked build only: an index left its array
};

// Bounds-checked debug build (compiled with -DLBIB_CHECKED): LBIB_IDX(i, n, st)
// is i when 0 <= i < n; otherwise it sets ST_BOUNDS in the status word st and
// gives 0, so the access lands on the array's first element instead of outside
// it (nothing traps: the host reads the bit at the next sync).  In the normal
// build it is i, and st is not evaluated.
#ifdef LBIB_CHECKED
__device__ __forceinline__ long long lbib_idx(long long i, long long n, uint32_t* st)
{
    if (i >= 0 && i < n) return i;
    atomicOr(st, (uint32_t)ST_BOUNDS);
    return 0;
}
#define LBIB_IDX(i, n, st) lbib_idx((long long)(i), (long long)(n), (st))
#else
#define LBIB_IDX(i, n, st) (i)
#endif

enum { PREC_F64 = 0, PREC_F32 = 1 };  // compute type of the kernels

// Population storage type (values of lbib_storage): FP64 and FP32 store the
// deviations f_i - w_i as is; BF16 stores them rounded to bfloat16; FP16
// stores them times HALF_SCALE (an exact power of two that keeps deviations of
// 1e-9 .. 3 in the normal range of binary16).  The 16-bit kinds compute in FP32.
enum { STORE_F64 = 0, STORE_F32 = 1, STORE_BF16 = 2, STORE_F16 = 3 };
constexpr float HALF_SCALE = 16384.0f;

// A context holds one or more capillary instances (a sweep) side by side
// along x in one lattice: instance i occupies the node columns
// [x0_i, x0_i + nx_i) with x0_i a multiple of TX, so that every tile column
// belongs to exactly one instance; all instances share ny and the fluid
// parameters.  A single capillary is the batch of one.
struct Lattice {
    int nx, ny, nxp;          // nx: node columns of the whole batch; nxp: row pitch (multiple of TX)
    int ntx, nty, ntiles;     // tiles of the whole batch
    int bc;                   // lbib_bc_mode
    int qstride;              // ny * nxp
    double tau, omega, nu, umax, rho_out, gx, gy;
    // the same parameters rounded to FP32 once on the host: FP32 kernels read
    // these instead of converting the doubles per node (FP64 is a narrow pipe)
    float omega_f, umax_f, rho_out_f, gx_f, gy_f;
    // fields added later go last: moving the ones above changed the bulk
    // kernel's register allocation (40 -> 48 at two nodes per thread), which
    // cost 3.5 % of the step
    int transfer;             // lbib_transfer
#ifdef LBIB_CHECKED
    uint32_t* chk_status;     // the context's status word (LBIB_IDX)
#endif
};

// Lattice parameter in the compute type R: the double for R = double, the
// host-rounded float for R = float.
template <typename R>
__host__ __device__ __forceinline__ R lat_param(double d, float f);
template <>
__host__ __device__ __forceinline__ double lat_param<double>(double d, float) { return d; }
template <>
__host__ __device__ __forceinline__ float lat_param<float>(double, float f) { return f; }

inline void set_float_params(Lattice& L)
{
    L.omega_f = (float)L.omega;
    L.umax_f = (float)L.umax;
    L.rho_out_f = (float)L.rho_out;
    L.gx_f = (float)L.gx;
    L.gy_f = (float)L.gy;
}

// Per tile column: origin and width of its instance, the instance's first
// marker (marker ids in the tile bit masks are local to the instance) and the
// instance index.  Layout of an int4.
struct ColInfo {
    int x0, nx, moff, inst;
};

struct InstConst {
    int x0, nx;               // node columns [x0, x0 + nx)
    int moff, nmark;          // markers (= vertices) of the instance's bodies
    int body0, nbodies;       // bodies [body0, body0 + nbodies)
    int lig0, nlig;           // ligand sites
    int first_cell, first_particle;  // global body ids or -1
    int pad0, pad1;
    uint64_t seed;            // Philox key of the instance's bond kinetics
};

struct BodyConst {
    int kind, motion, nv, off;        // off: global index of vertex 0 / element 0
    int adhesive, nlig, lig_off, nl0;
    int sigma_inf, inst, x0, nxi;     // instance and its node columns [x0, x0 + nxi)
    int moff, lig0, b0, nbi;          // instance's first marker, first site, first body, body count
    double A0, P0, inv_A0, inv_P0;
    double ks, kb, ka, mv, mass, inertia;
    double sigma, ycr, yeq, Pf, kr0_dt, xi;
};

// rigid-body state per body (FP64): centroid, angle, BDF2 history
enum { RG_XC = 0, RG_YC, RG_ANG, RG_U1X, RG_U1Y, RG_U2X, RG_U2Y, RG_W1, RG_W2, RG_N };
// per-body observables/extent written by the Lagrangian kernel (FP64)
// BO_DPERIM: perimeter minus stress-free perimeter, sum of (l - l_0)
enum { BO_AREA = 0, BO_DPERIM, BO_CX, BO_CY, BO_NBOUND, BO_XMIN, BO_XMAX, BO_YMIN, BO_YMAX, BO_N };

// Every device pointer of a context.  Passed by value to the kernels.
struct Dev {
    Lattice L;
    int store;                 // STORE_*: element type of f
    // lattice state
    void* f[2];                // Store
    void* drho;                // Real [ny][nxp]: rho - 1 on near tiles
    void* ux;                  // Real [ny][nxp]
    void* uy;                  // Real [ny][nxp]
    void* fx;                  // Real [ny][nxp]: total force density (g + F_E) the near update used
    void* fy;                  // Real [ny][nxp]
    int32_t* fresh;            // [ntiles]: lattice step whose near update wrote rho/u
    // nearflag[m % 3][t]: tile t is updated by the near kernel at lattice step m.
    // Set by k_activate_next after the membrane update of step m - 2 (or by
    // k_activate at set-up and restore), read by the
    // bulk and near updates of step m, cleared by the membrane update of step m;
    // three slots so that the bulk update of step m + 1, which runs alongside
    // the membrane update of step m, reads a slot nobody writes.
    uint32_t* nearflag[3];
    int32_t* list[3];          // [list_cap]: near tiles of lattice step m, m % 3
    int32_t* count;            // [3]
    uint32_t* mask[2];         // [ntiles][mw], bit k: the instance's marker k
    int mw, list_cap;
    // markers consumed by lattice step m, parity m & 1:
    //   mki[p] = int32 [2][nmark]: floor(X), floor(Y - 1/2)
    //   mkf[p] = Real [4][nmark]: X - floor(X), Y - 1/2 - floor(Y - 1/2), Fx ds, Fy ds
    int32_t* mki[2];
    void* mkf[2];
    const int4* colinfo;       // [ntx] ColInfo of each tile column
    int ninst;
    const InstConst* inst;     // [ninst]
    // Lagrangian state
    int nbodies, nmark, nlig, nv_max;
    int lag_threads;           // Lagrangian block size: 256 or 512 (results do not depend on it)
    int bulk_tiles_y;          // tiles per bulk-kernel block, stacked in y: 1, 2 or 4 (likewise)
    int bulk_nodes_per_thread; // nodes per bulk-kernel thread: 1 or 2 (likewise)
    double* pos[2];            // [2][nmark] (x block then y block); X^n in pos[n & 1]
    void* posf[2];             // Real [4][nmark]: X^n as float-float pairs (x hi, x lo, y hi, y lo)
    const BodyConst* body;     // [nbodies]
    double* rigid;             // [nbodies][RG_N]
    const void* l0;            // Real [nmark] stress-free element lengths
    const void* th0;           // Real [nmark] stress-free turning angles
    const double* rref;        // [2][nmark] rigid vertex offsets at angle 0
    const int32_t* lig_el;     // [nlig] element (global index) of each ligand site
    const void* lig_t;         // Real [nlig] fraction along the element
    int32_t* bound;            // [nlig]
    double* anchor;            // [2][nlig]
    void* margin;              // Real [nlig]
    const int32_t* site_off;   // [nmark + 1] sites of element e: [site_off[e], site_off[e+1])
    void* diag;                // Real [NDIAG][nmark]
    double* body_obs[2];       // [nbodies][BO_N] of X^k in body_obs[k & 1]
    lbib_obs* ring;            // [ninst][ring_cap]
    int ring_cap;
    int64_t* step;             // Lagrangian step counter n (advanced by the last Lagrangian block)
    uint32_t* status;
    uint32_t* ticket;
    // every act_stride-th element centroid activates the tiles within reach of
    // itself and the elements up to the next activating one (from the current
    // positions)
    int act_stride;            // 1, 2 or 4 (results do not depend on it)
    int chain_priority;        // stream priority of the membrane and near launches (0: default)
    double dcut;               // repulsion cut-off (Eq. 12)
    double probe;              // probe length (Sec. 2.6)
    double uscale;             // observables: u_max / H
    // fields added later go last
    int bulk_tma;              // 1: the bulk update stages its populations with tensor copies
    const void* fmaps;         // host copy of the two population tensor maps (parity 0, 1), or null
};

// ------------------------------------------------------------------ launchers
// (defined in lbib_lbm.cu and lbib_lag.cu; `prec` selects FP64 or FP32)
// bulk update of lattice step m: parity = m & 1, slot = m % 3
cudaError_t launch_lbm_bulk(const Dev& d, int prec, int parity, int slot, cudaStream_t s);
// pdl: k_spread and k_near_lbm are launched as programmatic dependents of the
// kernel enqueued before them (the membrane update, then k_spread)
cudaError_t launch_lbm_near(const Dev& d, int prec, int parity, int grid, int update_grid, cudaStream_t s, bool pdl);
cudaError_t launch_init_populations(const Dev& d, int prec, int buf, cudaStream_t s);
// tensor maps of the two population buffers for the TMA-staged bulk update
// (out: two CUtensorMap, 64-byte aligned); and its kernel attributes
cudaError_t make_population_maps(const Dev& d, void* out);
cudaError_t configure_bulk_tma(int store);
// moments of one instance (node columns [x0, x0 + inx)) into [ny][inx] arrays
cudaError_t launch_macro(const Dev& d, int prec, int buf, int64_t m, int x0, int inx, double* rho, double* ux,
                         double* uy, cudaStream_t s);
cudaError_t launch_macro_typed(const Dev& d, int prec, int buf, int64_t m, int x0, int inx, void* ux, void* uy,
                               int dtype, cudaStream_t s);
cudaError_t launch_lagrangian(const Dev& d, int prec, int parity, cudaStream_t s);
// the observables record of the step the last membrane update completed
// pdl: a programmatic dependent of the kernel enqueued before it
cudaError_t launch_observables(const Dev& d, cudaStream_t s, bool urgent, bool pdl);
// near tiles of the step after next, from the positions the membrane kernel stored
cudaError_t launch_activate_next(const Dev& d, cudaStream_t s);
cudaError_t launch_activate(const Dev& d, int prec, int64_t m, int which, cudaStream_t s);
cudaError_t launch_rebuild_mask(const Dev& d, int prec, int64_t m, cudaStream_t s);
size_t lagrangian_smem_bytes(int prec, int nv_max);
// message returned by lbib_last_error(NULL) (calls that have no context)
void set_global_error(const char* msg);
// cudaMalloc through the allocation-failure countdown of
// lbib_inject_alloc_failure (every device allocation of the library goes here)
cudaError_t device_malloc(void** p, size_t bytes);
// the same through cudaMallocAsync on stream s (the device's default memory pool)
cudaError_t device_malloc_async(void** p, size_t bytes, cudaStream_t s);
cudaError_t configure_kernels(int prec, int nv_max);

}  // namespace lbib
