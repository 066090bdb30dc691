/*
 * lbib_oracle.c -- plain FP64 CPU oracle of one time step of the hybrid
 * lattice-Boltzmann / immersed-boundary method of Coclite, Pascazio,
 * de Tullio and Decuzzi, "Predicting the vascular adhesion of deformable drug
 * carriers in narrow capillaries traversed by blood cells" (J. Fluids Struct.).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark load this file.  It shares no
 * source, header, table or helper with the CUDA library; it is written from the
 * paper's equations, plainly, in double precision, with no blocking, fusion or
 * reordering beyond what the equations state.
 *
 * State convention: the stored populations are the post-collision values
 * f*(x, t) of Eq. 1's right-hand side.  One call of orc_step performs, in
 * order:
 *   1. streaming (Eq. 1 left-hand side) with the wall and inlet/outlet
 *      conditions (Sec. 2.2, Sec. 3.1);
 *   2. moments with the half-force shift (Eqs. 5-6);
 *   3. BGK collision with the Hermite equilibrium and Guo's forcing term
 *      (Eqs. 1, 2, 4);
 *   4. the Lagrangian update from the velocity of step 2: interpolation at
 *      the vertices (Sec. 2.8), probes for pressure and velocity gradients
 *      (Sec. 2.6), ligand-receptor kinetics and force (Eq. 13), membrane
 *      forces (Eqs. 8, 10, 11), repulsion (Eq. 12), tractions (Eqs. 14-15),
 *      Verlet + BDF2 (Eqs. 17-18) or rigid BDF2 (Eq. 19);
 *   5. explicit direct forcing at the element centroids and spreading to the
 *      lattice; the result is the body force of the next collision.
 *
 * Readings where the paper is silent or garbled (all shared with the library
 * through the written design, never through code):
 *   - Eq. 6's "dt/2 F_i" is the body force f_ib (Guo et al. 2002).
 *   - Walls: halfway bounce-back; node (i, j) sits at (i, j + 1/2); walls at
 *     y = 0 and y = ny.  Inlet: Zou-He velocity with the plane-Poiseuille
 *     profile; outlet: Zou-He pressure with rho = rho_out.  Bounce-back first,
 *     then Zou-He overrides the three unknown populations on the inlet and
 *     outlet columns, corners included.
 *   - Interpolation and spreading use Peskin's 4-point discrete delta over a
 *     4 x 4 stencil.  Stencil nodes beyond a wall are wall nodes: they carry
 *     the wall's zero velocity (velocity interpolation is the plainly truncated
 *     sum) and absorb the share of a spread force that falls on them.  Density
 *     has no wall value: its weights are renormalised over the fluid nodes.
 *     Gradients are the exact derivatives of these interpolants.
 *   - The alternative transfer (orc_set_transfer): the moving-least-squares
 *     reconstruction of Vanella and Balaras (2009) that Sec. 2.2 cites, with
 *     a linear basis and the cubic-spline weight of support half-width 2 (the
 *     same 4 x 4 stencil); walls as for the Peskin stencil (wall nodes in the
 *     fit, zero velocity, force absorbed, density renormalised), gradients
 *     the fit's linear coefficients, spreading with the same shape functions
 *     (the adjoint).
 *   - Direct forcing: F_L = rho (U_struct - U*) / dt at the new element
 *     centroids, U* and rho interpolated from the moments of step 2, spread
 *     with weight ds = element length.  A marker closer than half a spacing
 *     to a wall (below the first row of fluid nodes) is not forced: the
 *     wall's bounce-back condition already holds the fluid there.
 *   - A traction probe that would cross a wall stops at the wall.
 *   - Bending: theta is the signed turning angle at the vertex of a
 *     counter-clockwise chain; the "t" in Eq. 10's denominators is "+";
 *     l_right is the length of the edge on the left of the vertex and l_left
 *     that of the edge on its right (the order in which Sec. 2.3 defines
 *     them), which makes the three forces torque-free.
 *   - Area: shoelace formula (Green's theorem with the factor 1/2).
 *   - Bond laws (cited, not printed): P_f = 1 - exp(-k_f dt) when the gap to
 *     the nearest wall is below y_cr; P_r = 1 - exp(-k_r dt) with
 *     k_r = k_r0 exp(xi (y - y_eq)^2).  One uniform draw per ligand site and
 *     step from Philox4x32-10 (Salmon et al., SC'11).
 *   - Vertex mass m_v = rho_body A_0 / nv; rigid mass rho_body A_0 and polar
 *     moment rho_body J_c of the polygon.
 *
 * Host threads: the node loops of streaming and collision may run on several
 * threads (OpenMP over rows and nodes, orc_set_threads); every node's
 * arithmetic and every sum keep one order, so the results are the same bits
 * for any thread count.  Everything else runs on one thread.
 *
 * Parity status: every numbered piece above is pinned by the CPU tests
 * (closed forms, moment identities, brute force).  The coupled trajectory as a
 * whole has no printed numbers to pin it ("parity unpinned" for the full
 * trajectory beyond its pieces and invariants).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_Q 9
#define ORC_MAX_BODIES 16

enum { ORC_BC_INLET_OUTLET = 0, ORC_BC_PERIODIC_FORCE = 1 };
/* Eulerian-Lagrangian transfer kernel: Peskin's 4-point delta (the default
 * reading) or the moving-least-squares reconstruction the paper cites. */
enum { ORC_TRANSFER_PESKIN = 0, ORC_TRANSFER_MLS = 1 };
enum { ORC_CELL = 0, ORC_PARTICLE = 1 };
enum { ORC_DEFORMABLE = 0, ORC_RIGID = 1, ORC_FIXED = 2 };

/* ---------------------------------------------------------------- lattice */

/* Host threads for the node loops (1: serial); returns the count in use. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Eq. 3 evaluated literally: rest, four axis and four diagonal speeds. */
static int EX[ORC_Q], EY[ORC_Q], OPP[ORC_Q];
static double WQ[ORC_Q];
static const double CS2 = 1.0 / 3.0; /* c_s^2, Sec. 2.1 */

static int lattice_ready = 0;

static void lattice_init(void)
{
    if (lattice_ready) return;
    for (int i = 0; i < ORC_Q; ++i) {
        double ex, ey;
        if (i == 0) {
            ex = 0.0;
            ey = 0.0;
        } else if (i <= 4) {
            ex = cos((i - 1) * M_PI / 2.0);
            ey = sin((i - 1) * M_PI / 2.0);
        } else {
            ex = sqrt(2.0) * cos((2 * i - 9) * M_PI / 4.0);
            ey = sqrt(2.0) * sin((2 * i - 9) * M_PI / 4.0);
        }
        EX[i] = (int)lround(ex);
        EY[i] = (int)lround(ey);
        WQ[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    for (int i = 0; i < ORC_Q; ++i)
        for (int j = 0; j < ORC_Q; ++j)
            if (EX[j] == -EX[i] && EY[j] == -EY[i]) OPP[i] = j;
    lattice_ready = 1;
}

void orc_lattice(int* ex, int* ey, double* w, int* opp)
{
    lattice_init();
    for (int i = 0; i < ORC_Q; ++i) {
        ex[i] = EX[i];
        ey[i] = EY[i];
        w[i] = WQ[i];
        opp[i] = OPP[i];
    }
}

/* Eq. 2: second-order Hermite equilibrium. */
void orc_equilibrium(double rho, double ux, double uy, double* feq)
{
    lattice_init();
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < ORC_Q; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        feq[i] = WQ[i] * rho * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Eq. 4: Guo forcing term for body force (fx, fy). */
void orc_guo_term(double ux, double uy, double fx, double fy, double tau, double* out)
{
    lattice_init();
    for (int i = 0; i < ORC_Q; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        double ax = (EX[i] - ux) / CS2 + eu * EX[i] / (CS2 * CS2);
        double ay = (EY[i] - uy) / CS2 + eu * EY[i] / (CS2 * CS2);
        out[i] = (1.0 - 1.0 / (2.0 * tau)) * WQ[i] * (ax * fx + ay * fy);
    }
}

/* Sec. 3.1: plane-Poiseuille inlet profile, walls at y = 0 and y = H. */
static double inlet_u(double y, double H, double umax)
{
    return 4.0 * umax * y * (H - y) / (H * H);
}

/* Zou & He (1997) velocity condition on a left boundary node: the three
 * populations entering from x < 0 (i = 1, 5, 8) follow from mass, both
 * momentum components and bounce-back of the normal non-equilibrium part. */
static void zou_he_velocity_left(double* f, double u, double v)
{
    double rho = (f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7])) / (1.0 - u);
    f[1] = f[3] + (2.0 / 3.0) * rho * u;
    f[5] = f[7] - 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * rho * u + 0.5 * rho * v;
    f[8] = f[6] + 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * rho * u - 0.5 * rho * v;
}

/* Zou & He (1997) pressure (density) condition on a right boundary node,
 * zero transverse velocity: unknowns i = 3, 6, 7. */
static void zou_he_pressure_right(double* f, double rho)
{
    double u = -1.0 + (f[0] + f[2] + f[4] + 2.0 * (f[1] + f[5] + f[8])) / rho;
    f[3] = f[1] - (2.0 / 3.0) * rho * u;
    f[7] = f[5] + 0.5 * (f[2] - f[4]) - (1.0 / 6.0) * rho * u;
    f[6] = f[8] - 0.5 * (f[2] - f[4]) - (1.0 / 6.0) * rho * u;
}

/* Eq. 1 left-hand side: f(x + e_i, t + 1) = f*(x, t), then the boundary
 * conditions.  Layout [q][y][x]. */
void orc_stream_bc(int nx, int ny, int bc, double umax, double rho_out, const double* fpost, double* f)
{
    lattice_init();
    size_t n = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int q = 0; q < ORC_Q; ++q) {
                int xs = x - EX[q], ys = y - EY[q];
                double v;
                if (ys < 0 || ys >= ny) {
                    v = fpost[OPP[q] * n + (size_t)y * nx + x]; /* halfway bounce-back */
                } else if (xs < 0 || xs >= nx) {
                    if (bc == ORC_BC_PERIODIC_FORCE)
                        v = fpost[q * n + (size_t)ys * nx + (size_t)((xs + nx) % nx)];
                    else
                        v = NAN; /* unknown, set by Zou-He below */
                } else {
                    v = fpost[q * n + (size_t)ys * nx + xs];
                }
                f[q * n + (size_t)y * nx + x] = v;
            }
    if (bc != ORC_BC_INLET_OUTLET) return;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        double g[ORC_Q];
        for (int q = 0; q < ORC_Q; ++q) g[q] = f[q * n + (size_t)y * nx + 0];
        zou_he_velocity_left(g, inlet_u(y + 0.5, (double)ny, umax), 0.0);
        for (int q = 0; q < ORC_Q; ++q) f[q * n + (size_t)y * nx + 0] = g[q];
        for (int q = 0; q < ORC_Q; ++q) g[q] = f[q * n + (size_t)y * nx + (nx - 1)];
        zou_he_pressure_right(g, rho_out);
        for (int q = 0; q < ORC_Q; ++q) f[q * n + (size_t)y * nx + (nx - 1)] = g[q];
    }
}

/* --------------------------------------------------------- discrete delta */

/* Peskin (2002, Acta Numerica) 4-point kernel. */
double orc_phi(double r)
{
    double a = fabs(r);
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
    return 0.0;
}

/* d(phi)/dr, the derivative of the expression above. */
double orc_dphi(double r)
{
    double a = fabs(r), s = (r < 0.0) ? -1.0 : 1.0, d;
    if (a <= 1.0)
        d = (-2.0 + (4.0 - 8.0 * a) / (2.0 * sqrt(1.0 + 4.0 * a - 4.0 * a * a))) / 8.0;
    else if (a <= 2.0)
        d = (-2.0 - (12.0 - 8.0 * a) / (2.0 * sqrt(-7.0 + 12.0 * a - 4.0 * a * a))) / 8.0;
    else
        d = 0.0;
    return s * d;
}

/* ------------------------------------------ moving least squares (MLS) */

/* MLS weight along one direction: the cubic spline of |r| / 2, so its
 * support covers the same 4 x 4 nodes around a point as the Peskin stencil.
 * Values 2/3 at r = 0, 1/6 at |r| = 1, 0 from |r| = 2 on. */
double orc_mls_weight(double r)
{
    double q = fabs(r) / 2.0;
    if (q <= 0.5) return 2.0 / 3.0 - 4.0 * q * q + 4.0 * q * q * q;
    if (q <= 1.0) return (4.0 / 3.0) * (1.0 - q) * (1.0 - q) * (1.0 - q);
    return 0.0;
}

/* The moving-least-squares reconstruction cited in Sec. 2.2 (Vanella and
 * Balaras 2009), with the linear basis p(x, y) = (1, x - X, y - Y) about the
 * point (X, Y) and weights W_j = w(x_j - X) w(y_j - Y) over the 4 x 4 stencil
 * around it: the weighted least-squares fit of a nodal field f has
 * coefficients a = A^{-1} sum_j W_j p_j f_j with A = sum_j W_j p_j p_j^T;
 * a_0 is the reconstructed value at (X, Y) and (a_1, a_2) its gradient.  The
 * walls follow the same reading as the Peskin stencil: nodes beyond a wall
 * (or beyond the lattice ends) are wall nodes, so the fit always spans the
 * whole stencil and A depends on (X, Y) alone.  Writes A^{-1} (row-major
 * 3 x 3) to inv. */
static void mls_inverse(double X, double Y, double inv[9])
{
    double A[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int i0 = (int)floor(X) - 1, j0 = (int)floor(Y - 0.5) - 1;
    for (int j = j0; j <= j0 + 3; ++j)
        for (int i = i0; i <= i0 + 3; ++i) {
            double W = orc_mls_weight(i - X) * orc_mls_weight(j + 0.5 - Y);
            double pv[3] = {1.0, i - X, j + 0.5 - Y};
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) A[3 * r + c] += W * pv[r] * pv[c];
        }
    /* inverse by cofactors (A is symmetric; the full stencil keeps it regular) */
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    inv[0] = c00 / det;
    inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    inv[3] = c01 / det;
    inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    inv[6] = c02 / det;
    inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

/* MLS shape functions at (X, Y) of the stencil node (i, j): phi[0] weights the
 * nodal values into the reconstruction, phi[1] and phi[2] into its x- and
 * y-derivatives: phi[k] = W_j (A^{-1} p_j)_k. */
static void mls_shape(const double inv[9], double X, double Y, int i, int j, double phi[3])
{
    double W = orc_mls_weight(i - X) * orc_mls_weight(j + 0.5 - Y);
    double pv[3] = {1.0, i - X, j + 0.5 - Y};
    for (int k = 0; k < 3; ++k) phi[k] = W * (inv[3 * k] * pv[0] + inv[3 * k + 1] * pv[1] + inv[3 * k + 2] * pv[2]);
}

/* MLS interpolation of a nodal field at (X, Y).  Velocity-type (renorm = 0):
 * wall nodes carry the wall's zero velocity, so the sums simply skip them;
 * *val the reconstruction, *gx, *gy its gradient coefficients.  Density-type
 * (renorm = 1): no wall value, so the value's shape functions are
 * renormalised over the fluid nodes (as the Peskin weights are).  Returns the
 * sum S of the value's shape functions over the nodes inside the lattice (one
 * away from walls). */
static double interp_mls(int nx, int ny, const double* fld, double X, double Y, double* val, double* gx, double* gy,
                         int renorm)
{
    double inv[9];
    mls_inverse(X, Y, inv);
    double S = 0.0, Sx = 0.0, Sy = 0.0, a0 = 0.0, a1 = 0.0, a2 = 0.0;
    int i0 = (int)floor(X) - 1, j0 = (int)floor(Y - 0.5) - 1;
    for (int j = j0; j <= j0 + 3; ++j) {
        if (j < 0 || j >= ny) continue;
        for (int i = i0; i <= i0 + 3; ++i) {
            if (i < 0 || i >= nx) continue;
            double phi[3];
            mls_shape(inv, X, Y, i, j, phi);
            double u = fld[(size_t)j * nx + i];
            S += phi[0];
            Sx += phi[1];
            Sy += phi[2];
            a0 += phi[0] * u;
            a1 += phi[1] * u;
            a2 += phi[2] * u;
        }
    }
    if (!renorm) {
        if (val) *val = a0;
        if (gx) *gx = a1;
        if (gy) *gy = a2;
        return S;
    }
    double I = (S > 0.0) ? a0 / S : 0.0;
    if (val) *val = I;
    if (gx) *gx = (S > 0.0) ? (a1 - I * Sx) / S : 0.0;
    if (gy) *gy = (S > 0.0) ? (a2 - I * Sy) / S : 0.0;
    return S;
}

/* Interpolation of a nodal field at (X, Y) with the 4 x 4 Peskin stencil.
 * Nodes beyond the walls are wall nodes: for a velocity (renorm = 0) they hold
 * the wall's zero velocity, so the stencil is simply truncated; a density
 * (renorm = 1) has no wall value, so the weights of the fluid nodes are
 * renormalised to one.  Returns W = sum of weights of the nodes inside the
 * lattice; *val the interpolant, *gx, *gy its exact X- and Y-derivatives. */
static double interp_field(int nx, int ny, const double* fld, double X, double Y, double* val, double* gx,
                           double* gy, int renorm)
{
    double W = 0.0, N = 0.0, Wx = 0.0, Wy = 0.0, Nx = 0.0, Ny = 0.0;
    int i0 = (int)floor(X) - 1, j0 = (int)floor(Y - 0.5) - 1;
    for (int j = j0; j <= j0 + 3; ++j) {
        if (j < 0 || j >= ny) continue;
        double ry = Y - (j + 0.5);
        double py = orc_phi(ry), dpy = orc_dphi(ry);
        for (int i = i0; i <= i0 + 3; ++i) {
            if (i < 0 || i >= nx) continue;
            double rx = X - i;
            double px = orc_phi(rx), dpx = orc_dphi(rx);
            double u = fld[(size_t)j * nx + i];
            W += px * py;
            N += u * px * py;
            Wx += dpx * py;
            Wy += px * dpy;
            Nx += u * dpx * py;
            Ny += u * px * dpy;
        }
    }
    if (!renorm) {
        if (val) *val = N;
        if (gx) *gx = Nx;
        if (gy) *gy = Ny;
        return W;
    }
    double I = (W > 0.0) ? N / W : 0.0;
    if (val) *val = I;
    if (gx) *gx = (W > 0.0) ? (Nx - I * Wx) / W : 0.0;
    if (gy) *gy = (W > 0.0) ? (Ny - I * Wy) / W : 0.0;
    return W;
}

/* Interpolation with the transfer kernel `kind` (ORC_TRANSFER_*). */
static double interp_kind(int kind, int nx, int ny, const double* fld, double X, double Y, double* val, double* gx,
                          double* gy, int renorm)
{
    if (kind == ORC_TRANSFER_MLS) return interp_mls(nx, ny, fld, X, Y, val, gx, gy, renorm);
    return interp_field(nx, ny, fld, X, Y, val, gx, gy, renorm);
}

/* Stand-alone interpolation on a caller field (for the pins). */
double orc_interp(int nx, int ny, const double* fld, double X, double Y, double* val, double* gx, double* gy,
                  int renorm, int kind)
{
    return interp_kind(kind, nx, ny, fld, X, Y, val, gx, gy, renorm);
}

/* Spreading of point forces (Fx, Fy) with weights ds onto a field with the
 * same truncated stencil (the adjoint of the velocity interpolation), Peskin
 * weights or MLS shape functions: the share that would land on wall nodes is
 * taken up by the wall. */
void orc_spread(int nx, int ny, int n, const double* X, const double* Y, const double* Fx, const double* Fy,
                const double* ds, double* outx, double* outy, int kind)
{
    for (int m = 0; m < n; ++m) {
        int i0 = (int)floor(X[m]) - 1, j0 = (int)floor(Y[m] - 0.5) - 1;
        double inv[9];
        if (kind == ORC_TRANSFER_MLS) mls_inverse(X[m], Y[m], inv);
        for (int j = j0; j <= j0 + 3; ++j) {
            if (j < 0 || j >= ny) continue;
            for (int i = i0; i <= i0 + 3; ++i) {
                if (i < 0 || i >= nx) continue;
                double w;
                if (kind == ORC_TRANSFER_MLS) {
                    double phi[3];
                    mls_shape(inv, X[m], Y[m], i, j, phi);
                    w = phi[0];
                } else {
                    w = orc_phi(X[m] - i) * orc_phi(Y[m] - (j + 0.5));
                }
                outx[(size_t)j * nx + i] += Fx[m] * ds[m] * w;
                outy[(size_t)j * nx + i] += Fy[m] * ds[m] * w;
            }
        }
    }
}

/* ------------------------------------------------------------- Philox */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
 * 32x32->64 multiplies with a Weyl-sequence key schedule. */
void orc_philox4x32_10(const uint32_t* ctr_in, const uint32_t* key_in, uint32_t* out)
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* The uniform draw of ligand site `site` at step `step`: counter
 * (step_lo, step_hi, site, 0), key (seed_lo, seed_hi), u = (w0 >> 8) 2^-24. */
double orc_bond_uniform(uint64_t seed, int64_t step, uint32_t site)
{
    uint32_t ctr[4] = {(uint32_t)(uint64_t)step, (uint32_t)((uint64_t)step >> 32), site, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return (double)(out[0] >> 8) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------ polygon geometry */

/* Shoelace area, perimeter, area centroid and polar second moment about the
 * centroid of the closed chain (x, y).  out = {A, P, cx, cy, Jc}. */
void orc_polygon(int nv, const double* x, const double* y, double* out)
{
    double A2 = 0.0, P = 0.0, Cx = 0.0, Cy = 0.0, J = 0.0;
    for (int v = 0; v < nv; ++v) {
        int w = (v + 1) % nv;
        double cr = x[v] * y[w] - x[w] * y[v];
        A2 += cr;
        P += hypot(x[w] - x[v], y[w] - y[v]);
        Cx += (x[v] + x[w]) * cr;
        Cy += (y[v] + y[w]) * cr;
        J += cr * (x[v] * x[v] + x[v] * x[w] + x[w] * x[w] + y[v] * y[v] + y[v] * y[w] + y[w] * y[w]);
    }
    double A = 0.5 * A2;
    Cx /= (6.0 * A);
    Cy /= (6.0 * A);
    J /= 12.0;
    out[0] = A;
    out[1] = P;
    out[2] = Cx;
    out[3] = Cy;
    out[4] = J - A * (Cx * Cx + Cy * Cy);
}

/* Element lengths, outward normals (counter-clockwise chain), vertex
 * normals and signed turning angles. Element l joins vertex l and l+1. */
static void chain_geometry(int nv, const double* x, const double* y, double* len, double* nlx, double* nly,
                           double* nvx, double* nvy, double* th)
{
    for (int l = 0; l < nv; ++l) {
        int w = (l + 1) % nv;
        double dx = x[w] - x[l], dy = y[w] - y[l];
        double L = hypot(dx, dy);
        len[l] = L;
        nlx[l] = dy / L;
        nly[l] = -dx / L;
    }
    for (int v = 0; v < nv; ++v) {
        int lm = (v + nv - 1) % nv;
        double ax = x[v] - x[lm], ay = y[v] - y[lm];
        double bx = x[(v + 1) % nv] - x[v], by = y[(v + 1) % nv] - y[v];
        if (th) th[v] = atan2(ax * by - ay * bx, ax * bx + ay * by);
        if (nvx) {
            double sx = nlx[lm] + nlx[v], sy = nly[lm] + nly[v];
            double s = hypot(sx, sy);
            nvx[v] = sx / s;
            nvy[v] = sy / s;
        }
    }
}

/* Eq. 7: stretching energy of the chain. */
double orc_stretch_energy(int nv, const double* x, const double* y, const double* l0, double ks)
{
    double V = 0.0;
    for (int l = 0; l < nv; ++l) {
        int w = (l + 1) % nv;
        double L = hypot(x[w] - x[l], y[w] - y[l]);
        V += 0.5 * ks * (L - l0[l]) * (L - l0[l]);
    }
    return V;
}

/* Internal membrane forces on every vertex: stretching (Eq. 8), bending
 * (Eq. 10) and the area penalty (Eq. 11, half of each element's force to
 * each of its vertices).  All outputs are overwritten. */
void orc_membrane_forces(int nv, const double* x, const double* y, const double* l0, const double* th0, double A0,
                         double ks, double kb, double ka, double pref, double* fsx, double* fsy, double* fbx,
                         double* fby, double* fax, double* fay)
{
    double *len = malloc(sizeof(double) * nv), *nlx = malloc(sizeof(double) * nv),
           *nly = malloc(sizeof(double) * nv), *nvx = malloc(sizeof(double) * nv),
           *nvy = malloc(sizeof(double) * nv), *th = malloc(sizeof(double) * nv);
    chain_geometry(nv, x, y, len, nlx, nly, nvx, nvy, th);
    double poly[5];
    orc_polygon(nv, x, y, poly);
    double A = poly[0];
    for (int v = 0; v < nv; ++v) {
        fsx[v] = fsy[v] = fbx[v] = fby[v] = fax[v] = fay[v] = 0.0;
    }
    for (int l = 0; l < nv; ++l) {
        int a = l, b = (l + 1) % nv;
        /* Eq. 8: F_1 = -k_s (l - l_0) r_12 / l, F_2 = -k_s (l - l_0) r_21 / l */
        double c = -ks * (len[l] - l0[l]) / len[l];
        fsx[a] += c * (x[a] - x[b]);
        fsy[a] += c * (y[a] - y[b]);
        fsx[b] += c * (x[b] - x[a]);
        fsy[b] += c * (y[b] - y[a]);
        /* Eq. 11 with the inward normal n^- = -n: F = k_a (1 - A/A0) p_ref n l */
        double fa = -ka * (1.0 - A / A0) * pref * len[l];
        double fx = fa * (-nlx[l]), fy = fa * (-nly[l]);
        fax[a] += 0.5 * fx;
        fay[a] += 0.5 * fy;
        fax[b] += 0.5 * fx;
        fay[b] += 0.5 * fy;
    }
    for (int v = 0; v < nv; ++v) {
        /* Eq. 10 for the vertex triple (v-1, v, v+1).  Sec. 2.3 names l_right
         * the length of the edge on the left of v and l_left that of the edge
         * on its right; so the left vertex takes the right edge's share and
         * the right vertex the left edge's, and the three forces have no net
         * torque about any point. */
        int vl = (v + nv - 1) % nv, vr = (v + 1) % nv;
        double l_right = len[vl], l_left = len[v];
        double c = kb * (th[v] - th0[v]);
        fbx[vl] += c * l_left / (l_left + l_right) * nvx[v];
        fby[vl] += c * l_left / (l_left + l_right) * nvy[v];
        fbx[v] += -c * nvx[v];
        fby[v] += -c * nvy[v];
        fbx[vr] += c * l_right / (l_left + l_right) * nvx[v];
        fby[vr] += c * l_right / (l_left + l_right) * nvy[v];
    }
    free(len);
    free(nlx);
    free(nly);
    free(nvx);
    free(nvy);
    free(th);
}

/* Eq. 12 magnitude at distance d (lattice units, dx = 1). */
double orc_repulsion_magnitude(double d)
{
    return 1e-4 / (8.0 * sqrt(2.0)) * sqrt(1.0 / (d * d * d * d * d));
}

/* Eq. 19: one BDF2 update of a rigid velocity component. */
double orc_rigid_bdf2(double u1, double u2, double acc)
{
    return (2.0 / 3.0) * (2.0 * u1 - 0.5 * u2 + acc);
}

/* ------------------------------------------------- storage of deviations */

/* The precisions a library may store the post-collision deviations
 * g = f* - w_i in: exact (FP64), binary32, bfloat16 (8 significant bits) and
 * binary16 after scaling by 2^14 (11 significant bits).  The 16-bit kinds
 * round the binary32 value of g, as a store from FP32 arithmetic would; every
 * rounding is to nearest, ties to even (nearbyint in the default mode). */
enum { ORC_STORE_EXACT = 0, ORC_STORE_F32 = 1, ORC_STORE_BF16 = 2, ORC_STORE_F16 = 3 };

/* v rounded to `bits` significant bits; subnormal results below 2^emin keep
 * the absolute quantum 2^(emin - bits + 1) */
static double round_bits(double v, int bits, int emin)
{
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    frexp(v, &e); /* |v| = m 2^e, 1/2 <= m < 1: the leading bit has weight 2^(e-1) */
    int lead = e - 1;
    if (lead < emin) lead = emin;
    const int sh = bits - 1 - lead; /* scale that puts the last kept bit at weight 1 */
    return ldexp(nearbyint(ldexp(v, sh)), -sh);
}

double orc_round_store(int kind, double g)
{
    switch (kind) {
    case ORC_STORE_F32: return (double)(float)g;
    case ORC_STORE_BF16: return round_bits((double)(float)g, 8, -126);
    case ORC_STORE_F16: {
        const double v = round_bits((double)(float)g * 16384.0, 11, -14);
        return fabs(v) > 65504.0 ? copysign(INFINITY, v) : v / 16384.0;
    }
    default: return g;
    }
}

/* ------------------------------------------------------------ simulation */

typedef struct {
    int kind, motion, nv;
    double *x, *y, *xp, *yp; /* X^n, X^{n-1} */
    double *l0, *th0;        /* stress-free element lengths, turning angles */
    double A0, P0, ks, kb, ka, rho_b, mv;
    /* rigid state */
    double xc, yc, ang, u1x, u1y, u2x, u2y, w1, w2, mass, inertia;
    double *rx, *ry;
    /* adhesion */
    int nlig, nl0, adhesive;
    double sigma, ycr, yeq, kf_dt, kr0_dt, xi;
    int *lig_el, *bound;
    double *lig_t, *ax, *ay, *margin;
    /* per-step records (diagnostics) */
    double *uvx, *uvy;                  /* interpolated fluid velocity at vertices */
    double *fsx, *fsy, *fbx, *fby, *fax, *fay, *fpx, *fpy, *fwx, *fwy, *fhx, *fhy;
    double *ftx, *fty;                  /* total vertex force */
    double *vx, *vy;                    /* structure vertex velocity at n+1 */
    double *mx, *my, *mfx, *mfy, *mds;  /* markers at n+1, direct force, ds */
    double area, perim, cx, cy;         /* geometry at n+1 */
} orc_body;

typedef struct orc_sim {
    int nx, ny, bc, nb, diverged, transfer;
    int store_round; /* ORC_STORE_*: rounding of the stored deviations after each collision */
    double tau, nu, umax, rho_out, gx, gy, dcut, probe;
    uint64_t seed;
    int64_t step;
    double *f, *fs, *rho, *ux, *uy, *Fx, *Fy;
    orc_body b[ORC_MAX_BODIES];
    double obs[6]; /* step, t*, delta_p, r, N_L, n_bound */
} orc_sim;

static double* zalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

orc_sim* orc_create(int nx, int ny, double tau, double re, double rho_out, int bc, double gx, double gy,
                    uint64_t seed)
{
    lattice_init();
    if (nx < 3 || ny < 2 || !(tau > 0.5)) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->nx = nx;
    s->ny = ny;
    s->bc = bc;
    s->tau = tau;
    s->nu = CS2 * (tau - 0.5); /* Sec. 2.1 */
    s->umax = re * s->nu / ny; /* Re = u_max H / nu, Sec. 3.1 */
    s->rho_out = rho_out;
    s->gx = gx;
    s->gy = gy;
    s->seed = seed;
    s->dcut = 2.0;
    s->probe = 1.2; /* Sec. 2.6 */
    size_t n = (size_t)nx * ny;
    s->f = zalloc(ORC_Q * n);
    s->fs = zalloc(ORC_Q * n);
    s->rho = zalloc(n);
    s->ux = zalloc(n);
    s->uy = zalloc(n);
    s->Fx = zalloc(n);
    s->Fy = zalloc(n);
    /* initial post-collision state: equilibrium at rho = 1 with the inlet
     * profile (inlet/outlet) or at rest (periodic) */
    for (int y = 0; y < ny; ++y) {
        double u0 = (bc == ORC_BC_INLET_OUTLET) ? inlet_u(y + 0.5, (double)ny, s->umax) : 0.0;
        double feq[ORC_Q];
        orc_equilibrium(1.0, u0, 0.0, feq);
        for (int x = 0; x < nx; ++x)
            for (int q = 0; q < ORC_Q; ++q) s->f[q * n + (size_t)y * nx + x] = feq[q];
    }
    for (size_t k = 0; k < n; ++k) s->rho[k] = 1.0;
    return s;
}

static void body_free(orc_body* b)
{
    double** ptrs[] = {&b->x,   &b->y,   &b->xp,  &b->yp,  &b->l0,  &b->th0, &b->rx,  &b->ry,  &b->lig_t,
                       &b->ax,  &b->ay,  &b->margin, &b->uvx, &b->uvy, &b->fsx, &b->fsy, &b->fbx, &b->fby,
                       &b->fax, &b->fay, &b->fpx, &b->fpy, &b->fwx, &b->fwy, &b->fhx, &b->fhy, &b->ftx, &b->fty,
                       &b->vx,  &b->vy,  &b->mx,  &b->my,  &b->mfx, &b->mfy, &b->mds};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) {
        free(*ptrs[i]);
        *ptrs[i] = NULL;
    }
    free(b->lig_el);
    free(b->bound);
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    for (int k = 0; k < s->nb; ++k) body_free(&s->b[k]);
    free(s->f);
    free(s->fs);
    free(s->rho);
    free(s->ux);
    free(s->uy);
    free(s->Fx);
    free(s->Fy);
    free(s);
}

void orc_set_repulsion_cutoff(orc_sim* s, double d) { s->dcut = d; }

/* Stores the post-collision deviations in the given precision from now on
 * (the current state is rounded at once); -1 for an unknown kind. */
int orc_set_storage_rounding(orc_sim* s, int kind)
{
    if (kind < ORC_STORE_EXACT || kind > ORC_STORE_F16) return -1;
    lattice_init();
    s->store_round = kind;
    const size_t n = (size_t)s->nx * s->ny;
    for (int q = 0; q < ORC_Q; ++q)
        for (size_t k = 0; k < n; ++k) s->f[q * n + k] = WQ[q] + orc_round_store(kind, s->f[q * n + k] - WQ[q]);
    return 0;
}

/* Selects the transfer kernel (ORC_TRANSFER_*) of the interpolation and the
 * spreading; returns -1 for an unknown kind. */
int orc_set_transfer(orc_sim* s, int kind)
{
    if (kind != ORC_TRANSFER_PESKIN && kind != ORC_TRANSFER_MLS) return -1;
    s->transfer = kind;
    return 0;
}

/* Adds a closed counter-clockwise chain.  xy: interleaved (x0, y0, x1, ...);
 * xy_ref: stress-free shape or NULL.  k_s = rho nu u_max / Ca (Sec. 3.1),
 * k_b = beta k_s (Sec. 2.3).  Returns the body index or -1. */
int orc_add_body(orc_sim* s, int kind, int motion, int nv, const double* xy, const double* xy_ref, double ca,
                 double beta, double ka, double density_ratio)
{
    if (s->nb >= ORC_MAX_BODIES || nv < 3) return -1;
    if (motion == ORC_DEFORMABLE && !(ca > 0.0)) return -1;
    orc_body* b = &s->b[s->nb];
    memset(b, 0, sizeof(*b));
    b->kind = kind;
    b->motion = motion;
    b->nv = nv;
    double** arrs[] = {&b->x,   &b->y,   &b->xp,  &b->yp,  &b->l0,  &b->th0, &b->rx,  &b->ry,  &b->uvx,
                       &b->uvy, &b->fsx, &b->fsy, &b->fbx, &b->fby, &b->fax, &b->fay, &b->fpx, &b->fpy,
                       &b->fwx, &b->fwy, &b->fhx, &b->fhy, &b->ftx, &b->fty, &b->vx,  &b->vy,  &b->mx,
                       &b->my,  &b->mfx, &b->mfy, &b->mds};
    for (size_t i = 0; i < sizeof(arrs) / sizeof(arrs[0]); ++i) *arrs[i] = zalloc(nv);
    for (int v = 0; v < nv; ++v) {
        b->x[v] = b->xp[v] = xy[2 * v];
        b->y[v] = b->yp[v] = xy[2 * v + 1];
    }
    double *xr = zalloc(nv), *yr = zalloc(nv);
    for (int v = 0; v < nv; ++v) {
        xr[v] = xy_ref ? xy_ref[2 * v] : xy[2 * v];
        yr[v] = xy_ref ? xy_ref[2 * v + 1] : xy[2 * v + 1];
    }
    double *len = zalloc(nv), *nlx = zalloc(nv), *nly = zalloc(nv);
    chain_geometry(nv, xr, yr, len, nlx, nly, NULL, NULL, b->th0);
    for (int l = 0; l < nv; ++l) b->l0[l] = len[l];
    double poly[5];
    orc_polygon(nv, xr, yr, poly);
    b->A0 = poly[0];
    b->P0 = poly[1];
    b->ks = (motion == ORC_DEFORMABLE) ? 1.0 * s->nu * s->umax / ca : 0.0;
    b->kb = beta * b->ks;
    b->ka = ka;
    b->rho_b = density_ratio;
    b->mv = density_ratio * b->A0 / nv; /* Sec. 2.8: mass spread evenly on the vertices */
    orc_polygon(nv, b->x, b->y, poly);
    b->mass = density_ratio * poly[0];
    b->inertia = density_ratio * poly[4];
    b->xc = poly[2];
    b->yc = poly[3];
    for (int v = 0; v < nv; ++v) {
        b->rx[v] = b->x[v] - b->xc;
        b->ry[v] = b->y[v] - b->yc;
    }
    b->area = poly[0];
    b->perim = poly[1];
    b->cx = poly[2];
    b->cy = poly[3];
    free(xr);
    free(yr);
    free(len);
    free(nlx);
    free(nly);
    return s->nb++;
}

static double wall_gap(const orc_sim* s, double y) { return fmin(y, s->ny - y); }

/* Ligand sites equally spaced in arc length along the chain (Sec. 2.5 and
 * Sec. 3.1); sites within y_cr of a wall at t = 0 start bound (Sec. 3.3). */
int orc_set_adhesion(orc_sim* s, int body, int nlig, double sigma, double ycr, double yeq, double kf_dt,
                     double kr0_dt, double xi)
{
    if (body < 0 || body >= s->nb || nlig <= 0) return -1;
    orc_body* b = &s->b[body];
    b->adhesive = 1;
    b->nlig = nlig;
    b->sigma = isinf(sigma) ? sigma : sigma * 1.0 * s->nu * s->nu / s->ny; /* units rho nu^2 / H */
    b->ycr = ycr;
    b->yeq = yeq;
    b->kf_dt = kf_dt;
    b->kr0_dt = kr0_dt;
    b->xi = xi;
    b->lig_el = (int*)calloc(nlig, sizeof(int));
    b->bound = (int*)calloc(nlig, sizeof(int));
    b->lig_t = zalloc(nlig);
    b->ax = zalloc(nlig);
    b->ay = zalloc(nlig);
    b->margin = zalloc(nlig);
    int nv = b->nv;
    double P = 0.0;
    for (int l = 0; l < nv; ++l) P += hypot(b->x[(l + 1) % nv] - b->x[l], b->y[(l + 1) % nv] - b->y[l]);
    int l = 0;
    double acc = 0.0;
    for (int k = 0; k < nlig; ++k) {
        double sk = (k + 0.5) * P / nlig;
        for (;;) {
            double L = hypot(b->x[(l + 1) % nv] - b->x[l], b->y[(l + 1) % nv] - b->y[l]);
            if (sk <= acc + L || l == nv - 1) {
                b->lig_el[k] = l;
                double t = (sk - acc) / L;
                b->lig_t[k] = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
                break;
            }
            acc += L;
            ++l;
        }
    }
    b->nl0 = 0;
    for (int k = 0; k < nlig; ++k) {
        int a = b->lig_el[k], c = (a + 1) % nv;
        double px = b->x[a] + b->lig_t[k] * (b->x[c] - b->x[a]);
        double py = b->y[a] + b->lig_t[k] * (b->y[c] - b->y[a]);
        if (wall_gap(s, py) < ycr) {
            b->bound[k] = 1;
            b->ax[k] = px;
            b->ay[k] = (py < s->ny - py) ? 0.0 : (double)s->ny;
            b->nl0++;
        }
    }
    return 0;
}

/* Overwrite / read the stored post-collision populations, layout [q][y][x]. */
void orc_set_fpost(orc_sim* s, const double* f) { memcpy(s->f, f, sizeof(double) * ORC_Q * s->nx * s->ny); }
void orc_get_fpost(const orc_sim* s, double* f) { memcpy(f, s->f, sizeof(double) * ORC_Q * s->nx * s->ny); }
void orc_get_macro(const orc_sim* s, double* rho, double* ux, double* uy)
{
    size_t n = (size_t)s->nx * s->ny;
    memcpy(rho, s->rho, sizeof(double) * n);
    memcpy(ux, s->ux, sizeof(double) * n);
    memcpy(uy, s->uy, sizeof(double) * n);
}
void orc_set_macro(orc_sim* s, const double* rho, const double* ux, const double* uy)
{
    size_t n = (size_t)s->nx * s->ny;
    memcpy(s->rho, rho, sizeof(double) * n);
    memcpy(s->ux, ux, sizeof(double) * n);
    memcpy(s->uy, uy, sizeof(double) * n);
}
void orc_get_force(const orc_sim* s, double* fx, double* fy)
{
    size_t n = (size_t)s->nx * s->ny;
    memcpy(fx, s->Fx, sizeof(double) * n);
    memcpy(fy, s->Fy, sizeof(double) * n);
}
double orc_umax(const orc_sim* s) { return s->umax; }
int64_t orc_step_count(const orc_sim* s) { return s->step; }
int orc_diverged(const orc_sim* s) { return s->diverged; }
void orc_get_obs(const orc_sim* s, double* out) { memcpy(out, s->obs, sizeof(s->obs)); }

/* Body arrays by field id (see the Python wrapper for the list). */
int orc_get_body(const orc_sim* s, int body, int field, double* out)
{
    if (body < 0 || body >= s->nb) return -1;
    const orc_body* b = &s->b[body];
    const double* a[] = {b->x,   b->y,   b->xp,  b->yp,  b->uvx, b->uvy, b->fsx, b->fsy, b->fbx, b->fby,
                         b->fax, b->fay, b->fpx, b->fpy, b->fwx, b->fwy, b->fhx, b->fhy, b->ftx, b->fty,
                         b->vx,  b->vy,  b->mx,  b->my,  b->mfx, b->mfy, b->mds};
    int na = (int)(sizeof(a) / sizeof(a[0]));
    if (field < 0 || field >= na) return -1;
    memcpy(out, a[field], sizeof(double) * b->nv);
    return b->nv;
}

/* Scalars: {A0, P0, ks, kb, mv, mass, inertia, xc, yc, ang, area, perim, cx, cy, sigma, nl0} */
void orc_get_body_scalars(const orc_sim* s, int body, double* out)
{
    const orc_body* b = &s->b[body];
    double v[] = {b->A0,   b->P0,    b->ks, b->kb,   b->mv,    b->mass, b->inertia, b->xc,
                  b->yc,   b->ang,   b->area, b->perim, b->cx,   b->cy,   b->sigma,   (double)b->nl0};
    memcpy(out, v, sizeof(v));
}

int orc_get_bonds(const orc_sim* s, int body, int* bound, double* ax, double* ay, double* margin)
{
    const orc_body* b = &s->b[body];
    for (int k = 0; k < b->nlig; ++k) {
        bound[k] = b->bound[k];
        ax[k] = b->ax[k];
        ay[k] = b->ay[k];
        margin[k] = b->margin[k];
    }
    return b->nlig;
}

/* Pressure and viscous traction of every element from a probe 1.2 dx along
 * the outward normal (Eqs. 14-15, Sec. 2.6): p = c_s^2 rho - p_ref and
 * tau = rho nu (grad u + grad u^T).  A probe that would leave the channel is
 * stopped at the wall it crosses. */
static void body_traction(const orc_sim* s, const orc_body* b, const double* len, const double* nlx,
                          const double* nly, double* fex, double* fey)
{
    int nv = b->nv;
    for (int l = 0; l < nv; ++l) {
        int w = (l + 1) % nv;
        double cx = 0.5 * (b->x[l] + b->x[w]), cy = 0.5 * (b->y[l] + b->y[w]);
        double px = cx + s->probe * nlx[l], py = cy + s->probe * nly[l];
        fex[l] = fey[l] = 0.0;
        if (py < 0.0) py = 0.0; /* a probe that would cross a wall stops at it */
        if (py > s->ny) py = (double)s->ny;
        double rho, u, v, ux, uy, vx, vy;
        double W = interp_kind(s->transfer, s->nx, s->ny, s->rho, px, py, &rho, NULL, NULL, 1);
        if (!(W > 0.0)) continue;
        interp_kind(s->transfer, s->nx, s->ny, s->ux, px, py, &u, &ux, &uy, 0);
        interp_kind(s->transfer, s->nx, s->ny, s->uy, px, py, &v, &vx, &vy, 0);
        double p = CS2 * rho - CS2 * 1.0;
        double mu = rho * s->nu;
        double txx = 2.0 * mu * ux, txy = mu * (uy + vx), tyy = 2.0 * mu * vy;
        fex[l] = (-p * nlx[l] + txx * nlx[l] + txy * nly[l]) * len[l];
        fey[l] = (-p * nly[l] + txy * nlx[l] + tyy * nly[l]) * len[l];
    }
}

/* Element tractions of body `body` on the current macroscopic fields. */
void orc_body_traction(const orc_sim* s, int body, double* fex, double* fey)
{
    const orc_body* b = &s->b[body];
    int nv = b->nv;
    double *len = zalloc(nv), *nlx = zalloc(nv), *nly = zalloc(nv);
    chain_geometry(nv, b->x, b->y, len, nlx, nly, NULL, NULL, NULL);
    body_traction(s, b, len, nlx, nly, fex, fey);
    free(len);
    free(nlx);
    free(nly);
}

/* Global ligand-site id: sites of earlier bodies first. */
static uint32_t site_base(const orc_sim* s, int body)
{
    uint32_t base = 0;
    for (int k = 0; k < body; ++k) base += (uint32_t)(s->b[k].adhesive ? s->b[k].nlig : 0);
    return base;
}

/* Ligand-receptor kinetics (Sec. 2.5) and the resulting element forces
 * (Eq. 13) of one body at positions X^n. */
static void body_bonds(orc_sim* s, int bi, const double* nlx, const double* nly, double* fex, double* fey)
{
    orc_body* b = &s->b[bi];
    int nv = b->nv;
    for (int l = 0; l < nv; ++l) fex[l] = fey[l] = 0.0;
    if (!b->adhesive) return;
    uint32_t base = site_base(s, bi);
    double Pf = 1.0 - exp(-b->kf_dt);
    for (int k = 0; k < b->nlig; ++k) {
        int a = b->lig_el[k], c = (a + 1) % nv;
        double px = b->x[a] + b->lig_t[k] * (b->x[c] - b->x[a]);
        double py = b->y[a] + b->lig_t[k] * (b->y[c] - b->y[a]);
        if (b->motion != ORC_FIXED) {
            double u = orc_bond_uniform(s->seed, s->step, base + (uint32_t)k);
            if (b->bound[k]) {
                double yl = hypot(px - b->ax[k], py - b->ay[k]);
                double kr = b->kr0_dt * exp(b->xi * (yl - b->yeq) * (yl - b->yeq));
                double Pr = 1.0 - exp(-kr);
                b->margin[k] = fabs(u - Pr);
                if (u < Pr) b->bound[k] = 0;
            } else if (wall_gap(s, py) < b->ycr) {
                b->margin[k] = fabs(u - Pf);
                if (u < Pf) {
                    b->bound[k] = 1;
                    b->ax[k] = px;
                    b->ay[k] = (py < s->ny - py) ? 0.0 : (double)s->ny;
                }
            }
        }
        if (b->bound[k] && !isinf(b->sigma)) {
            /* Eq. 13: a linear spring, F = sigma (y_l - y_eq) along n_l, the unit
             * vector from the ligand site to its receptor (the element's outward
             * normal for a bond perpendicular to the wall under a base element);
             * the element normal if the site sits on its anchor */
            double dx = b->ax[k] - px, dy = b->ay[k] - py;
            double yl = hypot(dx, dy);
            double F = b->sigma * (yl - b->yeq);
            double ex = (yl > 0.0) ? dx / yl : nlx[a], ey = (yl > 0.0) ? dy / yl : nly[a];
            fex[a] += F * ex;
            fey[a] += F * ey;
        }
    }
}

/* Eq. 12: repulsion on every vertex of body bi from the vertices of every
 * other body closer than the cut-off, along bi's own inward vertex normal. */
static void body_repulsion(const orc_sim* s, int bi, const double* nvx, const double* nvy, double* fx, double* fy)
{
    const orc_body* b = &s->b[bi];
    for (int v = 0; v < b->nv; ++v) {
        fx[v] = fy[v] = 0.0;
        for (int o = 0; o < s->nb; ++o) {
            if (o == bi) continue;
            const orc_body* c = &s->b[o];
            for (int w = 0; w < c->nv; ++w) {
                double d = hypot(b->x[v] - c->x[w], b->y[v] - c->y[w]);
                if (d < s->dcut) {
                    double m = orc_repulsion_magnitude(d);
                    fx[v] += m * (-nvx[v]);
                    fy[v] += m * (-nvy[v]);
                }
            }
        }
    }
}

/* One time step, in the order listed in the file header. */
void orc_step(orc_sim* s)
{
    int nx = s->nx, ny = s->ny;
    size_t n = (size_t)nx * ny;
    /* 1. streaming + boundary conditions */
    orc_stream_bc(nx, ny, s->bc, s->umax, s->rho_out, s->f, s->fs);
    /* 2.-3. moments (Eqs. 5-6) and collision (Eqs. 1, 2, 4) */
    int diverged = 0;
#pragma omp parallel for schedule(static) reduction(| : diverged)
    for (size_t k = 0; k < n; ++k) {
        double fk[ORC_Q], feq[ORC_Q], gq[ORC_Q];
        double rho = 0.0, jx = 0.0, jy = 0.0;
        for (int q = 0; q < ORC_Q; ++q) {
            fk[q] = s->fs[q * n + k];
            rho += fk[q];
            jx += fk[q] * EX[q];
            jy += fk[q] * EY[q];
        }
        double Fx = s->Fx[k] + s->gx, Fy = s->Fy[k] + s->gy;
        double ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho;
        s->rho[k] = rho;
        s->ux[k] = ux;
        s->uy[k] = uy;
        if (!(rho > 0.0) || !isfinite(ux) || !isfinite(uy)) diverged = 1;
        orc_equilibrium(rho, ux, uy, feq);
        orc_guo_term(ux, uy, Fx, Fy, s->tau, gq);
        for (int q = 0; q < ORC_Q; ++q) s->f[q * n + k] = fk[q] - (fk[q] - feq[q]) / s->tau + gq[q];
        if (s->store_round)
            for (int q = 0; q < ORC_Q; ++q)
                s->f[q * n + k] = WQ[q] + orc_round_store(s->store_round, s->f[q * n + k] - WQ[q]);
    }
    if (diverged) s->diverged = 1;
    /* 4. Lagrangian update from (rho^n, u^n) at X^n */
    int nb = s->nb;
    double *len[ORC_MAX_BODIES], *nlx[ORC_MAX_BODIES], *nly[ORC_MAX_BODIES], *nvx[ORC_MAX_BODIES],
        *nvy[ORC_MAX_BODIES], *th[ORC_MAX_BODIES];
    for (int bi = 0; bi < nb; ++bi) {
        orc_body* b = &s->b[bi];
        int nv = b->nv;
        len[bi] = zalloc(nv);
        nlx[bi] = zalloc(nv);
        nly[bi] = zalloc(nv);
        nvx[bi] = zalloc(nv);
        nvy[bi] = zalloc(nv);
        th[bi] = zalloc(nv);
        chain_geometry(nv, b->x, b->y, len[bi], nlx[bi], nly[bi], nvx[bi], nvy[bi], th[bi]);
        /* tentative vertex velocity: fluid velocity at the vertex (Eq. 17) */
        for (int v = 0; v < nv; ++v) {
            interp_kind(s->transfer, nx, ny, s->ux, b->x[v], b->y[v], &b->uvx[v], NULL, NULL, 0);
            interp_kind(s->transfer, nx, ny, s->uy, b->x[v], b->y[v], &b->uvy[v], NULL, NULL, 0);
        }
    }
    for (int bi = 0; bi < nb; ++bi) {
        orc_body* b = &s->b[bi];
        int nv = b->nv;
        double *ewx = zalloc(nv), *ewy = zalloc(nv), *ehx = zalloc(nv), *ehy = zalloc(nv);
        body_bonds(s, bi, nlx[bi], nly[bi], ewx, ewy);
        body_traction(s, b, len[bi], nlx[bi], nly[bi], ehx, ehy);
        body_repulsion(s, bi, nvx[bi], nvy[bi], b->fpx, b->fpy);
        if (b->motion == ORC_DEFORMABLE) {
            orc_membrane_forces(nv, b->x, b->y, b->l0, b->th0, b->A0, b->ks, b->kb, b->ka, CS2 * 1.0, b->fsx,
                                b->fsy, b->fbx, b->fby, b->fax, b->fay);
        } else {
            for (int v = 0; v < nv; ++v) b->fsx[v] = b->fsy[v] = b->fbx[v] = b->fby[v] = b->fax[v] = b->fay[v] = 0.0;
        }
        for (int v = 0; v < nv; ++v) {
            int lm = (v + nv - 1) % nv;
            b->fwx[v] = 0.5 * (ewx[lm] + ewx[v]);
            b->fwy[v] = 0.5 * (ewy[lm] + ewy[v]);
            b->fhx[v] = 0.5 * (ehx[lm] + ehx[v]);
            b->fhy[v] = 0.5 * (ehy[lm] + ehy[v]);
            b->ftx[v] = b->fsx[v] + b->fbx[v] + b->fax[v] + b->fpx[v] + b->fwx[v] + b->fhx[v];
            b->fty[v] = b->fsy[v] + b->fby[v] + b->fay[v] + b->fpy[v] + b->fwy[v] + b->fhy[v];
        }
        free(ewx);
        free(ewy);
        free(ehx);
        free(ehy);
    }
    /* integration: all forces above used X^n of every body */
    for (int bi = 0; bi < nb; ++bi) {
        orc_body* b = &s->b[bi];
        int nv = b->nv;
        if (b->motion == ORC_DEFORMABLE) {
            for (int v = 0; v < nv; ++v) {
                /* Eq. 17 (dt = 1) then Eq. 18 */
                double xn = b->x[v] + b->uvx[v] + 0.5 * b->ftx[v] / b->mv;
                double yn = b->y[v] + b->uvy[v] + 0.5 * b->fty[v] / b->mv;
                b->vx[v] = 1.5 * xn - 2.0 * b->x[v] + 0.5 * b->xp[v];
                b->vy[v] = 1.5 * yn - 2.0 * b->y[v] + 0.5 * b->yp[v];
                b->xp[v] = b->x[v];
                b->yp[v] = b->y[v];
                b->x[v] = xn;
                b->y[v] = yn;
            }
        } else if (b->motion == ORC_RIGID) {
            double Fx = 0.0, Fy = 0.0, M = 0.0;
            for (int v = 0; v < nv; ++v) {
                Fx += b->ftx[v];
                Fy += b->fty[v];
                M += (b->x[v] - b->xc) * b->fty[v] - (b->y[v] - b->yc) * b->ftx[v];
            }
            /* Eq. 19 */
            double ux = orc_rigid_bdf2(b->u1x, b->u2x, Fx / b->mass);
            double uy = orc_rigid_bdf2(b->u1y, b->u2y, Fy / b->mass);
            double w = orc_rigid_bdf2(b->w1, b->w2, M / b->inertia);
            b->u2x = b->u1x;
            b->u1x = ux;
            b->u2y = b->u1y;
            b->u1y = uy;
            b->w2 = b->w1;
            b->w1 = w;
            b->xc += ux;
            b->yc += uy;
            b->ang += w;
            double c = cos(b->ang), sn = sin(b->ang);
            for (int v = 0; v < nv; ++v) {
                double rx = c * b->rx[v] - sn * b->ry[v], ry = sn * b->rx[v] + c * b->ry[v];
                b->xp[v] = b->x[v];
                b->yp[v] = b->y[v];
                b->x[v] = b->xc + rx;
                b->y[v] = b->yc + ry;
                b->vx[v] = ux - w * ry;
                b->vy[v] = uy + w * rx;
            }
        } else {
            for (int v = 0; v < nv; ++v) {
                b->xp[v] = b->x[v];
                b->yp[v] = b->y[v];
                b->vx[v] = b->vy[v] = 0.0;
            }
        }
    }
    /* 5. direct forcing at the new element centroids and spreading */
    for (size_t k = 0; k < n; ++k) s->Fx[k] = s->Fy[k] = 0.0;
    for (int bi = 0; bi < nb; ++bi) {
        orc_body* b = &s->b[bi];
        int nv = b->nv;
        for (int l = 0; l < nv; ++l) {
            int w = (l + 1) % nv;
            double cx = 0.5 * (b->x[l] + b->x[w]), cy = 0.5 * (b->y[l] + b->y[w]);
            double usx = 0.5 * (b->vx[l] + b->vx[w]), usy = 0.5 * (b->vy[l] + b->vy[w]);
            double rho, ux, uy;
            double W = interp_kind(s->transfer, nx, ny, s->rho, cx, cy, &rho, NULL, NULL, 1);
            interp_kind(s->transfer, nx, ny, s->ux, cx, cy, &ux, NULL, NULL, 0);
            interp_kind(s->transfer, nx, ny, s->uy, cx, cy, &uy, NULL, NULL, 0);
            b->mx[l] = cx;
            b->my[l] = cy;
            b->mds[l] = hypot(b->x[w] - b->x[l], b->y[w] - b->y[l]);
            /* a marker within half a spacing of a wall is held by the wall's
             * bounce-back condition and is not forced */
            int held = (cy < 0.5 || cy > ny - 0.5);
            b->mfx[l] = (W > 0.0 && !held) ? rho * (usx - ux) : 0.0;
            b->mfy[l] = (W > 0.0 && !held) ? rho * (usy - uy) : 0.0;
        }
        orc_spread(nx, ny, nv, b->mx, b->my, b->mfx, b->mfy, b->mds, s->Fx, s->Fy, s->transfer);
        double poly[5];
        orc_polygon(nv, b->x, b->y, poly);
        b->area = poly[0];
        b->perim = poly[1];
        b->cx = poly[2];
        b->cy = poly[3];
        for (int v = 0; v < nv; ++v)
            if (!isfinite(b->x[v]) || !isfinite(b->y[v])) s->diverged = 1;
    }
    for (int bi = 0; bi < nb; ++bi) {
        free(len[bi]);
        free(nlx[bi]);
        free(nly[bi]);
        free(nvx[bi]);
        free(nvy[bi]);
        free(th[bi]);
    }
    s->step += 1;
    /* observables (Sec. 3.1): delta_p of the first cell, r between the first
     * cell and the first particle, N_L over all adhesive bodies */
    int ic = -1, ip = -1, nbound = 0, nl0 = 0;
    for (int bi = 0; bi < nb; ++bi) {
        if (s->b[bi].kind == ORC_CELL && ic < 0) ic = bi;
        if (s->b[bi].kind == ORC_PARTICLE && ip < 0) ip = bi;
        if (s->b[bi].adhesive) {
            nl0 += s->b[bi].nl0;
            for (int k = 0; k < s->b[bi].nlig; ++k) nbound += s->b[bi].bound[k];
        }
    }
    s->obs[0] = (double)s->step;
    s->obs[1] = (double)s->step * s->umax / ny;
    s->obs[2] = (ic >= 0) ? (s->b[ic].perim - s->b[ic].P0) / s->b[ic].P0 : NAN;
    s->obs[3] = (ic >= 0 && ip >= 0) ? hypot(s->b[ic].cx - s->b[ip].cx, s->b[ic].cy - s->b[ip].cy) : NAN;
    s->obs[4] = (nl0 > 0) ? (double)nbound / nl0 : NAN;
    s->obs[5] = (double)nbound;
}

void orc_run(orc_sim* s, int64_t nsteps)
{
    for (int64_t k = 0; k < nsteps; ++k) orc_step(s);
}
