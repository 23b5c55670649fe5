/*
 * dufwi_oracle.c -- plain FP64 CPU oracle for the damped 2-D acoustic
 * simulator and its misfit gradient (test infrastructure only).
 *
 * This file is the reference that the CUDA path is checked against. It is
 * deliberately slow and literal: every routine follows one passage of the
 * paper (arXiv 2603.04070, "Physics Informed Deep Unfolded Full Waveform
 * Inversion for Edema Detection") and nothing is blocked, fused or reordered
 * beyond what that passage states. It shares no code, header, table or
 * constant with the GPU library; only tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.
 *
 * Notation (paper Sec. II-A):
 *   C  speed of sound (m/s), D  damping profile (1/s), dt time step (s),
 *   dx grid spacing (m), U[t] field at time sample t, S[t] source term.
 * Grid layout: padded grid nzp x nxp, row-major [z][x] (x fastest).
 *   nxp = nx + 2P, nzp = nz + 2P, with P absorbing cells added on each side.
 *
 * Readings of points the paper leaves open (each is listed in the design
 * notes of the repository):
 *   - Eq. 2 prints the Laplacian coefficient as C^2 dt/(1+D dt); the
 *     dimensionally consistent coefficient, used here, is C^2 dt^2/(1+D dt).
 *   - The Laplacian "convolution kernel" of Eq. 2 is the textbook central
 *     second-difference stencil of order 2, 4, 6 or 8 along x plus the same
 *     along z, divided by dx^2, with zero field outside the padded grid.
 *   - The absorbing profile (Sec. IV) is quadratic, d(xi) = d0 (xi/L)^2,
 *     L = P dx, d0 = 3 c_ref ln(1/R) / (2L); D = d(xi_x) + d(xi_z), xi the
 *     depth into the layer (P - i) dx for layer index i (outermost i = 0).
 *     With c_ref = 1500 m/s, R = 1e-3, P = 20, dx = 0.1 m / 188 this gives
 *     the 1.46e6 printed in Sec. IV.
 *   - The SoS map covers the physical grid; inside the absorbing layer it is
 *     extended by edge replication, so the gradient of a padded cell is
 *     folded back onto the physical edge cell it copies.
 *   - Source: a point source w(t) at one node, S[t] = dt^2 w((t-1) dt)/dx^2,
 *     i.e. the step that produces U[t+1] adds dt^2 w[t]/dx^2 at the node.
 *   - Receivers record M[t][r] = U[t](x_r) for t = 0..nt-1, U[0] = U[-1] = 0.
 *   - Variable density (Eq. 1 with rho(x,z)): the density term
 *     rho div((1/rho) grad u) is discretised on a staggered grid,
 *     D-_x(b D+_x u) + D-_z(b D+_z u), divided by dx^2. D+ and D- are the
 *     textbook staggered first differences of the same order as the
 *     Laplacian; the buoyancy b = 1/rho at a half point is the inverse of the
 *     mean density of its two nodes; b = 0 at half points outside the padded
 *     grid. rho multiplies at the node: kappa = rho C^2 dt^2/(1 + D dt). The
 *     density is extended into the absorbing layer by edge replication. With
 *     no density array the compact Laplacian above is used (constant rho,
 *     which then drops out).
 *   - Absorbing boundary, alternative to the damping term D: a convolutional
 *     PML (CPML) on the same staggered operator. Each first difference is
 *     stretched by 1/s with s = 1 + d/(alpha + i omega) (kappa = 1), realised
 *     by one memory variable per difference and axis (recursive convolution
 *     with b = exp(-(d + alpha) dt), a = d (b - 1)/(d + alpha)):
 *       psi^n = b psi^{n-1} + a D+u^n,   F = b_rho (D+u^n + psi^n),
 *       xi^n  = b xi^{n-1} + a D-F,      G = D-F + xi^n,
 *     U^{n+1} = 2U^n - U^{n-1} + kappa G/dx^2 + s^n, kappa = rho C^2 dt^2.
 *     d(xi) = d0 (xi/L)^2 as for D, alpha(xi) = alpha_max (1 - xi/L) inside the
 *     layer, both 0 outside; profiles are evaluated at the nodes (xi) and at
 *     the half points (psi) of each axis. Without a density map, rho = 1.
 *   - Misfit J = sum over transmits, samples and receivers of
 *     (M_sim - M_obs)^2 (Eq. 5 data term, lambda = 0); g = dJ/dC (Eq. 6), the
 *     exact gradient of the discrete J, obtained with the discrete adjoint.
 *
 * Parity pins (tests marked "not gpu"): analytic 2-D Green's function trace,
 * source-receiver reciprocity, adjoint dot-product test, central finite
 * differences of J, the printed d0, stencil moment conditions, linearity and
 * time-shift equivariance, mirror symmetry, J = 0 and g = 0 at the truth.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, nz;          /* physical grid (cells) */
    double dx, dt;       /* m, s */
    int nt;              /* recorded samples t = 0..nt-1 */
    int pml;             /* absorbing cells per side (P) */
    double pml_R;        /* target reflection factor */
    double pml_cref;     /* reference SoS for d0 (m/s) */
    int fd_order;        /* 2, 4, 6 or 8 */
    int boundary;        /* 0: damping term D of Eq. 1; 1: convolutional PML (CPML) */
    double pml_alpha;    /* CPML frequency shift at the inner edge of the layer (1/s) */
} orc_problem;

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 5

/* ------------------------------------------------------------------ */
/* Laplacian stencil weights (the "convolution with a Laplacian kernel"
 * of Sec. II-A): c[k] multiplies u(x+k dx) + u(x-k dx) for k >= 1 and
 * c[0] multiplies u(x). Textbook central second-difference weights. */
int orc_fd_coeffs(int order, double *c)
{
    switch (order) {
    case 2:
        c[0] = -2.0; c[1] = 1.0;
        return ORC_OK;
    case 4:
        c[0] = -5.0 / 2.0; c[1] = 4.0 / 3.0; c[2] = -1.0 / 12.0;
        return ORC_OK;
    case 6:
        c[0] = -49.0 / 18.0; c[1] = 3.0 / 2.0; c[2] = -3.0 / 20.0;
        c[3] = 1.0 / 90.0;
        return ORC_OK;
    case 8:
        c[0] = -205.0 / 72.0; c[1] = 8.0 / 5.0; c[2] = -1.0 / 5.0;
        c[3] = 8.0 / 315.0; c[4] = -1.0 / 560.0;
        return ORC_OK;
    default:
        return ORC_EINVAL;
    }
}

static int padded_nx(const orc_problem *p) { return p->nx + 2 * p->pml; }
static int padded_nz(const orc_problem *p) { return p->nz + 2 * p->pml; }

/* Maximum damping of the quadratic layer (Sec. IV). */
double orc_d0(const orc_problem *p)
{
    double L = p->pml * p->dx;
    return 3.0 * p->pml_cref * log(1.0 / p->pml_R) / (2.0 * L);
}

/* Depth into the absorbing layer of padded index i along an axis with n
 * physical cells: (P - i) dx on the low side, (i - (P + n - 1)) dx on the
 * high side, 0 inside the physical grid. */
static double layer_depth(const orc_problem *p, int i, int n)
{
    int P = p->pml;
    if (i < P) return (double)(P - i) * p->dx;
    if (i > P + n - 1) return (double)(i - (P + n - 1)) * p->dx;
    return 0.0;
}

/* D(x,z) of Eq. 1 over the padded grid. */
int orc_damping(const orc_problem *p, double *D)
{
    int nxp = padded_nx(p), nzp = padded_nz(p);
    double L = p->pml * p->dx, d0 = orc_d0(p);
    for (int z = 0; z < nzp; ++z)
        for (int x = 0; x < nxp; ++x) {
            double xi_x = layer_depth(p, x, p->nx) / L;
            double xi_z = layer_depth(p, z, p->nz) / L;
            D[(size_t)z * nxp + x] = d0 * xi_x * xi_x + d0 * xi_z * xi_z;
        }
    return ORC_OK;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* SoS on the padded grid: edge replication of the physical map. */
int orc_pad(const orc_problem *p, const double *C, double *Cpad)
{
    int nxp = padded_nx(p), nzp = padded_nz(p), P = p->pml;
    for (int z = 0; z < nzp; ++z)
        for (int x = 0; x < nxp; ++x) {
            int zs = clampi(z - P, 0, p->nz - 1), xs = clampi(x - P, 0, p->nx - 1);
            Cpad[(size_t)z * nxp + x] = C[(size_t)zs * p->nx + xs];
        }
    return ORC_OK;
}

/* The three element-wise coefficient maps of Eq. 2:
 *   a = (2 - D^2 dt^2)/(1 + D dt), b = (D dt - 1)/(1 + D dt),
 *   kappa = rho C^2 dt^2/(1 + D dt)  (rho = 1 without a density map). */
static void coefficient_maps(const orc_problem *p, const double *Cpad, const double *rho_pad, const double *D,
                             double *a, double *b, double *kappa)
{
    size_t n = (size_t)padded_nx(p) * padded_nz(p);
    double dt = p->dt;
    for (size_t i = 0; i < n; ++i) {
        double den = 1.0 + D[i] * dt;
        a[i] = (2.0 - D[i] * D[i] * dt * dt) / den;
        b[i] = (D[i] * dt - 1.0) / den;
        kappa[i] = (rho_pad ? rho_pad[i] : 1.0) * Cpad[i] * Cpad[i] * dt * dt / den;
    }
}

/* out = Laplacian of u on the padded grid (Sec. II-A), zero outside. */
int orc_laplacian(const orc_problem *p, const double *u, double *out)
{
    int nxp = padded_nx(p), nzp = padded_nz(p);
    int h = p->fd_order / 2;
    double c[5];
    if (orc_fd_coeffs(p->fd_order, c) != ORC_OK) return ORC_EINVAL;
    double inv_dx2 = 1.0 / (p->dx * p->dx);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nzp; ++z)
        for (int x = 0; x < nxp; ++x) {
            double s = 0.0;
            for (int k = -h; k <= h; ++k) {
                double w = c[k < 0 ? -k : k];
                if (x + k >= 0 && x + k < nxp) s += w * u[(size_t)z * nxp + (x + k)];
                if (z + k >= 0 && z + k < nzp) s += w * u[(size_t)(z + k) * nxp + x];
            }
            out[(size_t)z * nxp + x] = s * inv_dx2;
        }
    return ORC_OK;
}

/* Staggered first-difference weights of order 2, 4, 6 or 8: s[k-1]
 * multiplies u(x + (k - 1/2) dx) - u(x - (k - 1/2) dx), k = 1..order/2
 * (the Taylor weights of the centred derivative on a half-shifted grid). */
int orc_stagger_coeffs(int order, double *s)
{
    switch (order) {
    case 2:
        s[0] = 1.0;
        return ORC_OK;
    case 4:
        s[0] = 9.0 / 8.0; s[1] = -1.0 / 24.0;
        return ORC_OK;
    case 6:
        s[0] = 75.0 / 64.0; s[1] = -25.0 / 384.0; s[2] = 3.0 / 640.0;
        return ORC_OK;
    case 8:
        s[0] = 1225.0 / 1024.0; s[1] = -245.0 / 3072.0; s[2] = 49.0 / 5120.0;
        s[3] = -5.0 / 7168.0;
        return ORC_OK;
    default:
        return ORC_EINVAL;
    }
}

/* Buoyancy at the half points of the padded grid:
 *   bx[z][x] = b at (x + 1/2, z) = 2 / (rho[z][x] + rho[z][x+1]),  x < nxp - 1
 *   bz[z][x] = b at (x, z + 1/2) = 2 / (rho[z][x] + rho[z+1][x]),  z < nzp - 1
 * and 0 at the half point past the last node of each row or column. */
int orc_buoyancy(const orc_problem *p, const double *rho, double *bx, double *bz)
{
    int nxp = padded_nx(p), nzp = padded_nz(p);
    for (int z = 0; z < nzp; ++z)
        for (int x = 0; x < nxp; ++x) {
            size_t i = (size_t)z * nxp + x;
            bx[i] = x < nxp - 1 ? 2.0 / (rho[i] + rho[i + 1]) : 0.0;
            bz[i] = z < nzp - 1 ? 2.0 / (rho[i] + rho[i + nxp]) : 0.0;
        }
    return ORC_OK;
}

/* u at (z, x) with zero outside the padded grid. */
static double u_at(const double *u, int nxp, int nzp, int z, int x)
{
    return (x >= 0 && x < nxp && z >= 0 && z < nzp) ? u[(size_t)z * nxp + x] : 0.0;
}

/* Flux b D+u at the x half point (j + 1/2, z), zero where b is outside. */
static double flux_x(const double *bx, const double *u, int nxp, int nzp, const double *s, int h, int z, int j)
{
    if (j < 0 || j >= nxp) return 0.0;
    double d = 0.0;
    for (int k = 1; k <= h; ++k) d += s[k - 1] * (u_at(u, nxp, nzp, z, j + k) - u_at(u, nxp, nzp, z, j - k + 1));
    return bx[(size_t)z * nxp + j] * d;
}

static double flux_z(const double *bz, const double *u, int nxp, int nzp, const double *s, int h, int j, int x)
{
    if (j < 0 || j >= nzp) return 0.0;
    double d = 0.0;
    for (int k = 1; k <= h; ++k) d += s[k - 1] * (u_at(u, nxp, nzp, j + k, x) - u_at(u, nxp, nzp, j - k + 1, x));
    return bz[(size_t)j * nxp + x] * d;
}

/* out = (1/dx^2) [D-_x (bx D+_x u) + D-_z (bz D+_z u)] on the padded grid:
 * D- of a flux f at node x is sum_k s_k (f(x + k - 1/2) - f(x - k + 1/2)). */
int orc_div_b_grad(const orc_problem *p, const double *bx, const double *bz, const double *u, double *out)
{
    int nxp = padded_nx(p), nzp = padded_nz(p);
    int h = p->fd_order / 2;
    double s[4];
    if (orc_stagger_coeffs(p->fd_order, s) != ORC_OK) return ORC_EINVAL;
    double inv_dx2 = 1.0 / (p->dx * p->dx);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nzp; ++z)
        for (int x = 0; x < nxp; ++x) {
            double acc = 0.0;
            for (int k = 1; k <= h; ++k) {
                acc += s[k - 1] * (flux_x(bx, u, nxp, nzp, s, h, z, x + k - 1) - flux_x(bx, u, nxp, nzp, s, h, z, x - k));
                acc += s[k - 1] * (flux_z(bz, u, nxp, nzp, s, h, z + k - 1, x) - flux_z(bz, u, nxp, nzp, s, h, z - k, x));
            }
            out[(size_t)z * nxp + x] = acc * inv_dx2;
        }
    return ORC_OK;
}

/* The spatial operator of one simulation: the compact Laplacian (constant
 * density), or the staggered density operator when bx, bz are given. */
typedef struct {
    const double *bx, *bz;
} orc_op;

static void apply_op(const orc_problem *p, const orc_op *op, const double *u, double *out)
{
    if (op && op->bx) orc_div_b_grad(p, op->bx, op->bz, u, out);
    else orc_laplacian(p, u, out);
}

/* One application of Eq. 2 without the source:
 *   next = a*cur + b*prev + kappa*lap(cur). lapc receives lap(cur). */
static void eq2_step(const orc_problem *p, const orc_op *op, const double *a, const double *b,
                     const double *kappa, const double *cur, const double *prev,
                     double *next, double *lapc)
{
    size_t n = (size_t)padded_nx(p) * padded_nz(p);
    apply_op(p, op, cur, lapc);
    for (size_t i = 0; i < n; ++i)
        next[i] = a[i] * cur[i] + b[i] * prev[i] + kappa[i] * lapc[i];
}

static int node_index(const orc_problem *p, int ix, int iz, size_t *out)
{
    if (ix < 0 || ix >= p->nx || iz < 0 || iz >= p->nz) return ORC_EINVAL;
    *out = (size_t)(iz + p->pml) * padded_nx(p) + (size_t)(ix + p->pml);
    return ORC_OK;
}

static int valid_problem(const orc_problem *p)
{
    double c[5];
    if (p->nx < 1 || p->nz < 1 || p->nt < 1 || p->pml < 1) return 0;
    if (p->boundary != 0 && p->boundary != 1) return 0;
    if (p->boundary == 1 && !(p->pml_alpha >= 0.0)) return 0;
    if (!(p->dx > 0) || !(p->dt > 0) || !(p->pml_R > 0 && p->pml_R < 1) || !(p->pml_cref > 0)) return 0;
    return orc_fd_coeffs(p->fd_order, c) == ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Convolutional PML (see the header notes). */

/* Depth (m) into the absorbing layer of position pos (padded index; half
 * points at j + 0.5) along an axis with n physical cells. */
static double depth_at(const orc_problem *p, double pos, int n)
{
    double P = p->pml, hi = P + n - 1;
    if (pos < P) return (P - pos) * p->dx;
    if (pos > hi) return (pos - hi) * p->dx;
    return 0.0;
}

/* Recursion coefficients at depth xi: b = exp(-(d + alpha) dt), a = d (b - 1)/(d + alpha). */
static void cpml_ab(const orc_problem *p, double xi, double *a, double *b)
{
    double L = p->pml * p->dx;
    if (xi <= 0.0) { *a = 0.0; *b = 1.0; return; }
    double d = orc_d0(p) * (xi / L) * (xi / L);
    double al = p->pml_alpha * (1.0 - xi / L);
    *b = exp(-(d + al) * p->dt);
    *a = d > 0.0 ? d * (*b - 1.0) / (d + al) : 0.0;
}

/* Coefficient tables along x (length nxp) and z (length nzp): nodes (n) and
 * half points j + 1/2 (h). */
int orc_cpml_coeffs(const orc_problem *p, double *anx, double *bnx, double *ahx, double *bhx,
                    double *anz, double *bnz, double *ahz, double *bhz)
{
    for (int i = 0; i < padded_nx(p); ++i) {
        cpml_ab(p, depth_at(p, i, p->nx), &anx[i], &bnx[i]);
        cpml_ab(p, depth_at(p, i + 0.5, p->nx), &ahx[i], &bhx[i]);
    }
    for (int i = 0; i < padded_nz(p); ++i) {
        cpml_ab(p, depth_at(p, i, p->nz), &anz[i], &bnz[i]);
        cpml_ab(p, depth_at(p, i + 0.5, p->nz), &ahz[i], &bhz[i]);
    }
    return ORC_OK;
}

typedef struct {
    double s[4];
    double *anx, *bnx, *ahx, *bhx, *anz, *bnz, *ahz, *bhz;
    double *Fx, *Fz;       /* scratch: half-point fluxes (or their adjoints) */
    double *ex, *ez;       /* scratch: node values */
} orc_cpml;

static void cpml_free(orc_cpml *c)
{
    free(c->anx); free(c->Fx); free(c->ex);
    memset(c, 0, sizeof(*c));
}

static int cpml_init(const orc_problem *p, orc_cpml *c)
{
    memset(c, 0, sizeof(*c));
    int nxp = padded_nx(p), nzp = padded_nz(p);
    size_t n = (size_t)nxp * nzp;
    if (orc_stagger_coeffs(p->fd_order, c->s) != ORC_OK) return ORC_EINVAL;
    c->anx = malloc(sizeof(double) * 4 * (size_t)(nxp + nzp));
    c->Fx = malloc(sizeof(double) * 2 * n);
    c->ex = malloc(sizeof(double) * 2 * n);
    if (!c->anx || !c->Fx || !c->ex) { cpml_free(c); return ORC_ENOMEM; }
    c->bnx = c->anx + nxp; c->ahx = c->bnx + nxp; c->bhx = c->ahx + nxp;
    c->anz = c->bhx + nxp; c->bnz = c->anz + nzp; c->ahz = c->bnz + nzp; c->bhz = c->ahz + nzp;
    c->Fz = c->Fx + n;
    c->ez = c->ex + n;
    orc_cpml_coeffs(p, c->anx, c->bnx, c->ahx, c->bhx, c->anz, c->bnz, c->ahz, c->bhz);
    return ORC_OK;
}

/* Value of a half-point or node array at (z, x), zero outside the padded grid. */
static double at0(const double *v, int nxp, int nzp, int z, int x)
{
    return (x >= 0 && x < nxp && z >= 0 && z < nzp) ? v[(size_t)z * nxp + x] : 0.0;
}

/* CPML operator at step n: G = (1/dx^2) sum over axes of (D-F + xi), F = b (D+u + psi), with
 * psi and xi advanced in place to their step-n values. */
static void cpml_apply(const orc_problem *p, orc_cpml *c, const double *bx, const double *bz, const double *u,
                       double *psx, double *psz, double *xix, double *xiz, double *G)
{
    int nxp = padded_nx(p), nzp = padded_nz(p), h = p->fd_order / 2;
    double inv_dx2 = 1.0 / (p->dx * p->dx);
    for (int z = 0; z < nzp; ++z)
        for (int j = 0; j < nxp; ++j) {
            size_t i = (size_t)z * nxp + j;
            double d = 0.0;
            for (int k = 1; k <= h; ++k) d += c->s[k - 1] * (at0(u, nxp, nzp, z, j + k) - at0(u, nxp, nzp, z, j - k + 1));
            psx[i] = c->bhx[j] * psx[i] + c->ahx[j] * d;
            c->Fx[i] = bx[i] * (d + psx[i]);
            double dz = 0.0;
            for (int k = 1; k <= h; ++k) dz += c->s[k - 1] * (at0(u, nxp, nzp, z + k, j) - at0(u, nxp, nzp, z - k + 1, j));
            psz[i] = c->bhz[z] * psz[i] + c->ahz[z] * dz;
            c->Fz[i] = bz[i] * (dz + psz[i]);
        }
    for (int z = 0; z < nzp; ++z)
        for (int x = 0; x < nxp; ++x) {
            size_t i = (size_t)z * nxp + x;
            double ex = 0.0, ez = 0.0;
            for (int k = 1; k <= h; ++k) {
                ex += c->s[k - 1] * (at0(c->Fx, nxp, nzp, z, x + k - 1) - at0(c->Fx, nxp, nzp, z, x - k));
                ez += c->s[k - 1] * (at0(c->Fz, nxp, nzp, z + k - 1, x) - at0(c->Fz, nxp, nzp, z - k, x));
            }
            xix[i] = c->bnx[x] * xix[i] + c->anx[x] * ex;
            xiz[i] = c->bnz[z] * xiz[i] + c->anz[z] * ez;
            G[i] = (ex + xix[i] + ez + xiz[i]) * inv_dx2;
        }
}

/* Reverse of cpml_apply (the transpose of the forward statements in reverse order). Input: Gbar =
 * the adjoint of G; the adjoints of the step-n memory variables in psxb, pszb, xixb, xizb, which
 * leave holding those of step n - 1. Output: out = the adjoint of u (D+^T of the flux adjoints). */
static void cpml_reverse(const orc_problem *p, orc_cpml *c, const double *bx, const double *bz, const double *Gbar,
                         double *psxb, double *pszb, double *xixb, double *xizb, double *out)
{
    int nxp = padded_nx(p), nzp = padded_nz(p), h = p->fd_order / 2;
    double inv_dx2 = 1.0 / (p->dx * p->dx);
    /* G = (ex + xix + ez + xiz)/dx^2 and xi = b xi + a e */
    for (int z = 0; z < nzp; ++z)
        for (int x = 0; x < nxp; ++x) {
            size_t i = (size_t)z * nxp + x;
            double g = Gbar[i] * inv_dx2;
            double tx = xixb[i] + g, tz = xizb[i] + g;
            c->ex[i] = g + c->anx[x] * tx;
            c->ez[i] = g + c->anz[z] * tz;
            xixb[i] = c->bnx[x] * tx;
            xizb[i] = c->bnz[z] * tz;
        }
    /* e = D-F: Fbar_j = sum_k s_k (ebar_{j-k+1} - ebar_{j+k}); F = b (d + psi); psi = b_h psi + a_h d */
    for (int z = 0; z < nzp; ++z)
        for (int j = 0; j < nxp; ++j) {
            size_t i = (size_t)z * nxp + j;
            double fx = 0.0, fz = 0.0;
            for (int k = 1; k <= h; ++k) {
                fx += c->s[k - 1] * (at0(c->ex, nxp, nzp, z, j - k + 1) - at0(c->ex, nxp, nzp, z, j + k));
                fz += c->s[k - 1] * (at0(c->ez, nxp, nzp, z - k + 1, j) - at0(c->ez, nxp, nzp, z + k, j));
            }
            double px = psxb[i] + bx[i] * fx, pz = pszb[i] + bz[i] * fz;
            c->Fx[i] = bx[i] * fx + c->ahx[j] * px;     /* adjoint of d (x) */
            c->Fz[i] = bz[i] * fz + c->ahz[z] * pz;
            psxb[i] = c->bhx[j] * px;
            pszb[i] = c->bhz[z] * pz;
        }
    /* d = D+u: ubar_i = sum_k s_k (dbar_{i-k} - dbar_{i+k-1}) */
    for (int z = 0; z < nzp; ++z)
        for (int x = 0; x < nxp; ++x) {
            double acc = 0.0;
            for (int k = 1; k <= h; ++k) {
                acc += c->s[k - 1] * (at0(c->Fx, nxp, nzp, z, x - k) - at0(c->Fx, nxp, nzp, z, x + k - 1));
                acc += c->s[k - 1] * (at0(c->Fz, nxp, nzp, z - k, x) - at0(c->Fz, nxp, nzp, z + k - 1, x));
            }
            out[(size_t)z * nxp + x] = acc;
        }
}

/* Density of one map on the padded grid and its half-point buoyancies
 * (rho == NULL: constant density, compact Laplacian). */
typedef struct {
    double *rho_pad, *bx, *bz;
    orc_op op;
} orc_medium;

static void medium_free(orc_medium *m)
{
    free(m->rho_pad); free(m->bx); free(m->bz);
    memset(m, 0, sizeof(*m));
}

static int medium_init(const orc_problem *p, const double *rho, orc_medium *m)
{
    memset(m, 0, sizeof(*m));
    if (!rho) return ORC_OK;
    for (size_t i = 0; i < (size_t)p->nx * p->nz; ++i)
        if (!(rho[i] > 0.0) || !isfinite(rho[i])) return ORC_EINVAL;
    size_t n = (size_t)padded_nx(p) * padded_nz(p);
    m->rho_pad = malloc(n * sizeof(double));
    m->bx = malloc(n * sizeof(double));
    m->bz = malloc(n * sizeof(double));
    if (!m->rho_pad || !m->bx || !m->bz) { medium_free(m); return ORC_ENOMEM; }
    orc_pad(p, rho, m->rho_pad);
    orc_buoyancy(p, m->rho_pad, m->bx, m->bz);
    m->op.bx = m->bx;
    m->op.bz = m->bz;
    return ORC_OK;
}

/* CPML medium: the given density, or rho = 1 (buoyancy 1 between nodes). */
static int cpml_medium(const orc_problem *p, const double *rho, orc_medium *m)
{
    if (rho) return medium_init(p, rho, m);
    size_t n = (size_t)p->nx * p->nz;
    double *ones = malloc(n * sizeof(double));
    if (!ones) return ORC_ENOMEM;
    for (size_t i = 0; i < n; ++i) ones[i] = 1.0;
    int rc = medium_init(p, ones, m);
    free(ones);
    return rc;
}

/* kappa = rho C^2 dt^2 on the padded grid (the CPML replaces the damping term). */
static void cpml_kappa(const orc_problem *p, const double *Cpad, const double *rho_pad, double *kap)
{
    size_t n = (size_t)padded_nx(p) * padded_nz(p);
    for (size_t i = 0; i < n; ++i) kap[i] = rho_pad[i] * Cpad[i] * Cpad[i] * p->dt * p->dt;
}

/* Forward model with the CPML: traces [nt][n_rx] of a point source at (sx, sz). */
static int cpml_forward(const orc_problem *p, const double *C, const double *rho, int sx, int sz, const double *w,
                        int n_rx, const int *rx_ix, const int *rx_iz, double *traces)
{
    size_t n = (size_t)padded_nx(p) * padded_nz(p), src;
    if (node_index(p, sx, sz, &src)) return ORC_EINVAL;
    orc_medium med;
    orc_cpml cp;
    int rc = cpml_medium(p, rho, &med);
    if (rc) return rc;
    if ((rc = cpml_init(p, &cp))) { medium_free(&med); return rc; }
    size_t *rx = malloc(sizeof(size_t) * (n_rx > 0 ? n_rx : 1));
    double *buf = calloc(n * 10, sizeof(double));
    if (!rx || !buf) { rc = ORC_ENOMEM; goto done; }
    for (int r = 0; r < n_rx; ++r)
        if (node_index(p, rx_ix[r], rx_iz[r], &rx[r])) { rc = ORC_EINVAL; goto done; }
    double *Cpad = buf, *kap = buf + n, *prev = buf + 2 * n, *cur = buf + 3 * n, *next = buf + 4 * n;
    double *G = buf + 5 * n, *psx = buf + 6 * n, *psz = buf + 7 * n, *xix = buf + 8 * n, *xiz = buf + 9 * n;
    orc_pad(p, C, Cpad);
    cpml_kappa(p, Cpad, med.rho_pad, kap);
    double src_scale = p->dt * p->dt / (p->dx * p->dx);
    for (int t = 0; t < p->nt; ++t) {
        for (int r = 0; r < n_rx; ++r) traces[(size_t)t * n_rx + r] = cur[rx[r]];
        if (t == p->nt - 1) break;
        cpml_apply(p, &cp, med.bx, med.bz, cur, psx, psz, xix, xiz, G);
        for (size_t i = 0; i < n; ++i) next[i] = 2.0 * cur[i] - prev[i] + kap[i] * G[i];
        next[src] += src_scale * w[t];
        double *tmp = prev; prev = cur; cur = next; next = tmp;
    }
done:
    free(rx); free(buf); cpml_free(&cp); medium_free(&med);
    return rc;
}

/* Adjoint fields with the CPML (reverse of cpml_forward's recursion), driven by receiver series
 * q[nt][n_rx]; returns lam[t] at the probe node. */
static int cpml_adjoint_probe(const orc_problem *p, const double *C, const double *rho, int n_rx, const int *rx_ix,
                              const int *rx_iz, const double *q, int px, int pz, double *lam_probe)
{
    size_t n = (size_t)padded_nx(p) * padded_nz(p), probe;
    if (node_index(p, px, pz, &probe)) return ORC_EINVAL;
    orc_medium med;
    orc_cpml cp;
    int rc = cpml_medium(p, rho, &med);
    if (rc) return rc;
    if ((rc = cpml_init(p, &cp))) { medium_free(&med); return rc; }
    size_t *rx = malloc(sizeof(size_t) * (n_rx > 0 ? n_rx : 1));
    double *buf = calloc(n * 11, sizeof(double));
    if (!rx || !buf) { rc = ORC_ENOMEM; goto done; }
    for (int r = 0; r < n_rx; ++r)
        if (node_index(p, rx_ix[r], rx_iz[r], &rx[r])) { rc = ORC_EINVAL; goto done; }
    double *Cpad = buf, *kap = buf + n, *l2 = buf + 2 * n, *l1 = buf + 3 * n, *l0 = buf + 4 * n;
    double *Gb = buf + 5 * n, *out = buf + 6 * n, *psxb = buf + 7 * n, *pszb = buf + 8 * n;
    double *xixb = buf + 9 * n, *xizb = buf + 10 * n;
    orc_pad(p, C, Cpad);
    cpml_kappa(p, Cpad, med.rho_pad, kap);
    for (int t = p->nt - 1; t >= 0; --t) {
        /* reverse of the step that produced U[t+1] from U[t] */
        for (size_t i = 0; i < n; ++i) Gb[i] = kap[i] * l1[i];
        cpml_reverse(p, &cp, med.bx, med.bz, Gb, psxb, pszb, xixb, xizb, out);
        for (size_t i = 0; i < n; ++i) l0[i] = 2.0 * l1[i] - l2[i] + out[i];
        for (int r = 0; r < n_rx; ++r) l0[rx[r]] += q[(size_t)t * n_rx + r];
        lam_probe[t] = l0[probe];
        double *tmp = l2; l2 = l1; l1 = l0; l0 = tmp;
    }
done:
    free(rx); free(buf); cpml_free(&cp); medium_free(&med);
    return rc;
}

/* Misfit and gradient with the CPML (all G^t kept; the adjoint runs the reverse recursion). */
static int cpml_misfit_gradient(const orc_problem *p, const double *C, const double *rho, int n_tx, const int *tx_ix,
                                const int *tx_iz, const double *wavelet, int n_wav, int n_rx, const int *rx_ix,
                                const int *rx_iz, const double *M_obs, double *J, double *g, double *M_sim)
{
    int nxp = padded_nx(p), nzp = padded_nz(p), nt = p->nt;
    size_t n = (size_t)nxp * nzp;
    orc_medium med;
    orc_cpml cp;
    int rc = cpml_medium(p, rho, &med);
    if (rc) return rc;
    if ((rc = cpml_init(p, &cp))) { medium_free(&med); return rc; }
    size_t *rx = malloc(sizeof(size_t) * (n_rx > 0 ? n_rx : 1));
    double *buf = calloc(n * 17, sizeof(double));
    double *hist = calloc(n * (size_t)(nt > 1 ? nt - 1 : 1), sizeof(double));
    double *trace = calloc((size_t)nt * (n_rx > 0 ? n_rx : 1), sizeof(double));
    double *q = calloc((size_t)nt * (n_rx > 0 ? n_rx : 1), sizeof(double));
    if (!rx || !buf || !hist || !trace || !q) { rc = ORC_ENOMEM; goto done; }
    double *Cpad = buf, *kap = buf + n, *prev = buf + 2 * n, *cur = buf + 3 * n, *next = buf + 4 * n;
    double *psx = buf + 5 * n, *psz = buf + 6 * n, *xix = buf + 7 * n, *xiz = buf + 8 * n;
    double *l2 = buf + 9 * n, *l1 = buf + 10 * n, *l0 = buf + 11 * n, *Gb = buf + 12 * n, *out = buf + 13 * n;
    double *gpad = buf + 14 * n, *xixb = buf + 15 * n, *xizb = buf + 16 * n;
    double *psxb = psx, *pszb = psz;     /* reused after the forward sweep */
    orc_pad(p, C, Cpad);
    cpml_kappa(p, Cpad, med.rho_pad, kap);
    double src_scale = p->dt * p->dt / (p->dx * p->dx), Jsum = 0.0;
    for (int tx = 0; tx < n_tx && rc == ORC_OK; ++tx) {
        size_t src;
        const double *w = wavelet + (size_t)(n_wav == 1 ? 0 : tx) * nt;
        if (node_index(p, tx_ix[tx], tx_iz[tx], &src)) { rc = ORC_EINVAL; break; }
        for (int r = 0; r < n_rx; ++r)
            if (node_index(p, rx_ix[(size_t)tx * n_rx + r], rx_iz[(size_t)tx * n_rx + r], &rx[r])) rc = ORC_EINVAL;
        if (rc) break;
        memset(prev, 0, n * sizeof(double)); memset(cur, 0, n * sizeof(double));
        memset(psx, 0, n * sizeof(double)); memset(psz, 0, n * sizeof(double));
        memset(xix, 0, n * sizeof(double)); memset(xiz, 0, n * sizeof(double));
        for (int t = 0; t < nt; ++t) {
            for (int r = 0; r < n_rx; ++r) trace[(size_t)t * n_rx + r] = cur[rx[r]];
            if (t == nt - 1) break;
            double *G = hist + (size_t)t * n;             /* G^t, used by the step producing U[t+1] */
            cpml_apply(p, &cp, med.bx, med.bz, cur, psx, psz, xix, xiz, G);
            for (size_t i = 0; i < n; ++i) next[i] = 2.0 * cur[i] - prev[i] + kap[i] * G[i];
            next[src] += src_scale * w[t];
            double *tmp = prev; prev = cur; cur = next; next = tmp;
        }
        const double *obs = M_obs + (size_t)tx * nt * n_rx;
        for (size_t i = 0; i < (size_t)nt * n_rx; ++i) {
            double r = trace[i] - obs[i];
            Jsum += r * r;
            q[i] = 2.0 * r;
        }
        if (M_sim) memcpy(M_sim + (size_t)tx * nt * n_rx, trace, sizeof(double) * (size_t)nt * n_rx);
        memset(l1, 0, n * sizeof(double)); memset(l2, 0, n * sizeof(double));
        memset(psxb, 0, n * sizeof(double)); memset(pszb, 0, n * sizeof(double));
        memset(xixb, 0, n * sizeof(double)); memset(xizb, 0, n * sizeof(double));
        for (int t = nt - 1; t >= 1; --t) {
            for (size_t i = 0; i < n; ++i) Gb[i] = kap[i] * l1[i];
            cpml_reverse(p, &cp, med.bx, med.bz, Gb, psxb, pszb, xixb, xizb, out);
            for (size_t i = 0; i < n; ++i) l0[i] = 2.0 * l1[i] - l2[i] + out[i];
            for (int r = 0; r < n_rx; ++r) l0[rx[r]] += q[(size_t)t * n_rx + r];
            const double *G = hist + (size_t)(t - 1) * n;  /* lam[t] pairs with G^{t-1} */
            for (size_t i = 0; i < n; ++i) gpad[i] += l0[i] * G[i];
            double *tmp = l2; l2 = l1; l1 = l0; l0 = tmp;
        }
    }
    if (rc == ORC_OK) {
        for (size_t i = 0; i < n; ++i) gpad[i] *= 2.0 * med.rho_pad[i] * Cpad[i] * p->dt * p->dt;
        memset(g, 0, sizeof(double) * (size_t)p->nx * p->nz);
        for (int z = 0; z < nzp; ++z)
            for (int x = 0; x < nxp; ++x) {
                int zs = clampi(z - p->pml, 0, p->nz - 1), xs = clampi(x - p->pml, 0, p->nx - 1);
                g[(size_t)zs * p->nx + xs] += gpad[(size_t)z * nxp + x];
            }
        *J = Jsum;
    }
done:
    free(rx); free(buf); free(hist); free(trace); free(q); cpml_free(&cp); medium_free(&med);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Forward model of one transmit, Eqs. 2-3: a point source at (sx, sz)
 * driven by w[0..nt-1], traces M[t][r] = U[t] at the receivers. */
int orc_forward_rho(const orc_problem *p, const double *C, const double *rho,
                    int sx, int sz, const double *w,
                    int n_rx, const int *rx_ix, const int *rx_iz,
                    double *traces /* [nt][n_rx] */)
{
    if (!valid_problem(p)) return ORC_EINVAL;
    if (p->boundary == 1) return cpml_forward(p, C, rho, sx, sz, w, n_rx, rx_ix, rx_iz, traces);
    orc_medium med;
    int mrc = medium_init(p, rho, &med);
    if (mrc) return mrc;
    size_t n = (size_t)padded_nx(p) * padded_nz(p), src;
    if (node_index(p, sx, sz, &src)) return ORC_EINVAL;
    size_t *rx = malloc(sizeof(size_t) * (n_rx > 0 ? n_rx : 1));
    double *buf = calloc(n * 9, sizeof(double));
    if (!rx || !buf) { free(rx); free(buf); medium_free(&med); return ORC_ENOMEM; }
    for (int r = 0; r < n_rx; ++r)
        if (node_index(p, rx_ix[r], rx_iz[r], &rx[r])) { free(rx); free(buf); medium_free(&med); return ORC_EINVAL; }
    double *D = buf, *Cpad = buf + n, *a = buf + 2 * n, *b = buf + 3 * n, *kap = buf + 4 * n;
    double *prev = buf + 5 * n, *cur = buf + 6 * n, *next = buf + 7 * n, *lap = buf + 8 * n;
    orc_damping(p, D);
    orc_pad(p, C, Cpad);
    coefficient_maps(p, Cpad, med.rho_pad, D, a, b, kap);
    double src_scale = p->dt * p->dt / (p->dx * p->dx);

    for (int t = 0; t < p->nt; ++t) {
        /* cur holds U[t] */
        for (int r = 0; r < n_rx; ++r) traces[(size_t)t * n_rx + r] = cur[rx[r]];
        if (t == p->nt - 1) break;
        eq2_step(p, &med.op, a, b, kap, cur, prev, next, lap);
        next[src] += src_scale * w[t];
        double *tmp = prev; prev = cur; cur = next; next = tmp;
    }
    free(rx); free(buf); medium_free(&med);
    return ORC_OK;
}

int orc_forward(const orc_problem *p, const double *C,
                int sx, int sz, const double *w,
                int n_rx, const int *rx_ix, const int *rx_iz,
                double *traces /* [nt][n_rx] */)
{
    return orc_forward_rho(p, C, NULL, sx, sz, w, n_rx, rx_ix, rx_iz, traces);
}

/* ------------------------------------------------------------------ */
/* Discrete adjoint of Eq. 2 (exact transpose of the forward recursion).
 * With q[t][r] the derivative of the objective w.r.t. M[t][r], the adjoint
 * fields lam[t] (t = nt-1 .. 1) obey
 *   lam[t] = R^T q[t] + a*lam[t+1] + Lap(kappa*lam[t+1]) + b*lam[t+2],
 *   lam[nt] = lam[nt+1] = 0,
 * because the Laplacian with zero exterior is a symmetric matrix. The
 * staggered density operator is symmetric too: it is -G^T B G with G the
 * D+ differences (zero exterior) and B the diagonal of half-point buoyancies,
 * since D- = -G^T. */
static void adjoint_step(const orc_problem *p, const orc_op *op, const double *a, const double *b,
                         const double *kappa, const double *lam1, const double *lam2,
                         double *lam0, double *work, double *lapw)
{
    size_t n = (size_t)padded_nx(p) * padded_nz(p);
    for (size_t i = 0; i < n; ++i) work[i] = kappa[i] * lam1[i];
    apply_op(p, op, work, lapw);
    for (size_t i = 0; i < n; ++i)
        lam0[i] = a[i] * lam1[i] + lapw[i] + b[i] * lam2[i];
}

/* Adjoint fields driven by receiver series q[nt][n_rx]; returns lam[t] at
 * one probe node for t = 0..nt-1 (lam[0] included for completeness).
 * For a source w at the probe node, <F w, q> = sum_t w[t] dt^2/dx^2 lam[t+1]. */
int orc_adjoint_probe_rho(const orc_problem *p, const double *C, const double *rho,
                          int n_rx, const int *rx_ix, const int *rx_iz, const double *q,
                          int px, int pz, double *lam_probe /* [nt] */)
{
    if (!valid_problem(p)) return ORC_EINVAL;
    if (p->boundary == 1) return cpml_adjoint_probe(p, C, rho, n_rx, rx_ix, rx_iz, q, px, pz, lam_probe);
    orc_medium med;
    int mrc = medium_init(p, rho, &med);
    if (mrc) return mrc;
    size_t n = (size_t)padded_nx(p) * padded_nz(p), probe;
    if (node_index(p, px, pz, &probe)) return ORC_EINVAL;
    size_t *rx = malloc(sizeof(size_t) * (n_rx > 0 ? n_rx : 1));
    double *buf = calloc(n * 10, sizeof(double));
    if (!rx || !buf) { free(rx); free(buf); medium_free(&med); return ORC_ENOMEM; }
    for (int r = 0; r < n_rx; ++r)
        if (node_index(p, rx_ix[r], rx_iz[r], &rx[r])) { free(rx); free(buf); medium_free(&med); return ORC_EINVAL; }
    double *D = buf, *Cpad = buf + n, *a = buf + 2 * n, *b = buf + 3 * n, *kap = buf + 4 * n;
    double *l2 = buf + 5 * n, *l1 = buf + 6 * n, *l0 = buf + 7 * n, *work = buf + 8 * n, *lapw = buf + 9 * n;
    orc_damping(p, D);
    orc_pad(p, C, Cpad);
    coefficient_maps(p, Cpad, med.rho_pad, D, a, b, kap);
    /* l1 = lam[t+1], l2 = lam[t+2] */
    for (int t = p->nt - 1; t >= 0; --t) {
        adjoint_step(p, &med.op, a, b, kap, l1, l2, l0, work, lapw);
        for (int r = 0; r < n_rx; ++r) l0[rx[r]] += q[(size_t)t * n_rx + r];
        lam_probe[t] = l0[probe];
        double *tmp = l2; l2 = l1; l1 = l0; l0 = tmp;
    }
    free(rx); free(buf); medium_free(&med);
    return ORC_OK;
}

int orc_adjoint_probe(const orc_problem *p, const double *C,
                      int n_rx, const int *rx_ix, const int *rx_iz, const double *q,
                      int px, int pz, double *lam_probe /* [nt] */)
{
    return orc_adjoint_probe_rho(p, C, NULL, n_rx, rx_ix, rx_iz, q, px, pz, lam_probe);
}

/* ------------------------------------------------------------------ */
/* Misfit and gradient of one SoS map over n_tx transmits (Eqs. 5-6).
 *
 *   J = sum_p sum_t sum_r (M_sim[p][t][r] - M_obs[p][t][r])^2
 *   g = dJ/dC on the physical grid.
 *
 * dJ/dkappa = sum_{t=1}^{nt-1} lam[t] * Lap(U[t-1]) (kappa multiplies
 * Lap(U[t-1]) in the step producing U[t]); dkappa/dC = 2 C dt^2/(1 + D dt);
 * the padded-grid gradient is then summed onto the physical cell each padded
 * cell replicates. The forward fields needed by the adjoint sweep are kept
 * as snapshots (U[t], U[t-1]) every `ckpt` samples and recomputed segment by
 * segment in FP64, which reproduces them exactly; ckpt >= nt keeps them all.
 *
 * wavelet: [n_wav][nt] with n_wav = 1 (shared) or n_tx (one per transmit).
 * rx_ix, rx_iz: [n_tx][n_rx]. M_obs: [n_tx][nt][n_rx]. M_sim (optional
 * output): [n_tx][nt][n_rx]. g: [nz][nx]. */
int orc_misfit_gradient_rho(const orc_problem *p, const double *C, const double *rho,
                            int n_tx, const int *tx_ix, const int *tx_iz,
                            const double *wavelet, int n_wav,
                            int n_rx, const int *rx_ix, const int *rx_iz,
                            const double *M_obs, int ckpt,
                            double *J, double *g, double *M_sim)
{
    if (!valid_problem(p) || n_tx < 1 || n_rx < 0 || (n_wav != 1 && n_wav != n_tx)) return ORC_EINVAL;
    if (p->boundary == 1)
        return cpml_misfit_gradient(p, C, rho, n_tx, tx_ix, tx_iz, wavelet, n_wav, n_rx, rx_ix, rx_iz, M_obs, J, g,
                                    M_sim);
    orc_medium med;
    int mrc = medium_init(p, rho, &med);
    if (mrc) return mrc;
    int nxp = padded_nx(p), nzp = padded_nz(p), nt = p->nt;
    size_t n = (size_t)nxp * nzp;
    if (ckpt < 1 || ckpt > nt) ckpt = nt;
    int n_seg = (nt - 1 + ckpt - 1) / ckpt;     /* steps t -> t+1 for t = 0..nt-2 */
    if (n_seg < 1) n_seg = 1;

    double *base = calloc(n * 13, sizeof(double));
    double *snap = calloc((size_t)n_seg * 2 * n, sizeof(double));
    double *seg = calloc((size_t)(ckpt + 1) * n, sizeof(double));
    double *gpad = calloc(n, sizeof(double));
    double *trace = calloc((size_t)nt * (n_rx > 0 ? n_rx : 1), sizeof(double));
    double *q = calloc((size_t)nt * (n_rx > 0 ? n_rx : 1), sizeof(double));
    size_t *rx = malloc(sizeof(size_t) * (n_rx > 0 ? n_rx : 1));
    if (!base || !snap || !seg || !gpad || !trace || !q || !rx) {
        free(base); free(snap); free(seg); free(gpad); free(trace); free(q); free(rx);
        medium_free(&med);
        return ORC_ENOMEM;
    }
    double *D = base, *Cpad = base + n, *a = base + 2 * n, *b = base + 3 * n, *kap = base + 4 * n;
    double *prev = base + 5 * n, *cur = base + 6 * n, *next = base + 7 * n, *lap = base + 8 * n;
    double *l2 = base + 9 * n, *l1 = base + 10 * n, *l0 = base + 11 * n, *work = base + 12 * n;
    orc_damping(p, D);
    orc_pad(p, C, Cpad);
    coefficient_maps(p, Cpad, med.rho_pad, D, a, b, kap);
    double src_scale = p->dt * p->dt / (p->dx * p->dx);
    double Jsum = 0.0;
    int status = ORC_OK;

    for (int tx = 0; tx < n_tx && status == ORC_OK; ++tx) {
        size_t src;
        const double *w = wavelet + (size_t)(n_wav == 1 ? 0 : tx) * nt;
        if (node_index(p, tx_ix[tx], tx_iz[tx], &src)) { status = ORC_EINVAL; break; }
        for (int r = 0; r < n_rx; ++r)
            if (node_index(p, rx_ix[(size_t)tx * n_rx + r], rx_iz[(size_t)tx * n_rx + r], &rx[r])) status = ORC_EINVAL;
        if (status) break;

        /* forward sweep: traces and snapshots (U[s*ckpt], U[s*ckpt-1]) */
        memset(prev, 0, n * sizeof(double));
        memset(cur, 0, n * sizeof(double));
        for (int t = 0; t < nt; ++t) {
            if (t % ckpt == 0 && t / ckpt < n_seg) {
                memcpy(snap + (size_t)(t / ckpt) * 2 * n, cur, n * sizeof(double));
                memcpy(snap + (size_t)(t / ckpt) * 2 * n + n, prev, n * sizeof(double));
            }
            for (int r = 0; r < n_rx; ++r) trace[(size_t)t * n_rx + r] = cur[rx[r]];
            if (t == nt - 1) break;
            eq2_step(p, &med.op, a, b, kap, cur, prev, next, lap);
            next[src] += src_scale * w[t];
            double *tmp = prev; prev = cur; cur = next; next = tmp;
        }
        /* residual and misfit; q[t][r] = dJ/dM_sim[t][r] = 2 (M_sim - M_obs) */
        const double *obs = M_obs + (size_t)tx * nt * n_rx;
        for (size_t i = 0; i < (size_t)nt * n_rx; ++i) {
            double r = trace[i] - obs[i];
            Jsum += r * r;
            q[i] = 2.0 * r;
        }
        if (M_sim) memcpy(M_sim + (size_t)tx * nt * n_rx, trace, sizeof(double) * (size_t)nt * n_rx);
        /* adjoint sweep, segment by segment from the last */
        memset(l1, 0, n * sizeof(double));
        memset(l2, 0, n * sizeof(double));
        int t_hi = nt - 1;                       /* next adjoint index to produce */
        for (int s = n_seg - 1; s >= 0; --s) {
            int t0 = s * ckpt;                   /* segment steps t0..t1-1 produce U[t0+1..t1] */
            int t1 = t0 + ckpt; if (t1 > nt - 1) t1 = nt - 1;
            /* seg[k] = U[t0 + k] for k = 0..t1-t0 */
            memcpy(seg, snap + (size_t)s * 2 * n, n * sizeof(double));
            memcpy(prev, snap + (size_t)s * 2 * n + n, n * sizeof(double));
            for (int t = t0; t < t1; ++t) {
                double *u_t = seg + (size_t)(t - t0) * n;
                double *u_prev = (t == t0) ? prev : seg + (size_t)(t - t0 - 1) * n;
                double *u_next = seg + (size_t)(t - t0 + 1) * n;
                eq2_step(p, &med.op, a, b, kap, u_t, u_prev, u_next, lap);
                u_next[src] += src_scale * w[t];
            }
            /* adjoint indices t = t_hi .. t0+1 pair with U[t-1] in this segment */
            for (int t = t_hi; t >= t0 + 1; --t) {
                adjoint_step(p, &med.op, a, b, kap, l1, l2, l0, work, lap);
                for (int r = 0; r < n_rx; ++r) l0[rx[r]] += q[(size_t)t * n_rx + r];
                apply_op(p, &med.op, seg + (size_t)(t - 1 - t0) * n, lap);
                for (size_t i = 0; i < n; ++i) gpad[i] += l0[i] * lap[i];
                double *tmp = l2; l2 = l1; l1 = l0; l0 = tmp;
            }
            t_hi = t0;
        }
    }
    if (status == ORC_OK) {
        /* chain rule through kappa = rho C^2 dt^2/(1 + D dt), then fold the padding */
        for (size_t i = 0; i < n; ++i)
            gpad[i] *= 2.0 * (med.rho_pad ? med.rho_pad[i] : 1.0) * Cpad[i] * p->dt * p->dt / (1.0 + D[i] * p->dt);
        memset(g, 0, sizeof(double) * (size_t)p->nx * p->nz);
        for (int z = 0; z < nzp; ++z)
            for (int x = 0; x < nxp; ++x) {
                int zs = clampi(z - p->pml, 0, p->nz - 1), xs = clampi(x - p->pml, 0, p->nx - 1);
                g[(size_t)zs * p->nx + xs] += gpad[(size_t)z * nxp + x];
            }
        *J = Jsum;
    }
    free(base); free(snap); free(seg); free(gpad); free(trace); free(q); free(rx);
    medium_free(&med);
    return status;
}

int orc_misfit_gradient(const orc_problem *p, const double *C,
                        int n_tx, const int *tx_ix, const int *tx_iz,
                        const double *wavelet, int n_wav,
                        int n_rx, const int *rx_ix, const int *rx_iz,
                        const double *M_obs, int ckpt,
                        double *J, double *g, double *M_sim)
{
    return orc_misfit_gradient_rho(p, C, NULL, n_tx, tx_ix, tx_iz, wavelet, n_wav, n_rx, rx_ix, rx_iz, M_obs,
                                   ckpt, J, g, M_sim);
}
