/*
 * hlbm_oracle.c -- TEST INFRASTRUCTURE, not product code.
 *
 * A plain, slow, FP64 CPU restatement of the improved compressible hybrid
 * lattice Boltzmann method (HLBM) of Renard, Feng, Boussuge and Sagaut,
 * "Improved compressible Hybrid Lattice Boltzmann Method on standard lattice
 * for subsonic and supersonic flows" (arXiv 2002.03644).  It is organised by
 * the equations it evaluates: the regularised collision and pull-streaming
 * of the D2Q9 populations (eq streamalgo, Sec. 3.3), their moments (eqs
 * rhoalgo, ualgo), the finite-volume entropy update (eq sequaalgo, Sec. 3.4)
 * and temperature recovery (eq Entropie expression, Sec. 2.4), the closure
 * correction psi (eq Psialgo, Sec. 3.2), the equilibrium (eq Equilibrium,
 * Sec. 2.3) and the off-equilibrium moment a1 (eqs a1sigalgo, a1FD,
 * Sec. 3.3).  One full array holds every intermediate quantity, and each is
 * computed by a straightforward loop over cells.
 *
 * Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * may load this library.  The CUDA library shares no code, header, table or
 * helper with it, and neither side imports the other.
 *
 * Units: lattice units, dx = dt = 1 (Sec. 2.1: variables made dimensionless
 * with T_r, rho_r, dx and dt = dx / C_0), so c_s^2 = 1/3 and D = 2.
 *
 * Readings of points the paper leaves open:
 *  - mu is a constant per case and tau = mu / p per cell (mu = tau p, Sec. 2.4).
 *  - E1 is diagonal: E1_xx = d_x Gamma_x, E1_yy = d_y Gamma_y, E1_xy = 0, with
 *    Gamma_y built like Gamma_x; sgn(0) = 0 (Sec. 3.2).
 *  - The MUSCL / Van Albada advection of s is written in non-conservative
 *    form u . grad s with cell-velocity upwinding (Sec. 3.4; see muscl_term).
 *  - Every quantity in the entropy right-hand side is taken at level n
 *    (the entropy equation is explicit in time); lambda = mu c_p / Pr is constant (the printed
 *    mu / (c_p Pr) contradicts the paper's own decay and Couette formulas).
 *  - Boundaries: a ghost frame of width 2.  Periodic sides wrap, zero-gradient
 *    sides copy the nearest interior value, Dirichlet sides hold a fixed state
 *    (rho, u, theta) with a1 = 0 and populations at equilibrium.  Ghosts of a
 *    level are refilled from the interior of the same level.  At corners a
 *    Dirichlet or wall y side wins, then a Dirichlet or wall x side, else both
 *    axes are mapped.
 *    Wall sides are no-slip, fixed-temperature walls half-way between the
 *    first ghost layer and the first interior layer: ghost layer g mirrors
 *    interior layer g - 1 with the pressure kept, u reflected about the wall
 *    velocity (u_g = 2 u_w - u) and theta about the wall temperature
 *    (theta_g = 2 theta_w - theta), s from that rho and theta, and ghost
 *    populations rebuilt by the regularised formula of the collision from
 *    the ghost macros and the mirrored cell's a1, without psi.
 *    Parity unpinned for the boundary forms: the paper defers them to an
 *    earlier work that is not available.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The rows of a per-cell pass are independent: each cell writes its own
 * entries and reads only arrays that the pass does not write.  So they may
 * be split over threads (OpenMP, when the library is built with it) without
 * changing any result; one thread (the default) runs them in order. */
#ifdef _OPENMP
#define ROWS_PARALLEL _Pragma("omp parallel for schedule(static) if(o->threads > 1) num_threads(o->threads)")
#else
#define ROWS_PARALLEL
#endif

#define Q 9
#define G 2                      /* ghost width: MUSCL needs s at i +- 2 */
#define CS2 (1.0 / 3.0)          /* c_s^2, Sec. 2.1 */
#define DIM 2

enum { BC_PERIODIC = 0, BC_ZEROGRAD = 1, BC_DIRICHLET = 2, BC_WALL = 3 };

/* D2Q9 velocities and weights, Sec. 2.1 */
static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static double cc(int i, int a) { return (double)(a == 0 ? CX[i] : CY[i]); }
static double kd(int a, int b) { return a == b ? 1.0 : 0.0; }

/* ---- Hermite polynomials, eqs (H0)-(H4) of Sec. 2.2 ---------------------- */
static double herm2(int i, int a, int b) { return cc(i, a) * cc(i, b) - CS2 * kd(a, b); }

static double herm3(int i, int a, int b, int g)
{
    return cc(i, a) * cc(i, b) * cc(i, g)
         - CS2 * (cc(i, a) * kd(b, g) + cc(i, b) * kd(a, g) + cc(i, g) * kd(a, b));
}

static double herm4(int i, int a, int b, int g, int e)
{
    return cc(i, a) * cc(i, b) * cc(i, g) * cc(i, e)
         - CS2 * (cc(i, a) * cc(i, b) * kd(g, e) + cc(i, a) * cc(i, g) * kd(b, e)
                  + cc(i, a) * cc(i, e) * kd(b, g) + cc(i, b) * cc(i, g) * kd(a, e)
                  + cc(i, b) * cc(i, e) * kd(a, g) + cc(i, g) * cc(i, e) * kd(a, b))
         + CS2 * CS2 * (kd(a, b) * kd(g, e) + kd(a, g) * kd(b, e) + kd(a, e) * kd(b, g));
}

/* The D2Q9 basis keeps H_xxy, H_yyx (all index orders) at third order and
 * H_xxyy at fourth order (Sec. 2.3); H_xxx, H_yyy, H_xxxx, ... are dropped. */
static int supported3(int a, int b, int g) { return !(a == b && b == g); }
static int supported4(int a, int b, int g, int e) { return (a + b + g + e) == 2; }

/* Tables of H values; filled once from herm2..herm4. */
static double H2T[Q][2][2], H3T[Q][2][2][2], H4T[Q][2][2][2][2];
static int tables_ready = 0;

static void make_tables(void)
{
    if (tables_ready) return;
    for (int i = 0; i < Q; i++)
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                H2T[i][a][b] = herm2(i, a, b);
                for (int g = 0; g < 2; g++) {
                    H3T[i][a][b][g] = herm3(i, a, b, g);
                    for (int e = 0; e < 2; e++) H4T[i][a][b][g][e] = herm4(i, a, b, g, e);
                }
            }
    tables_ready = 1;
}

/* ---- Hermite expansion with the supported basis, eq (Equilibrium) -------- */
/* f_i = w_i sum_n 1/(n! cs^2n) a^(n) : H^(n), for n = 0..4 (only the orders
 * whose tensors are passed as non-NULL contribute). */
static void hermite_expand(const double *a0, const double a1[2], const double a2[2][2],
                           const double a3[2][2][2], const double a4[2][2][2][2], double out[Q])
{
    make_tables();
    for (int i = 0; i < Q; i++) {
        double sum = 0.0;
        if (a0) sum += *a0;
        if (a1) {
            double t = 0.0;
            for (int a = 0; a < 2; a++) t += a1[a] * cc(i, a);
            sum += t / CS2;
        }
        if (a2) {
            double t = 0.0;
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++) t += a2[a][b] * H2T[i][a][b];
            sum += t / (2.0 * CS2 * CS2);
        }
        if (a3) {
            double t = 0.0;
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++)
                    for (int g = 0; g < 2; g++)
                        if (supported3(a, b, g)) t += a3[a][b][g] * H3T[i][a][b][g];
            sum += t / (6.0 * CS2 * CS2 * CS2);
        }
        if (a4) {
            double t = 0.0;
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++)
                    for (int g = 0; g < 2; g++)
                        for (int e = 0; e < 2; e++)
                            if (supported4(a, b, g, e)) t += a4[a][b][g][e] * H4T[i][a][b][g][e];
            sum += t / (24.0 * CS2 * CS2 * CS2 * CS2);
        }
        out[i] = W[i] * sum;
    }
}

/* Equilibrium, eqs (a0)-(a4) and (Equilibrium), Sec. 2.2. */
void hlbmo_feq_cell(double rho, double ux, double uy, double th, double out[Q])
{
    const double u[2] = {ux, uy};
    const double t1 = th - 1.0;
    double a0 = rho, a1[2], a2[2][2], a3[2][2][2], a4[2][2][2][2];
    for (int a = 0; a < 2; a++) {
        a1[a] = rho * u[a];
        for (int b = 0; b < 2; b++) {
            a2[a][b] = rho * u[a] * u[b] + rho * CS2 * t1 * kd(a, b);
            for (int g = 0; g < 2; g++) {
                a3[a][b][g] = rho * u[a] * u[b] * u[g]
                            + rho * CS2 * t1 * (u[a] * kd(b, g) + u[b] * kd(a, g) + u[g] * kd(a, b));
                for (int e = 0; e < 2; e++)
                    a4[a][b][g][e] = rho * u[a] * u[b] * u[g] * u[e]
                        + rho * CS2 * CS2 * t1 * t1 * (kd(a, b) * kd(g, e) + kd(a, g) * kd(b, e) + kd(a, e) * kd(b, g))
                        + rho * CS2 * t1 * (u[a] * u[b] * kd(g, e) + u[a] * u[g] * kd(b, e) + u[a] * u[e] * kd(b, g)
                                            + u[b] * u[g] * kd(a, e) + u[b] * u[e] * kd(a, g) + u[g] * u[e] * kd(a, b));
            }
        }
    }
    hermite_expand(&a0, a1, a2, a3, a4, out);
}

/* Higher off-equilibrium moments by the recurrence of Sec. 3.3 (taken as
 * printed): out = {a1_xxy, a1_yyx, a1_xxyy}. */
void hlbmo_a1_high(double axx, double axy, double ayy, double ux, double uy, double th, double out[3])
{
    const double axxy = uy * axx + 2.0 * ux * axy;
    const double ayyx = ux * ayy + 2.0 * uy * axy;
    const double axxyy = 2.0 * (ux * ayyx + uy * axxy)
                       + (CS2 * (th - 1.0) - ux * ux) * ayy
                       + (CS2 * (th - 1.0) - uy * uy) * axx
                       - 4.0 * ux * uy * axy;
    out[0] = axxy;
    out[1] = ayyx;
    out[2] = axxyy;
}

/* Regularised off-equilibrium populations f1_i (Sec. 3.3, orders 2..4). */
void hlbmo_f1_cell(double axx, double axy, double ayy, double ux, double uy, double th, double out[Q])
{
    double hi[3];
    hlbmo_a1_high(axx, axy, ayy, ux, uy, th, hi);
    double a2[2][2] = {{axx, axy}, {axy, ayy}};
    double a3[2][2][2], a4[2][2][2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int g = 0; g < 2; g++) {
                const int nx = (a == 0) + (b == 0) + (g == 0);
                a3[a][b][g] = (nx == 2) ? hi[0] : (nx == 1) ? hi[1] : 0.0;
                for (int e = 0; e < 2; e++)
                    a4[a][b][g][e] = supported4(a, b, g, e) ? hi[2] : 0.0;
            }
    hermite_expand(NULL, NULL, a2, a3, a4, out);
}

/* Correction force, eq (Psialgo): psi_i = w_i H_i,ab (E1 + E2)_ab / (2 cs^4). */
void hlbmo_psi_cell(double Exx, double Exy, double Eyy, double out[Q])
{
    double e2[2][2] = {{Exx, Exy}, {Exy, Eyy}};
    hermite_expand(NULL, NULL, e2, NULL, NULL, out);
}

/* Closure defect Gamma_a = rho u_a (1 - theta - u_a^2) = -a^eq_aaa (Sec. 2.3). */
double hlbmo_gamma_closure(double rho, double ua, double th)
{
    return rho * ua * (1.0 - th - ua * ua);
}

double hlbmo_hermite(int i, int order, int a, int b, int g, int e)
{
    switch (order) {
    case 0: return 1.0;
    case 1: return cc(i, a);
    case 2: return herm2(i, a, b);
    case 3: return herm3(i, a, b, g);
    case 4: return herm4(i, a, b, g, e);
    default: return NAN;
    }
}

void hlbmo_lattice(double cx[Q], double cy[Q], double w[Q])
{
    for (int i = 0; i < Q; i++) { cx[i] = CX[i]; cy[i] = CY[i]; w[i] = W[i]; }
}

/* ---- Van Albada limited MUSCL term for u ds/dx (Sec. 3.4) ----------------- */
/* Limited slope of s at a cell from its two neighbours; zero at extrema. */
static double van_albada_slope(double sm, double s0, double sp)
{
    const double a = s0 - sm, b = sp - s0;
    if (a * b <= 0.0) return 0.0;
    return a * b * (a + b) / (a * a + b * b);
}

/* u ds/dx from the upwind reconstructed face values (cell velocity decides
 * the upwind side; zero velocity gives zero advection). */
static double muscl_term(double u, double smm, double sm, double s0, double sp, double spp)
{
    if (u > 0.0) {
        const double face_r = s0 + 0.5 * van_albada_slope(sm, s0, sp);
        const double face_l = sm + 0.5 * van_albada_slope(smm, sm, s0);
        return u * (face_r - face_l);
    }
    if (u < 0.0) {
        const double face_r = sp - 0.5 * van_albada_slope(s0, sp, spp);
        const double face_l = s0 - 0.5 * van_albada_slope(sm, s0, sp);
        return u * (face_r - face_l);
    }
    return 0.0;
}

double hlbmo_muscl_term(double u, double smm, double sm, double s0, double sp, double spp)
{
    return muscl_term(u, smm, sm, s0, sp, spp);
}

/* ---- the solver state ------------------------------------------------------ */
typedef struct {
    int nx, ny, px, py;
    double gamma, Pr, mu, sigma;
    int bc[4];              /* x-, x+, y-, y+ */
    double bcs[4][4];       /* Dirichlet (rho, ux, uy, theta) or wall (-, ux, uy, theta) per side */
    int phi_mode;           /* 0: Phi from a1 (eq viscous heat discret), 1: finite differences */
    int ablation;           /* bit 1: centred E1, bit 2: no E2 (parts of the original model) */
    double cv, cp, lambda;
    /* Dirichlet ghost values per side */
    double b_s[4], b_feq[4][Q], b_gx[4], b_gy[4];
    /* level-n fields (Algorithm 1 state) */
    double *rho, *ux, *uy, *th, *s, *axx, *axy, *ayy;
    double *feq[Q], *psi[Q];
    /* step work arrays */
    double *F[Q], *fb[Q];
    double *rho1, *ux1, *uy1, *th1, *s1, *axx1, *axy1, *ayy1;
    double *feq1[Q], *psi1[Q];
    double *gx, *gy;          /* Gamma_x, Gamma_y of the level being differentiated */
    long step;
    int threads;              /* threads for the per-cell passes (1: in order) */
} hlbmo;

static inline int IX(const hlbmo *o, int x, int y) { return (y + G) * o->px + (x + G); }

static int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

/* The ghost frame of one array is refilled in two passes: the x sides over
 * the interior rows, then the y sides over the full padded width, so that a
 * y side wins at a corner.  dv holds the Dirichlet value per side; wall
 * sides are skipped here and filled between and after the passes (see
 * fill_level, fill_a1_ghosts and collide). */
static void fill_x(const hlbmo *o, double *a, const double dv[4])
{
    for (int y = 0; y < o->ny; y++)
        for (int g = 1; g <= G; g++) {
            const int xl = -g, xr = o->nx - 1 + g;
            switch (o->bc[0]) {
            case BC_PERIODIC: a[IX(o, xl, y)] = a[IX(o, wrap(xl, o->nx), y)]; break;
            case BC_ZEROGRAD: a[IX(o, xl, y)] = a[IX(o, 0, y)]; break;
            case BC_WALL: break;
            default: a[IX(o, xl, y)] = dv[0];
            }
            switch (o->bc[1]) {
            case BC_PERIODIC: a[IX(o, xr, y)] = a[IX(o, wrap(xr, o->nx), y)]; break;
            case BC_ZEROGRAD: a[IX(o, xr, y)] = a[IX(o, o->nx - 1, y)]; break;
            case BC_WALL: break;
            default: a[IX(o, xr, y)] = dv[1];
            }
        }
}

static void fill_y(const hlbmo *o, double *a, const double dv[4])
{
    for (int x = -G; x < o->nx + G; x++)
        for (int g = 1; g <= G; g++) {
            const int yl = -g, yr = o->ny - 1 + g;
            switch (o->bc[2]) {
            case BC_PERIODIC: a[IX(o, x, yl)] = a[IX(o, x, wrap(yl, o->ny))]; break;
            case BC_ZEROGRAD: a[IX(o, x, yl)] = a[IX(o, x, 0)]; break;
            case BC_WALL: break;
            default: a[IX(o, x, yl)] = dv[2];
            }
            switch (o->bc[3]) {
            case BC_PERIODIC: a[IX(o, x, yr)] = a[IX(o, x, wrap(yr, o->ny))]; break;
            case BC_ZEROGRAD: a[IX(o, x, yr)] = a[IX(o, x, o->ny - 1)]; break;
            case BC_WALL: break;
            default: a[IX(o, x, yr)] = dv[3];
            }
        }
}

static void side_values(const hlbmo *o, int q, double dv[4])
{
    for (int k = 0; k < 4; k++) dv[k] = o->bcs[k][q];
}

/* Wall side k (0: x-, 1: x+, 2: y-, 3: y+), ghost layer g (1 or 2) and
 * position t along the wall (a row for an x side, over the interior rows; a
 * column for a y side, over the full padded width): the ghost cell and the
 * interior cell it mirrors about the wall, which lies half-way between the
 * first ghost layer and the first interior layer. */
static int wall_span(const hlbmo *o, int k, int *t0) { *t0 = k < 2 ? 0 : -G; return k < 2 ? o->ny : o->nx + 2 * G; }
static void wall_cells(const hlbmo *o, int k, int g, int t, int *kg, int *km)
{
    if (k < 2) {
        *kg = IX(o, k == 0 ? -g : o->nx - 1 + g, t);
        *km = IX(o, k == 0 ? g - 1 : o->nx - g, t);
    } else {
        *kg = IX(o, t, k == 2 ? -g : o->ny - 1 + g);
        *km = IX(o, t, k == 2 ? g - 1 : o->ny - g);
    }
}

static double entropy_of(const hlbmo *o, double rho, double th);

/* Ghost macros of the wall sides k0, k0 + 1: u reflected about the wall
 * velocity, theta about the wall temperature, the mirrored cell's pressure
 * (rho_g theta_g = rho theta), s of the ghost rho and theta. */
static void wall_macros(hlbmo *o, int k0, double *rho, double *ux, double *uy, double *th, double *s)
{
    for (int k = k0; k < k0 + 2; k++) {
        if (o->bc[k] != BC_WALL) continue;
        const double uw = o->bcs[k][1], vw = o->bcs[k][2], tw = o->bcs[k][3];
        int t0;
        const int n = wall_span(o, k, &t0);
        for (int g = 1; g <= G; g++)
            for (int t = t0; t < t0 + n; t++) {
                int kg, km;
                wall_cells(o, k, g, t, &kg, &km);
                ux[kg] = 2.0 * uw - ux[km];
                uy[kg] = 2.0 * vw - uy[km];
                th[kg] = 2.0 * tw - th[km];
                rho[kg] = rho[km] * th[km] / th[kg];
                s[kg] = entropy_of(o, rho[kg], th[kg]);
            }
    }
}

/* The ghost frame of a level's rho, u, theta and s: x sides (x walls
 * mirror the interior columns), then y sides over the full width (y walls
 * mirror rows whose x ghosts are already filled). */
static void fill_level(hlbmo *o, double *rho, double *ux, double *uy, double *th, double *s)
{
    double *f[4] = {rho, ux, uy, th};
    double dv[4];
    for (int q = 0; q < 4; q++) { side_values(o, q, dv); fill_x(o, f[q], dv); }
    fill_x(o, s, o->b_s);
    wall_macros(o, 0, rho, ux, uy, th, s);
    for (int q = 0; q < 4; q++) { side_values(o, q, dv); fill_y(o, f[q], dv); }
    fill_y(o, s, o->b_s);
    wall_macros(o, 2, rho, ux, uy, th, s);
}

static double *alloc_field(const hlbmo *o)
{
    return (double *)calloc((size_t)o->px * o->py, sizeof(double));
}

/* s = c_v ln(theta / rho^(gamma-1)), eq (Entropie expression). */
static double entropy_of(const hlbmo *o, double rho, double th)
{
    return o->cv * log(th / pow(rho, o->gamma - 1.0));
}

/* theta = rho^(gamma-1) exp(s / c_v), the same relation solved for theta. */
static double theta_of(const hlbmo *o, double rho, double s)
{
    return pow(rho, o->gamma - 1.0) * exp(s / o->cv);
}

void hlbmo_destroy(hlbmo *o);

hlbmo *hlbmo_create(int nx, int ny, double gamma, double Pr, double mu, double sigma,
                    const int bc[4], const double bc_state[16], int phi_mode, int ablation)
{
    if (nx < 1 || ny < 1) return NULL;
    hlbmo *o = (hlbmo *)calloc(1, sizeof(hlbmo));
    if (!o) return NULL;
    make_tables();
    o->threads = 1;
    o->nx = nx; o->ny = ny; o->px = nx + 2 * G; o->py = ny + 2 * G;
    o->gamma = gamma; o->Pr = Pr; o->mu = mu; o->sigma = sigma; o->phi_mode = phi_mode;
    o->ablation = ablation;
    for (int k = 0; k < 4; k++) {
        o->bc[k] = bc[k];
        for (int q = 0; q < 4; q++) o->bcs[k][q] = bc_state ? bc_state[4 * k + q] : 0.0;
        if (bc[k] < BC_PERIODIC || bc[k] > BC_WALL) { free(o); return NULL; }
        /* walls need a positive temperature and two interior layers to mirror */
        if (bc[k] == BC_WALL && ((k < 2 ? nx : ny) < 2 || !(o->bcs[k][3] > 0.0))) { free(o); return NULL; }
    }
    /* c_v = c_s^2/(gamma-1), c_p = gamma c_s^2/(gamma-1) (Sec. 2.4).
     * Heat conductivity lambda = mu c_p / Pr, the definition of the Prandtl
     * number.  Sec. 2.1 prints mu / (c_p Pr); the paper's own acoustic decay
     * rate (Sec. 4.3) and thermal Couette profile (Sec. 4.4) hold only with
     * mu c_p / Pr, so that is the reading taken here. */
    o->cv = CS2 / (gamma - 1.0);
    o->cp = gamma * CS2 / (gamma - 1.0);
    o->lambda = mu * o->cp / Pr;
    for (int k = 0; k < 4; k++) {
        if (o->bc[k] != BC_DIRICHLET) continue;
        const double r = o->bcs[k][0], u = o->bcs[k][1], v = o->bcs[k][2], t = o->bcs[k][3];
        o->b_s[k] = entropy_of(o, r, t);
        hlbmo_feq_cell(r, u, v, t, o->b_feq[k]);
        o->b_gx[k] = hlbmo_gamma_closure(r, u, t);
        o->b_gy[k] = hlbmo_gamma_closure(r, v, t);
    }
    double **fields[] = {&o->rho, &o->ux, &o->uy, &o->th, &o->s, &o->axx, &o->axy, &o->ayy,
                         &o->rho1, &o->ux1, &o->uy1, &o->th1, &o->s1, &o->axx1, &o->axy1, &o->ayy1,
                         &o->gx, &o->gy};
    for (size_t k = 0; k < sizeof(fields) / sizeof(fields[0]); k++) {
        *fields[k] = alloc_field(o);
        if (!*fields[k]) { hlbmo_destroy(o); return NULL; }
    }
    for (int i = 0; i < Q; i++) {
        o->feq[i] = alloc_field(o); o->psi[i] = alloc_field(o);
        o->F[i] = alloc_field(o); o->fb[i] = alloc_field(o);
        o->feq1[i] = alloc_field(o); o->psi1[i] = alloc_field(o);
        if (!o->feq[i] || !o->psi[i] || !o->F[i] || !o->fb[i] || !o->feq1[i] || !o->psi1[i]) {
            hlbmo_destroy(o);
            return NULL;
        }
    }
    return o;
}

void hlbmo_destroy(hlbmo *o)
{
    if (!o) return;
    double *fs[] = {o->rho, o->ux, o->uy, o->th, o->s, o->axx, o->axy, o->ayy,
                    o->rho1, o->ux1, o->uy1, o->th1, o->s1, o->axx1, o->axy1, o->ayy1, o->gx, o->gy};
    for (size_t k = 0; k < sizeof(fs) / sizeof(fs[0]); k++) free(fs[k]);
    for (int i = 0; i < Q; i++) {
        free(o->feq[i]); free(o->psi[i]); free(o->F[i]); free(o->fb[i]);
        free(o->feq1[i]); free(o->psi1[i]);
    }
    free(o);
}

/* Velocity gradient G[a][b] = d u_a / d x_b by second-order centred
 * differences of a ghost-filled level. */
static void velocity_gradient(const hlbmo *o, const double *ux, const double *uy, int x, int y,
                              double Gm[2][2])
{
    Gm[0][0] = 0.5 * (ux[IX(o, x + 1, y)] - ux[IX(o, x - 1, y)]);
    Gm[0][1] = 0.5 * (ux[IX(o, x, y + 1)] - ux[IX(o, x, y - 1)]);
    Gm[1][0] = 0.5 * (uy[IX(o, x + 1, y)] - uy[IX(o, x - 1, y)]);
    Gm[1][1] = 0.5 * (uy[IX(o, x, y + 1)] - uy[IX(o, x, y - 1)]);
}

/* sgn with sgn(0) = 0 */
static double sgn(double v) { return v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0); }

/* Correction force psi of one level (eq Psialgo, Sec. 3.2): Gamma from
 * the ghost-filled macros, E1 by the upwind difference of Sec. 3.2, E2 by
 * centred differences (eq E2 corr term), psi by eq (Psialgo).  The ablation
 * bits restore parts of the original model the paper improves on: bit 1
 * takes E1 by centred differences, bit 2 drops E2. */
static void compute_psi(hlbmo *o, const double *rho, const double *ux, const double *uy,
                        const double *th, double *psi[Q])
{
    ROWS_PARALLEL
    for (int y = -G; y < o->ny + G; y++)
        for (int x = -G; x < o->nx + G; x++) {
            const int k = IX(o, x, y);
            o->gx[k] = hlbmo_gamma_closure(rho[k], ux[k], th[k]);
            o->gy[k] = hlbmo_gamma_closure(rho[k], uy[k], th[k]);
        }
    ROWS_PARALLEL
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) {
            const int k = IX(o, x, y);
            const double sx = (o->ablation & 1) ? 0.0 : sgn(ux[k]);
            const double sy = (o->ablation & 1) ? 0.0 : sgn(uy[k]);
            const double e1xx = 0.5 * (1.0 + sx) * (o->gx[k] - o->gx[IX(o, x - 1, y)])
                              + 0.5 * (1.0 - sx) * (o->gx[IX(o, x + 1, y)] - o->gx[k]);
            const double e1yy = 0.5 * (1.0 + sy) * (o->gy[k] - o->gy[IX(o, x, y - 1)])
                              + 0.5 * (1.0 - sy) * (o->gy[IX(o, x, y + 1)] - o->gy[k]);
            double Gm[2][2];
            velocity_gradient(o, ux, uy, x, y, Gm);
            const double p = rho[k] * CS2 * th[k];                 /* eq (perfect gas) */
            const double divu = Gm[0][0] + Gm[1][1];
            const double e2 = (o->ablation & 2) ? 0.0 : p * ((DIM + 2.0) / DIM - o->gamma) * divu;
            double out[Q];
            hlbmo_psi_cell(e1xx + e2, 0.0, e1yy + e2, out);
            for (int i = 0; i < Q; i++) psi[i][k] = out[i];
        }
}

/* a1^FD of eq (a1FD) at one cell.  (tau_bar / tau) mu = tau_bar p because
 * mu = tau p (Sec. 2.4), which stays finite when mu = 0. */
static void a1_fd(const hlbmo *o, double rho, double th, const double Gm[2][2], double a[2][2])
{
    const double p = rho * CS2 * th;
    const double tau = o->mu / p;
    const double taub = tau + 0.5;
    const double divu = Gm[0][0] + Gm[1][1];
    for (int al = 0; al < 2; al++)
        for (int be = 0; be < 2; be++)
            a[al][be] = -taub * p * (Gm[al][be] + Gm[be][al] - (2.0 / DIM) * divu * kd(al, be));
}

int hlbmo_init(hlbmo *o, const double *rho0, const double *ux0, const double *uy0, const double *th0,
               const double *a1opt)
{
    const int n = o->nx * o->ny;
    /* the input state [rho, u, theta]^(0) and s from eq (Entropie expression) */
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) {
            const int c = y * o->nx + x, k = IX(o, x, y);
            o->rho[k] = rho0[c]; o->ux[k] = ux0[c]; o->uy[k] = uy0[c]; o->th[k] = th0[c];
            o->s[k] = entropy_of(o, rho0[c], th0[c]);
        }
    fill_level(o, o->rho, o->ux, o->uy, o->th, o->s);
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) {
            const int c = y * o->nx + x, k = IX(o, x, y);
            double out[Q];
            /* f^eq(0), eq (Equilibrium) */
            hlbmo_feq_cell(o->rho[k], o->ux[k], o->uy[k], o->th[k], out);
            for (int i = 0; i < Q; i++) o->feq[i][k] = out[i];
            /* a1(0) = a1^FD of eq (a1FD), or the given one */
            if (a1opt) {
                o->axx[k] = a1opt[c]; o->axy[k] = a1opt[n + c]; o->ayy[k] = a1opt[2 * n + c];
            } else {
                double Gm[2][2], a[2][2];
                velocity_gradient(o, o->ux, o->uy, x, y, Gm);
                a1_fd(o, o->rho[k], o->th[k], Gm, a);
                o->axx[k] = a[0][0]; o->axy[k] = a[0][1]; o->ayy[k] = a[1][1];
            }
        }
    /* psi(0), eq (Psialgo) */
    compute_psi(o, o->rho, o->ux, o->uy, o->th, o->psi);
    o->step = 0;
    return 0;
}

/* a1 on the ghost frame, for the wall populations: copies on periodic and
 * zero-gradient sides, 0 on Dirichlet sides, the mirrored cell's a1 on wall
 * sides (x sides first, then y sides over the full width). */
static void fill_a1_ghosts(hlbmo *o)
{
    const double zero[4] = {0.0, 0.0, 0.0, 0.0};
    double *a[3] = {o->axx, o->axy, o->ayy};
    for (int pass = 0; pass < 2; pass++) {
        for (int q = 0; q < 3; q++) (pass == 0 ? fill_x : fill_y)(o, a[q], zero);
        for (int k = 2 * pass; k < 2 * pass + 2; k++) {
            if (o->bc[k] != BC_WALL) continue;
            int t0;
            const int n = wall_span(o, k, &t0);
            for (int g = 1; g <= G; g++)
                for (int t = t0; t < t0 + n; t++) {
                    int kg, km;
                    wall_cells(o, k, g, t, &kg, &km);
                    for (int q = 0; q < 3; q++) a[q][kg] = a[q][km];
                }
        }
    }
}

/* Post-collision populations of the wall ghost layers of sides k0, k0 + 1:
 * the regularised formula of eq streamalgo from the ghost macros of level n
 * and the mirrored cell's a1, without psi. */
static void wall_populations(hlbmo *o, int k0)
{
    for (int k = k0; k < k0 + 2; k++) {
        if (o->bc[k] != BC_WALL) continue;
        int t0;
        const int n = wall_span(o, k, &t0);
        for (int g = 1; g <= G; g++)
            for (int t = t0; t < t0 + n; t++) {
                int kg, km;
                wall_cells(o, k, g, t, &kg, &km);
                const double p = o->rho[kg] * CS2 * o->th[kg];
                const double taub = o->mu / p + 0.5;
                double feq[Q], f1[Q];
                hlbmo_feq_cell(o->rho[kg], o->ux[kg], o->uy[kg], o->th[kg], feq);
                hlbmo_f1_cell(o->axx[kg], o->axy[kg], o->ayy[kg], o->ux[kg], o->uy[kg], o->th[kg], f1);
                for (int i = 0; i < Q; i++) o->F[i][kg] = feq[i] + (1.0 - 1.0 / taub) * f1[i];
            }
    }
}

static int has_wall(const hlbmo *o)
{
    for (int k = 0; k < 4; k++)
        if (o->bc[k] == BC_WALL) return 1;
    return 0;
}

/* The regularised collision for every interior cell: F_i = f^eq_i + (1 - 1/tau_bar)
 * f1_i + psi_i / 2 (eq streamalgo), the post-collision populations of level n. */
static void collide(hlbmo *o)
{
    ROWS_PARALLEL
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) {
            const int k = IX(o, x, y);
            const double p = o->rho[k] * CS2 * o->th[k];
            const double taub = o->mu / p + 0.5;
            double f1[Q];
            hlbmo_f1_cell(o->axx[k], o->axy[k], o->ayy[k], o->ux[k], o->uy[k], o->th[k], f1);
            for (int i = 0; i < Q; i++)
                o->F[i][k] = o->feq[i][k] + (1.0 - 1.0 / taub) * f1[i] + 0.5 * o->psi[i][k];
        }
    const int walls = has_wall(o);
    if (walls) fill_a1_ghosts(o);
    for (int pass = 0; pass < 2; pass++) {
        for (int i = 0; i < Q; i++) {
            double dv[4];
            for (int s = 0; s < 4; s++) dv[s] = o->b_feq[s][i];
            (pass == 0 ? fill_x : fill_y)(o, o->F[i], dv);
        }
        if (walls) wall_populations(o, 2 * pass);
    }
}

/* Entropy right-hand side of eq (sequaalgo), every term at level n:
 * -u . grad s (MUSCL, Van Albada) + div(lambda grad theta) / (rho theta)
 * + Phi / (rho theta). */
static double entropy_rhs(const hlbmo *o, int x, int y)
{
    const int k = IX(o, x, y);
    const double *s = o->s;
    const double adv = muscl_term(o->ux[k], s[IX(o, x - 2, y)], s[IX(o, x - 1, y)], s[k],
                                  s[IX(o, x + 1, y)], s[IX(o, x + 2, y)])
                     + muscl_term(o->uy[k], s[IX(o, x, y - 2)], s[IX(o, x, y - 1)], s[k],
                                  s[IX(o, x, y + 1)], s[IX(o, x, y + 2)]);
    const double *t = o->th;
    const double lap = (t[IX(o, x + 1, y)] - 2.0 * t[k] + t[IX(o, x - 1, y)])
                     + (t[IX(o, x, y + 1)] - 2.0 * t[k] + t[IX(o, x, y - 1)]);
    const double rho = o->rho[k], th = o->th[k];
    double Gm[2][2];
    velocity_gradient(o, o->ux, o->uy, x, y, Gm);
    double phi = 0.0;
    if (o->phi_mode == 0) {
        /* eq (viscous heat discret): Phi = -(tau / tau_bar) a1_ab d_b u_a */
        const double p = rho * CS2 * th;
        const double tau = o->mu / p, taub = tau + 0.5;
        const double a[2][2] = {{o->axx[k], o->axy[k]}, {o->axy[k], o->ayy[k]}};
        for (int al = 0; al < 2; al++)
            for (int be = 0; be < 2; be++) phi += a[al][be] * Gm[al][be];
        phi *= -(tau / taub);
    } else {
        /* eq (viscous heat): Phi = mu (d_b u_a + d_a u_b - (2/D) div u delta_ab) d_b u_a */
        const double divu = Gm[0][0] + Gm[1][1];
        for (int al = 0; al < 2; al++)
            for (int be = 0; be < 2; be++)
                phi += (Gm[al][be] + Gm[be][al] - (2.0 / DIM) * divu * kd(al, be)) * Gm[al][be];
        phi *= o->mu;
    }
    return -adv + o->lambda * lap / (rho * th) + phi / (rho * th);
}

void hlbmo_entropy_rhs(const hlbmo *o, double *out)
{
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) out[y * o->nx + x] = entropy_rhs(o, x, y);
}

static void swap_ptr(double **a, double **b) { double *t = *a; *a = *b; *b = t; }

int hlbmo_step(hlbmo *o, long nsteps)
{
    for (long it = 0; it < nsteps; it++) {
        /* collide with [f^eq, a1, psi]^(n), eq (streamalgo) ... */
        collide(o);
        /* ... and stream: fbar_i(x) = F_i(x - c_i) */
        ROWS_PARALLEL
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                const int k = IX(o, x, y);
                for (int i = 0; i < Q; i++) o->fb[i][k] = o->F[i][IX(o, x - CX[i], y - CY[i])];
            }
        /* rho, u at n+1, eqs (rhoalgo), (ualgo) */
        ROWS_PARALLEL
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                const int k = IX(o, x, y);
                double r = 0.0, mx = 0.0, my = 0.0;
                for (int i = 0; i < Q; i++) {
                    r += o->fb[i][k];
                    mx += CX[i] * o->fb[i][k];
                    my += CY[i] * o->fb[i][k];
                }
                o->rho1[k] = r; o->ux1[k] = mx / r; o->uy1[k] = my / r;
            }
        /* s at n+1 from level-n rho, u, theta, a1, eq (sequaalgo) (explicit Euler, dt = 1) */
        ROWS_PARALLEL
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                const int k = IX(o, x, y);
                o->s1[k] = o->s[k] + entropy_rhs(o, x, y);
            }
        /* theta at n+1, eq (Entropie expression) */
        ROWS_PARALLEL
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                const int k = IX(o, x, y);
                o->th1[k] = theta_of(o, o->rho1[k], o->s1[k]);
            }
        fill_level(o, o->rho1, o->ux1, o->uy1, o->th1, o->s1);
        /* psi at n+1, eq (Psialgo) */
        compute_psi(o, o->rho1, o->ux1, o->uy1, o->th1, o->psi1);
        /* f^eq at n+1, eq (Equilibrium) */
        ROWS_PARALLEL
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                const int k = IX(o, x, y);
                double out[Q];
                hlbmo_feq_cell(o->rho1[k], o->ux1[k], o->uy1[k], o->th1[k], out);
                for (int i = 0; i < Q; i++) o->feq1[i][k] = out[i];
            }
        /* a1 at n+1 = sigma a1^PR + (1 - sigma) a1^FD, eq (a1sigalgo) */
        ROWS_PARALLEL
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                const int k = IX(o, x, y);
                double pr[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
                for (int i = 0; i < Q; i++) {
                    const double neq = o->fb[i][k] - o->feq1[i][k] + 0.5 * o->psi1[i][k];
                    for (int al = 0; al < 2; al++)
                        for (int be = 0; be < 2; be++) pr[al][be] += H2T[i][al][be] * neq;
                }
                double Gm[2][2], fd[2][2];
                velocity_gradient(o, o->ux1, o->uy1, x, y, Gm);
                a1_fd(o, o->rho1[k], o->th1[k], Gm, fd);
                o->axx1[k] = o->sigma * pr[0][0] + (1.0 - o->sigma) * fd[0][0];
                o->axy1[k] = o->sigma * pr[0][1] + (1.0 - o->sigma) * fd[0][1];
                o->ayy1[k] = o->sigma * pr[1][1] + (1.0 - o->sigma) * fd[1][1];
            }
        /* level n+1 becomes level n */
        swap_ptr(&o->rho, &o->rho1); swap_ptr(&o->ux, &o->ux1); swap_ptr(&o->uy, &o->uy1);
        swap_ptr(&o->th, &o->th1); swap_ptr(&o->s, &o->s1);
        swap_ptr(&o->axx, &o->axx1); swap_ptr(&o->axy, &o->axy1); swap_ptr(&o->ayy, &o->ayy1);
        for (int i = 0; i < Q; i++) { swap_ptr(&o->feq[i], &o->feq1[i]); swap_ptr(&o->psi[i], &o->psi1[i]); }
        o->step++;
    }
    return 0;
}

/* ---- accessors (row-major [y][x] without ghosts) -------------------------- */
static void copy_out(const hlbmo *o, const double *a, double *out)
{
    if (!out) return;
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) out[y * o->nx + x] = a[IX(o, x, y)];
}

/* rho, ux, uy, theta, s, a1 (3 planes xx, xy, yy) of the current level. */
void hlbmo_get(const hlbmo *o, double *rho, double *ux, double *uy, double *th, double *s, double *a1)
{
    const int n = o->nx * o->ny;
    copy_out(o, o->rho, rho); copy_out(o, o->ux, ux); copy_out(o, o->uy, uy);
    copy_out(o, o->th, th); copy_out(o, o->s, s);
    if (a1) { copy_out(o, o->axx, a1); copy_out(o, o->axy, a1 + n); copy_out(o, o->ayy, a1 + 2 * n); }
}

void hlbmo_get_psi(const hlbmo *o, double *out9)
{
    const int n = o->nx * o->ny;
    for (int i = 0; i < Q; i++) copy_out(o, o->psi[i], out9 + (size_t)i * n);
}

void hlbmo_get_feq(const hlbmo *o, double *out9)
{
    const int n = o->nx * o->ny;
    for (int i = 0; i < Q; i++) copy_out(o, o->feq[i], out9 + (size_t)i * n);
}

/* Post-collision populations of the current level (eq streamalgo without streaming). */
void hlbmo_get_post_collision(hlbmo *o, double *out9)
{
    const int n = o->nx * o->ny;
    collide(o);
    for (int i = 0; i < Q; i++) copy_out(o, o->F[i], out9 + (size_t)i * n);
}

long hlbmo_step_count(const hlbmo *o) { return o->step; }

/* Threads for the per-cell passes of hlbmo_step (results do not depend on
 * it); without OpenMP every pass runs on the calling thread. */
void hlbmo_set_threads(hlbmo *o, int n) { o->threads = n > 1 ? n : 1; }

/* Processors OpenMP can use, or 1 when the library is built without it. */
int hlbmo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}
