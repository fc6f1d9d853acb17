/*
 * Plain, slow FP64 CPU oracle of the forcing-based free-energy D2Q9 lattice
 * Boltzmann step (Li, Yu & Huang, "Achieving thermodynamic consistency in a
 * class of free-energy multiphase lattice Boltzmann models").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do. It shares no source with the CUDA library.
 *
 * The step is written as the paper states it, one literal stage at a time,
 * over the whole periodic lattice, with no fusion:
 *   1. rho = sum_a f_a                                   (Eq. 12)
 *   2. lap = isotropic 9-point Laplacian of rho          (Eq. 2 needs it; the
 *      paper prints no stencil: reading 6 * sum_a w_a (rho(x+e_a) - rho(x)))
 *   3. mu_c = E_f'(rho) - kappa * lap                    (Eq. 2, Eq. 30 / CS)
 *   4. grad_h of mu_c (and of rho for the standard form)  (Eq. 17)
 *   5. F = grad_h(rho/3) - rho grad_h mu_c  (standard,  Eq. 13 right)
 *      F = (1/3 - rho) grad_h mu_c         (improved,  Eq. 24)
 *   6. u = (sum_a e_a f_a + F/2) / rho                   (Eq. 12)
 *   7. improved only: p_m = (c0 + mu_c)/3, phi = rho/3 - p_m,
 *      C1 = d_x(phi u_x) + d_y(phi u_y), C7 = d_x(phi u_x) - d_y(phi u_y),
 *      derivatives by the Eq. 17 stencil                  (Eqs. 24, 29);
 *      scheme 3 first replaces phi u_x, phi u_y by their lattice-weight
 *      averages sum_a w_a (phi u)(x + e_a) (a reading: the paper does not
 *      state how these derivatives are discretised)
 *   8. G_a from Eq. 14 for all nine a; S = M G; m = M f; m_eq from Eq. 11
 *      (standard) or Eq. 27 (improved), all as dense 9x9 products
 *   9. m* = m - Lambda (m - m_eq) + (I - Lambda/2)(S + C)  (Eqs. 9, 28, 8)
 *  10. f* = M^-1 m*, with M^-1 obtained by Gauss-Jordan elimination
 *  11. push streaming f_a(x + e_a) = f*_a(x), periodic     (Eq. 10); with
 *      walls, halfway bounce-back with the moving-wall term (Sec. IV C)
 *
 * Scheme 4 is the Lax-Wendroff propagation scheme the paper compares with
 * (Appendix A): stages 1-6 with the standard force (Eq. 13 right) and
 * u = (sum_a e_a f_a + dt F / 2) / rho, dt = A the CFL number; then the
 * BGK collision of Eq. A1 with the equilibrium of Eq. A3, whose tensor T
 * comes from the second moment of the populations by Eq. A4, and the
 * three-point propagation of Eq. A2 with a_0 = 1 - A^2,
 * a_1 = A (A - 1) / 2, a_-1 = A (A + 1) / 2.
 *
 * M is the Lallemand-Luo D2Q9 moment matrix with moments ordered
 * (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy): the order of the relaxation
 * vector of Eq. 8 and of the equilibria of Eqs. 11 and 27 (the paper cites
 * the matrix but does not print it).
 *
 * Layout: populations f[a][y][x] (a = 0..8, x fastest); fields [y][x].
 * Velocity order e0=(0,0), e1=(1,0), e2=(0,1), e3=(-1,0), e4=(0,-1),
 * e5=(1,1), e6=(-1,1), e7=(-1,-1), e8=(1,-1); weights from Eq. 14.
 *
 * Compile with -O2 -ffp-contract=off so that no fused multiply-add changes
 * the rounding of the literal expressions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 9

static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WA[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2, Eq. 13 */
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6}; /* e_OPP[a] = -e_a */

/* Lallemand-Luo transformation matrix, rows = moments. */
static const double MM[Q][Q] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},          /* rho  */
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},     /* e    */
    {4, -2, -2, -2, -2, 1, 1, 1, 1},      /* eps  */
    {0, 1, 0, -1, 0, 1, -1, -1, 1},       /* j_x  */
    {0, -2, 0, 2, 0, 1, -1, -1, 1},       /* q_x  */
    {0, 0, 1, 0, -1, 1, 1, -1, -1},       /* j_y  */
    {0, 0, -2, 0, 2, 1, 1, -1, -1},       /* q_y  */
    {0, 1, -1, 1, -1, 0, 0, 0, 0},        /* p_xx */
    {0, 0, 0, 0, 0, 1, -1, 1, -1},        /* p_xy */
};

typedef struct {
    int32_t nx, ny;
    int32_t scheme;    /* 0 = standard (Eq. 13 right), 1 = improved (Eqs. 24, 27, 28),
                          2 = standard with the pressure-tensor force (Eq. 13 left),
                          3 = improved with the derivatives of Eq. 29 taken on the
                              lattice-weight average of phi u,
                          4 = Lax-Wendroff propagation (Appendix A, Eqs. A1-A4) */
    int32_t collision; /* 0 = BGK (all rates 1/tau_v), 1 = MRT (Eq. 8) */
    int32_t eos;       /* 0 = van der Waals (Eq. 30), 1 = Carnahan-Starling */
    int32_t flags;     /* planted-mistake hooks for pin tests; 0 in normal use.
                          bit 0: drop the correction term C of Eq. 28
                          bit 1: flip the sign of the F/2 shift in Eq. 12
                          bit 2: the adjoint ignores C (forward unchanged)
                          bit 3: wall ghost rows copy j_y of the mirrored row
                                 unchanged instead of reflecting it
                          bit 4: constant-nu map with p_m / rho in place of
                                 rho / p_m (improved scheme)
                          bit 5: the improved scheme takes the standard
                                 scheme's constant-nu map */
    double a, b, R, T, kappa;
    double tau_v, tau_e, tau_s, tau_q; /* MRT rates of Eq. 8; tau_c = 1 */
    double pm_c0;                      /* p_m = (c0 + mu_c)/3; the paper's c0 is 1 */
    double nu;                         /* > 0: constant kinematic viscosity, tau_v set per
                                          node from it (Sec. III below Eq. 29; Sec. II A) */
    int32_t walls;                     /* 0: periodic in y; 1: no-slip walls half a node
                                          below y = 0 and above y = ny - 1 (Sec. IV C) */
    int32_t pad_;
    double wall_u;                     /* x velocity of both walls */
    double rho_wall;                   /* wall density of the moving-wall bounce-back term */
    double lw_A, lw_B;                 /* scheme 4: CFL number A (the time step) and B of Eq. A3 */
} orc_case;

/* ------------------------------------------------------------------ EOS */

/* Bulk free-energy density E_f(rho). vdW: Eq. 30's E_f. CS: the
 * Carnahan-Starling free energy E_f = RT rho ln rho + RT rho (4n - 3n^2)/(1-n)^2
 * - a rho^2 with n = b rho / 4 (not in the paper). */
double orc_Ef(const orc_case* c, double rho)
{
    if (c->eos == 0) return rho * c->R * c->T * log(rho / (1.0 - c->b * rho)) - c->a * rho * rho;
    double n = c->b * rho / 4.0;
    double om = 1.0 - n;
    return c->R * c->T * rho * log(rho) + c->R * c->T * rho * (4.0 * n - 3.0 * n * n) / (om * om) -
           c->a * rho * rho;
}

/* E_f'(rho), the bulk part of the chemical potential (Eq. 2; vdW Eq. 30). */
double orc_dEf(const orc_case* c, double rho)
{
    if (c->eos == 0) {
        double one_m = 1.0 - c->b * rho;
        return c->R * c->T * (log(rho / one_m) + 1.0 / one_m) - 2.0 * c->a * rho;
    }
    double n = c->b * rho / 4.0;
    double om = 1.0 - n;
    return c->R * c->T *
               (log(rho) + 1.0 + (4.0 * n - 3.0 * n * n) / (om * om) +
                n * (4.0 - 2.0 * n) / (om * om * om)) -
           2.0 * c->a * rho;
}

/* p_EOS = rho E_f' - E_f (the line after Eq. 4). */
double orc_pEOS(const orc_case* c, double rho) { return rho * orc_dEf(c, rho) - orc_Ef(c, rho); }

/* ------------------------------------------------------------- stencils */

static inline int wrap(int i, int n) { return ((i % n) + n) % n; }

/* Row of a stencil neighbour: periodic, or, with walls, the mirror image in
 * the wall (row -1 reads row 0, row ny reads row ny - 1). Scalar fields
 * (rho, mu_c) are continued evenly across a wall; orc_fields reflects the
 * momentum (j_y changes sign) so that every vector field is the mirror
 * image of the real one. */
static inline int yrow(int walls, int y, int ny)
{
    if (!walls) return wrap(y, ny);
    return y < 0 ? -1 - y : (y >= ny ? 2 * ny - 1 - y : y);
}

/* Eq. 17: grad_h phi = (1/c_s^2) sum_a w_a phi(x + e_a) e_a. */
static void grad_w(int nx, int ny, int walls, const double* phi, double* gx, double* gy)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double sx = 0.0, sy = 0.0;
            for (int a = 0; a < Q; ++a) {
                double v = phi[yrow(walls, y + EY[a], ny) * nx + wrap(x + EX[a], nx)];
                sx += WA[a] * v * EX[a];
                sy += WA[a] * v * EY[a];
            }
            gx[y * nx + x] = sx / CS2;
            gy[y * nx + x] = sy / CS2;
        }
}

/* Isotropic Laplacian: (2/c_s^2) sum_a w_a (phi(x + e_a) - phi(x)). The paper
 * needs a Laplacian in Eq. 2 but does not print its stencil; this is the
 * 9-point isotropic form built from the same weights as Eq. 17. */
static void lap_w(int nx, int ny, int walls, const double* phi, double* out)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double c0 = phi[y * nx + x];
            double s = 0.0;
            for (int a = 0; a < Q; ++a)
                s += WA[a] * (phi[yrow(walls, y + EY[a], ny) * nx + wrap(x + EX[a], nx)] - c0);
            out[y * nx + x] = 2.0 * s / CS2;
        }
}

/* Periodic lattice-weight average sum_a w_a phi(x + e_a) (scheme 3). */
static void avg_w(int nx, int ny, const double* phi, double* out)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double s = 0.0;
            for (int a = 0; a < Q; ++a) s += WA[a] * phi[wrap(y + EY[a], ny) * nx + wrap(x + EX[a], nx)];
            out[y * nx + x] = s;
        }
}

/* The periodic forms. */
void orc_grad(int nx, int ny, const double* phi, double* gx, double* gy) { grad_w(nx, ny, 0, phi, gx, gy); }
void orc_laplacian(int nx, int ny, const double* phi, double* out) { lap_w(nx, ny, 0, phi, out); }

/* ------------------------------------------------------- moment algebra */

void orc_M(double* out) { memcpy(out, MM, sizeof(MM)); }

/* Gauss-Jordan inverse of M with partial pivoting. */
void orc_Minv(double* out)
{
    double A[Q][2 * Q];
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < 2 * Q; ++j) A[i][j] = (j < Q) ? MM[i][j] : (j - Q == i ? 1.0 : 0.0);
    for (int col = 0; col < Q; ++col) {
        int piv = col;
        for (int r = col + 1; r < Q; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int j = 0; j < 2 * Q; ++j) {
                double t = A[col][j];
                A[col][j] = A[piv][j];
                A[piv][j] = t;
            }
        double d = A[col][col];
        for (int j = 0; j < 2 * Q; ++j) A[col][j] /= d;
        for (int r = 0; r < Q; ++r) {
            if (r == col) continue;
            double m = A[r][col];
            if (m == 0.0) continue;
            for (int j = 0; j < 2 * Q; ++j) A[r][j] -= m * A[col][j];
        }
    }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) out[i * Q + j] = A[i][Q + j];
}

static void matvec(const double* A, const double* v, double* out)
{
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int j = 0; j < Q; ++j) s += A[i * Q + j] * v[j];
        out[i] = s;
    }
}

/* Moment-space equilibrium: Eq. 11 (standard) or Eq. 27 with
 * gamma = 3 p_m / rho and p_m = (c0 + mu_c)/3 (improved, Eq. 24). */
/* Schemes 1 and 3 share Eqs. 24-28 and differ only in how Eq. 29 is discretised. */
static int improved(const orc_case* c) { return c->scheme == 1 || c->scheme == 3; }

void orc_meq(const orc_case* c, double rho, double ux, double uy, double mu, double* meq)
{
    double u2 = ux * ux + uy * uy;
    if (!improved(c)) {
        meq[0] = rho;
        meq[1] = rho * (-2.0 + ((c->flags & 64) ? 0.0 : 3.0 * u2));  /* hook 64: the kinetic term dropped */
        meq[2] = rho * (1.0 - 3.0 * u2);
        meq[3] = rho * ux;
        meq[4] = -rho * ux;
        meq[5] = rho * uy;
        meq[6] = -rho * uy;
    } else {
        double pm = (c->pm_c0 + mu) / 3.0;
        double g = 3.0 * pm / rho;
        meq[0] = rho;
        meq[1] = rho * (-4.0 + 3.0 * u2 + 2.0 * g);
        meq[2] = rho * (4.0 - 3.0 * u2 - 3.0 * g);
        meq[3] = rho * ux;
        meq[4] = rho * (g - 2.0) * ux;
        meq[5] = rho * uy;
        meq[6] = rho * (g - 2.0) * uy;
    }
    meq[7] = rho * (ux * ux - uy * uy);
    meq[8] = rho * ux * uy;
}

/* Population-space equilibrium f_eq = M^-1 m_eq. */
void orc_feq(const orc_case* c, double rho, double ux, double uy, double mu, double* feq)
{
    double Mi[Q * Q], meq[Q];
    orc_Minv(Mi);
    orc_meq(c, rho, ux, uy, mu, meq);
    matvec(Mi, meq, feq);
}

/* Eq. 14: G_a = w_a [ (e_a - u)/c_s^2 + (e_a . u) e_a / c_s^4 ] . F */
void orc_guo(double ux, double uy, double Fx, double Fy, double* G)
{
    for (int a = 0; a < Q; ++a) {
        double eu = EX[a] * ux + EY[a] * uy;
        double vx = (EX[a] - ux) / CS2 + eu * EX[a] / (CS2 * CS2);
        double vy = (EY[a] - uy) / CS2 + eu * EY[a] / (CS2 * CS2);
        G[a] = WA[a] * (vx * Fx + vy * Fy);
    }
}

/* Shear relaxation time at a node. With nu > 0 it follows from the dynamic
 * viscosity: eta = p_m (tau_v - 1/2) for the improved scheme (below Eq. 29) and
 * eta = rho c_s^2 (tau_v - 1/2) for the standard one (below Eq. 8), eta = nu rho. */
double orc_tau_v(const orc_case* c, double rho, double mu)
{
    if (!(c->nu > 0.0)) return c->tau_v;
    const double pm = (c->pm_c0 + mu) / 3.0;
    if (improved(c) && (c->flags & 16)) return 0.5 + c->nu * pm / rho;
    if (improved(c) && !(c->flags & 32)) return 0.5 + c->nu * rho / pm;
    return 0.5 + c->nu / CS2;
}

/* Diagonal of Lambda: Eq. 8 (tau_c = 1) for MRT, all 1/tau_v for BGK. */
static void relax_rates(const orc_case* c, double tau_v, double* lam)
{
    if (c->collision == 0) {
        for (int i = 0; i < Q; ++i) lam[i] = 1.0 / tau_v;
        return;
    }
    lam[0] = 1.0;
    lam[1] = 1.0 / c->tau_e;
    lam[2] = 1.0 / c->tau_s;
    lam[3] = 1.0;
    lam[4] = 1.0 / c->tau_q;
    lam[5] = 1.0;
    lam[6] = 1.0 / c->tau_q;
    lam[7] = 1.0 / tau_v;
    lam[8] = 1.0 / tau_v;
}

/* ------------------------------------------------- macroscopic fields */

/* Stages 2-7 of the fields on a periodic lattice from given density and
 * momentum (the populations' moments). */
static int fields_core(const orc_case* c, const double* rho_in, const double* jx_in, const double* jy_in,
                       double* rho_o, double* ux_o, double* uy_o, double* mu_o, double* Fx_o, double* Fy_o,
                       double* C1_o, double* C7_o)
{
    const int nx = c->nx, ny = c->ny, N = nx * ny;
    double* rho = calloc(N, sizeof(double));
    double* lap = calloc(N, sizeof(double));
    double* mu = calloc(N, sizeof(double));
    double* gmx = calloc(N, sizeof(double));
    double* gmy = calloc(N, sizeof(double));
    double* grx = calloc(N, sizeof(double));
    double* gry = calloc(N, sizeof(double));
    double* ux = calloc(N, sizeof(double));
    double* uy = calloc(N, sizeof(double));
    double* Fx = calloc(N, sizeof(double));
    double* Fy = calloc(N, sizeof(double));
    double* A = calloc(N, sizeof(double));
    double* B = calloc(N, sizeof(double));
    double* Ax = calloc(N, sizeof(double));
    double* Ay = calloc(N, sizeof(double));
    double* Bx = calloc(N, sizeof(double));
    double* By = calloc(N, sizeof(double));
    int bad = 0;

    /* 1. density (summed by the caller) */
    for (int i = 0; i < N; ++i) {
        rho[i] = rho_in[i];
        if (!(rho[i] > 0.0) || !isfinite(rho[i])) bad = 1;
    }
    /* 2-3. chemical potential */
    lap_w(nx, ny, 0, rho, lap);
    for (int i = 0; i < N; ++i) mu[i] = orc_dEf(c, rho[i]) - c->kappa * lap[i];
    /* 4-5. force */
    grad_w(nx, ny, 0, mu, gmx, gmy);
    if (c->scheme == 0 || c->scheme == 4) {
        double* r3 = calloc(N, sizeof(double));
        for (int i = 0; i < N; ++i) r3[i] = rho[i] * CS2;
        grad_w(nx, ny, 0, r3, grx, gry);
        free(r3);
        for (int i = 0; i < N; ++i) {
            Fx[i] = grx[i] - rho[i] * gmx[i];
            Fy[i] = gry[i] - rho[i] * gmy[i];
        }
    } else if (c->scheme == 2) {
        /* pressure-tensor form: F = grad(rho c_s^2) - div P, with the non-local
         * pressure of Eq. 4 and the tensor of Eq. 5 built at every node from the
         * Eq. 17 gradient and the Laplacian of rho, then div P by Eq. 17 applied
         * to each component */
        double* r3 = calloc(N, sizeof(double));
        double* drx = calloc(N, sizeof(double));
        double* dry = calloc(N, sizeof(double));
        double* Pxx = calloc(N, sizeof(double));
        double* Pxy = calloc(N, sizeof(double));
        double* Pyy = calloc(N, sizeof(double));
        double* gx = calloc(N, sizeof(double));
        double* gy = calloc(N, sizeof(double));
        for (int i = 0; i < N; ++i) r3[i] = rho[i] * CS2;
        grad_w(nx, ny, 0, r3, grx, gry);
        grad_w(nx, ny, 0, rho, drx, dry);
        for (int i = 0; i < N; ++i) {
            double p = orc_pEOS(c, rho[i]) - c->kappa * rho[i] * lap[i] -
                       0.5 * c->kappa * (drx[i] * drx[i] + dry[i] * dry[i]);
            Pxx[i] = p + c->kappa * drx[i] * drx[i];
            Pyy[i] = p + c->kappa * dry[i] * dry[i];
            Pxy[i] = c->kappa * drx[i] * dry[i];
        }
        for (int i = 0; i < N; ++i) Fx[i] = grx[i], Fy[i] = gry[i];
        grad_w(nx, ny, 0, Pxx, gx, gy);
        for (int i = 0; i < N; ++i) Fx[i] -= gx[i];
        grad_w(nx, ny, 0, Pxy, gx, gy);
        for (int i = 0; i < N; ++i) Fx[i] -= gy[i], Fy[i] -= gx[i];
        grad_w(nx, ny, 0, Pyy, gx, gy);
        for (int i = 0; i < N; ++i) Fy[i] -= gy[i];
        free(r3); free(drx); free(dry); free(Pxx); free(Pxy); free(Pyy); free(gx); free(gy);
    } else {
        for (int i = 0; i < N; ++i) {
            Fx[i] = (CS2 - rho[i]) * gmx[i];
            Fy[i] = (CS2 - rho[i]) * gmy[i];
        }
    }
    /* 6. velocity; the Lax-Wendroff scheme's time step is A (Appendix A) */
    double half = (c->flags & 2) ? -0.5 : 0.5;
    if (c->scheme == 4) half *= c->lw_A;
    for (int i = 0; i < N; ++i) {
        ux[i] = (jx_in[i] + half * Fx[i]) / rho[i];
        uy[i] = (jy_in[i] + half * Fy[i]) / rho[i];
    }
    /* 7. correction term (improved scheme) */
    if (improved(c)) {
        for (int i = 0; i < N; ++i) {
            double pm = (c->pm_c0 + mu[i]) / 3.0;
            double phi = rho[i] * CS2 - pm;
            A[i] = phi * ux[i];
            B[i] = phi * uy[i];
        }
        if (c->scheme == 3) {
            /* the fields phi u_x, phi u_y replaced by their averages
             * sum_a w_a (phi u)(x + e_a) before the Eq. 17 gradient */
            double* t = malloc(N * sizeof(double));
            avg_w(nx, ny, A, t);
            memcpy(A, t, N * sizeof(double));
            avg_w(nx, ny, B, t);
            memcpy(B, t, N * sizeof(double));
            free(t);
        }
        grad_w(nx, ny, 0, A, Ax, Ay);
        grad_w(nx, ny, 0, B, Bx, By);
    }
    for (int i = 0; i < N; ++i) {
        if (!isfinite(mu[i]) || !isfinite(ux[i]) || !isfinite(uy[i])) bad = 1;
        if (rho_o) rho_o[i] = rho[i];
        if (ux_o) ux_o[i] = ux[i];
        if (uy_o) uy_o[i] = uy[i];
        if (mu_o) mu_o[i] = mu[i];
        if (Fx_o) Fx_o[i] = Fx[i];
        if (Fy_o) Fy_o[i] = Fy[i];
        if (C1_o) C1_o[i] = improved(c) ? Ax[i] + By[i] : 0.0;
        if (C7_o) C7_o[i] = improved(c) ? Ax[i] - By[i] : 0.0;
    }
    free(rho); free(lap); free(mu); free(gmx); free(gmy); free(grx); free(gry);
    free(ux); free(uy); free(Fx); free(Fy); free(A); free(B);
    free(Ax); free(Ay); free(Bx); free(By);
    return bad ? -1 : 0;
}

/* Stages 1-6 (and p_m, C of stage 7) over the lattice, from the populations
 * at the start of a step. Any output pointer may be NULL except as noted.
 * Returns 0, or -1 when rho <= 0 or a value is not finite somewhere.
 *
 * With walls, the stencils see the lattice continued across each wall by
 * its mirror image in the wall plane (y = -1/2 and y = ny - 1/2): G ghost
 * rows below y = 0 and above y = ny - 1 carry the reflected state of the
 * mirrored rows (row -k that of row k - 1): the same density and j_x, and
 * j_y with its sign changed, as reflecting the populations across the wall
 * gives. Every field (mu_c, gradients, F, u, phi u, C, P) is then computed
 * by the same stencils on the extended lattice, so that scalar fields come
 * out even across the wall and the y components of vector fields odd. */
int orc_fields(const orc_case* c, const double* f, double* rho_o, double* ux_o, double* uy_o,
               double* mu_o, double* Fx_o, double* Fy_o, double* C1_o, double* C7_o)
{
    const int nx = c->nx, ny = c->ny, N = nx * ny;
    double* rho = malloc(N * sizeof(double));
    double* jx = malloc(N * sizeof(double));
    double* jy = malloc(N * sizeof(double));
    for (int i = 0; i < N; ++i) {
        double s = 0.0, sx = 0.0, sy = 0.0;
        for (int a = 0; a < Q; ++a) {
            s += f[a * N + i];
            sx += EX[a] * f[a * N + i];
            sy += EY[a] * f[a * N + i];
        }
        rho[i] = s;
        jx[i] = sx;
        jy[i] = sy;
    }
    int rc;
    if (!c->walls) {
        rc = fields_core(c, rho, jx, jy, rho_o, ux_o, uy_o, mu_o, Fx_o, Fy_o, C1_o, C7_o);
    } else {
        /* ghost rows each side: the deepest stencil chain (C of scheme 3) reaches
         * 4 rows; the periodic wrap of the extended lattice corrupts only ghost rows */
        enum { G = 4 };
        orc_case ce = *c;
        ce.ny = ny + 2 * G;
        ce.walls = 0;
        const int Ne = nx * ce.ny;
        double* buf = malloc((size_t)11 * Ne * sizeof(double));
        double *re = buf, *xe = buf + Ne, *ye = buf + 2 * Ne;
        double* out[8];
        for (int k = 0; k < 8; ++k) out[k] = buf + (3 + k) * Ne;
        for (int g = 0; g < ce.ny; ++g) {
            const int y = yrow(1, g - G, ny);
            const int ghost = g < G || g >= G + ny;
            const double sy = ghost && !(c->flags & 8) ? -1.0 : 1.0;
            for (int x = 0; x < nx; ++x) {
                re[g * nx + x] = rho[y * nx + x];
                xe[g * nx + x] = jx[y * nx + x];
                ye[g * nx + x] = sy * jy[y * nx + x];
            }
        }
        rc = fields_core(&ce, re, xe, ye, out[0], out[1], out[2], out[3], out[4], out[5], out[6], out[7]);
        /* a bad value in a ghost row is a bad value of its mirrored row */
        double* dst[8] = {rho_o, ux_o, uy_o, mu_o, Fx_o, Fy_o, C1_o, C7_o};
        for (int k = 0; k < 8; ++k)
            if (dst[k]) memcpy(dst[k], out[k] + G * nx, (size_t)N * sizeof(double));
        free(buf);
    }
    free(rho);
    free(jx);
    free(jy);
    return rc;
}

/* ---------------------------------------------------------------- step */

/* Scheme 4, the Lax-Wendroff propagation scheme of Appendix A, nsteps steps
 * of dt = A. Per node, from the populations f at the start of a step:
 * rho, u, F from orc_fields (standard force, u with dt F / 2), the second
 * moment Pi = sum_a e_a e_a f_a, the tensor T of Eq. A4,
 *   rho c_s^2 dt (B - tau) T = Pi - rho c_s^2 I - rho u u - (tau - 1/2) dt (u F + F u),
 * the equilibrium of Eq. A3,
 *   f_eq,a = rho w_a [1 + e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u^2/(2 c_s^2)
 *                     + B dt (e_a e_a - c_s^2 I) : T / (2 c_s^2)],
 * the guo term G of Eq. 14 and the BGK collision of Eq. A1,
 *   f*_a = f_a - (f_a - f_eq,a) / tau + dt (1 - 1/(2 tau)) G_a;
 * then the propagation of Eq. A2 over the periodic lattice,
 *   f_a(x) <- a_0 f*_a(x) + a_1 f*_a(x + e_a) + a_-1 f*_a(x - e_a). */
static int64_t lw_step(const orc_case* c, double* f, int64_t nsteps, double* rho, double* ux, double* uy,
                       double* mu, double* Fx, double* Fy, double* C1, double* C7, double* fs_all)
{
    const int nx = c->nx, ny = c->ny, N = nx * ny;
    const double A = c->lw_A, B = c->lw_B, dt = A, tau = c->tau_v;
    const double a0 = 1.0 - A * A, a1 = A * (A - 1.0) / 2.0, am1 = A * (A + 1.0) / 2.0;
    int64_t done = 0;
    for (int64_t n = 0; n < nsteps; ++n) {
        if (orc_fields(c, f, rho, ux, uy, mu, Fx, Fy, C1, C7) != 0) break;
        for (int i = 0; i < N; ++i) {
            double fl[Q], G[Q];
            for (int a = 0; a < Q; ++a) fl[a] = f[a * N + i];
            const double r = rho[i], u[2] = {ux[i], uy[i]}, F[2] = {Fx[i], Fy[i]};
            double Pi[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
            for (int a = 0; a < Q; ++a) {
                const double e[2] = {(double)EX[a], (double)EY[a]};
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q) Pi[p][q] += e[p] * e[q] * fl[a];
            }
            double Tt[2][2];
            for (int p = 0; p < 2; ++p)
                for (int q = 0; q < 2; ++q)
                    Tt[p][q] = (Pi[p][q] - r * CS2 * (p == q ? 1.0 : 0.0) - r * u[p] * u[q] -
                                (tau - 0.5) * dt * (u[p] * F[q] + F[p] * u[q])) /
                               (r * CS2 * dt * (B - tau));
            orc_guo(u[0], u[1], F[0], F[1], G);
            for (int a = 0; a < Q; ++a) {
                const double e[2] = {(double)EX[a], (double)EY[a]};
                const double eu = e[0] * u[0] + e[1] * u[1], u2 = u[0] * u[0] + u[1] * u[1];
                double eeT = 0.0;
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q) eeT += (e[p] * e[q] - CS2 * (p == q ? 1.0 : 0.0)) * Tt[p][q];
                const double feq = r * WA[a] *
                                   (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - u2 / (2.0 * CS2) +
                                    B * dt * eeT / (2.0 * CS2));
                fs_all[a * N + i] = fl[a] - (fl[a] - feq) / tau + dt * (1.0 - 1.0 / (2.0 * tau)) * G[a];
            }
        }
        for (int a = 0; a < Q; ++a)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const double* fs = fs_all + a * N;
                    const int ip = wrap(y + EY[a], ny) * nx + wrap(x + EX[a], nx);
                    const int im = wrap(y - EY[a], ny) * nx + wrap(x - EX[a], nx);
                    f[a * N + y * nx + x] = a0 * fs[y * nx + x] + a1 * fs[ip] + am1 * fs[im];
                }
        ++done;
    }
    return done;
}

/* Advance f (in place, f[a][y][x]) by nsteps time steps. Returns the number
 * of steps completed; fewer than nsteps means the state became non-physical
 * (rho <= 0 or a non-finite value) before the step that was not taken. */
int64_t orc_step(const orc_case* c, double* f, int64_t nsteps)
{
    const int nx = c->nx, ny = c->ny, N = nx * ny;
    double Mi[Q * Q], lam[Q];
    orc_Minv(Mi);
    double* rho = malloc(N * sizeof(double));
    double* ux = malloc(N * sizeof(double));
    double* uy = malloc(N * sizeof(double));
    double* mu = malloc(N * sizeof(double));
    double* Fx = malloc(N * sizeof(double));
    double* Fy = malloc(N * sizeof(double));
    double* C1 = malloc(N * sizeof(double));
    double* C7 = malloc(N * sizeof(double));
    double* fn = malloc((size_t)Q * N * sizeof(double));
    /* moving-wall bounce-back (walls): the returning population gains the
     * difference of the running scheme's equilibria at the wall state
     * (rho_wall, u = (wall_u, 0), mu_c = E_f'(rho_wall)) */
    double wall_feq[Q];
    if (c->walls) orc_feq(c, c->rho_wall, c->wall_u, 0.0, orc_dEf(c, c->rho_wall), wall_feq);
    int64_t done = 0;
    if (c->scheme == 4) {
        done = lw_step(c, f, nsteps, rho, ux, uy, mu, Fx, Fy, C1, C7, fn);
        nsteps = 0;
    }
    for (int64_t n = 0; n < nsteps; ++n) {
        if (orc_fields(c, f, rho, ux, uy, mu, Fx, Fy, C1, C7) != 0) break;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int i = y * nx + x;
                double fl[Q], m[Q], meq[Q], G[Q], S[Q], Cv[Q], ms[Q], fs[Q];
                for (int a = 0; a < Q; ++a) fl[a] = f[a * N + i];
                /* 8. forcing, moments, equilibria */
                orc_guo(ux[i], uy[i], Fx[i], Fy[i], G);
                matvec(&MM[0][0], G, S);
                matvec(&MM[0][0], fl, m);
                orc_meq(c, rho[i], ux[i], uy[i], mu[i], meq);
                for (int k = 0; k < Q; ++k) Cv[k] = 0.0;
                if (improved(c) && !(c->flags & 1)) {
                    Cv[1] = 9.0 * C1[i];
                    Cv[7] = 3.0 * C7[i];
                }
                /* 9. collision in moment space */
                relax_rates(c, orc_tau_v(c, rho[i], mu[i]), lam);
                for (int k = 0; k < Q; ++k)
                    ms[k] = m[k] - lam[k] * (m[k] - meq[k]) + (1.0 - 0.5 * lam[k]) * (S[k] + Cv[k]);
                /* 10. back to populations */
                matvec(Mi, ms, fs);
                /* 11. push streaming; with walls, a population that would
                 * cross a wall returns to its node in the opposite direction
                 * (halfway bounce-back) plus the moving-wall term
                 * f_eq,b - f_eq,a of the wall state */
                for (int a = 0; a < Q; ++a) {
                    const int yy = y + EY[a];
                    if (c->walls && (yy < 0 || yy >= ny)) {
                        const int b = OPP[a];
                        fn[b * N + y * nx + x] = fs[a] + (wall_feq[b] - wall_feq[a]);
                    } else {
                        fn[a * N + wrap(yy, ny) * nx + wrap(x + EX[a], nx)] = fs[a];
                    }
                }
            }
        memcpy(f, fn, (size_t)Q * N * sizeof(double));
        ++done;
    }
    free(rho); free(ux); free(uy); free(mu); free(Fx); free(Fy); free(C1); free(C7); free(fn);
    return done;
}

/* Initial populations (no rule in the paper): f(0) = M^-1 m_eq(rho0, u0) of
 * the running scheme, with mu_c (hence p_m) from rho0 through Eq. 2.
 * ux0/uy0 may be NULL for a fluid at rest. Returns 0, or -1 if rho0 <= 0. */
int orc_init(const orc_case* c, const double* rho0, const double* ux0, const double* uy0, double* f)
{
    const int nx = c->nx, ny = c->ny, N = nx * ny;
    double* lap = malloc(N * sizeof(double));
    double Mi[Q * Q];
    orc_Minv(Mi);
    lap_w(nx, ny, c->walls, rho0, lap);
    int bad = 0;
    for (int i = 0; i < N; ++i) {
        if (!(rho0[i] > 0.0)) bad = 1;
        double mu = orc_dEf(c, rho0[i]) - c->kappa * lap[i];
        double meq[Q], fe[Q];
        orc_meq(c, rho0[i], ux0 ? ux0[i] : 0.0, uy0 ? uy0[i] : 0.0, mu, meq);
        matvec(Mi, meq, fe);
        for (int a = 0; a < Q; ++a) f[a * N + i] = fe[a];
    }
    free(lap);
    return bad ? -1 : 0;
}

/* ====================================================================== */
/* Adjoint (reverse-mode derivative) of the literal step above.            */
/*                                                                         */
/* Loss: L = sum_{n = u_from}^{N} sum_x |u^n(x)|^2 + sum_x s(x) rho^N(x),   */
/* with u^n, rho^n the fields (Eq. 12) of the state after n steps from      */
/* f(0) = init(rho0, u0 = 0). Every stage of orc_step is transposed in      */
/* reverse order, following the forward's own intermediate quantities;     */
/* stencil transposes are written as their own gathers (x - e_a). The       */
/* trajectory is rebuilt from checkpoints every K steps. Constant tau only. */
/* ====================================================================== */

/* d E_f'(rho) / d rho */
static double d2Ef(const orc_case* c, double rho)
{
    if (c->eos == 0) {
        double q = 1.0 / (1.0 - c->b * rho);
        return c->R * c->T * (1.0 / rho + c->b * q + c->b * q * q) - 2.0 * c->a;
    }
    double n = c->b * rho / 4.0, q = 1.0 / (1.0 - n);
    return c->R * c->T * (1.0 / rho + 0.25 * c->b * (8.0 - 2.0 * n) * q * q * q * q) - 2.0 * c->a;
}

/* d E_f'(rho) / d T */
static double dEf_dT(const orc_case* c, double rho)
{
    orc_case u = *c;
    u.T = 1.0;
    u.a = 0.0;
    return orc_dEf(&u, rho); /* R h(rho) */
}

/* transpose of the Eq. 17 stencil component: (G^T v)(y) = 3 sum_a w_a e_a v(y - e_a) */
static void gradT(int nx, int ny, const double* vx, const double* vy, double* out)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double s = 0.0;
            for (int a = 0; a < Q; ++a) {
                int i = wrap(y - EY[a], ny) * nx + wrap(x - EX[a], nx);
                if (vx) s += 3.0 * WA[a] * EX[a] * vx[i];
                if (vy) s += 3.0 * WA[a] * EY[a] * vy[i];
            }
            out[y * nx + x] = s;
        }
}

/* transpose of the Laplacian: (L^T v)(y) = 6 sum_a w_a (v(y - e_a) - v(y)) */
static void lapT(int nx, int ny, const double* v, double* out)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double s = 0.0;
            for (int a = 0; a < Q; ++a) s += WA[a] * (v[wrap(y - EY[a], ny) * nx + wrap(x - EX[a], nx)] - v[y * nx + x]);
            out[y * nx + x] = 6.0 * s;
        }
}

typedef struct {
    double *rho, *lap, *mu, *gmx, *gmy, *Fx, *Fy, *jx, *jy, *ux, *uy, *phi, *C1, *C7;
} orc_fwd;

static void fwd_alloc(orc_fwd* w, int N)
{
    double** p = (double**)w;
    for (int k = 0; k < (int)(sizeof(orc_fwd) / sizeof(double*)); ++k) p[k] = calloc(N, sizeof(double));
}
static void fwd_free(orc_fwd* w)
{
    double** p = (double**)w;
    for (int k = 0; k < (int)(sizeof(orc_fwd) / sizeof(double*)); ++k) free(p[k]);
}

/* the intermediate fields of stages 1-7 at state f (same arithmetic as orc_fields) */
static void fwd_fields(const orc_case* c, const double* f, orc_fwd* w)
{
    const int nx = c->nx, ny = c->ny, N = nx * ny;
    double* r3 = calloc(N, sizeof(double));
    double* grx = calloc(N, sizeof(double));
    double* gry = calloc(N, sizeof(double));
    double* Ax = calloc(N, sizeof(double));
    double* Ay = calloc(N, sizeof(double));
    double* Bx = calloc(N, sizeof(double));
    double* By = calloc(N, sizeof(double));
    double* A = calloc(N, sizeof(double));
    double* B = calloc(N, sizeof(double));
    for (int i = 0; i < N; ++i) {
        double s = 0.0, jx = 0.0, jy = 0.0;
        for (int a = 0; a < Q; ++a) {
            s += f[a * N + i];
            jx += EX[a] * f[a * N + i];
            jy += EY[a] * f[a * N + i];
        }
        w->rho[i] = s;
        w->jx[i] = jx;
        w->jy[i] = jy;
    }
    orc_laplacian(nx, ny, w->rho, w->lap);
    for (int i = 0; i < N; ++i) w->mu[i] = orc_dEf(c, w->rho[i]) - c->kappa * w->lap[i];
    orc_grad(nx, ny, w->mu, w->gmx, w->gmy);
    if (c->scheme == 0) {
        for (int i = 0; i < N; ++i) r3[i] = w->rho[i] * CS2;
        orc_grad(nx, ny, r3, grx, gry);
    }
    for (int i = 0; i < N; ++i) {
        if (c->scheme == 0) {
            w->Fx[i] = grx[i] - w->rho[i] * w->gmx[i];
            w->Fy[i] = gry[i] - w->rho[i] * w->gmy[i];
        } else {
            w->Fx[i] = (CS2 - w->rho[i]) * w->gmx[i];
            w->Fy[i] = (CS2 - w->rho[i]) * w->gmy[i];
        }
        w->ux[i] = (w->jx[i] + 0.5 * w->Fx[i]) / w->rho[i];
        w->uy[i] = (w->jy[i] + 0.5 * w->Fy[i]) / w->rho[i];
    }
    if (c->scheme == 1) {
        for (int i = 0; i < N; ++i) {
            double pm = (c->pm_c0 + w->mu[i]) / 3.0;
            w->phi[i] = w->rho[i] * CS2 - pm;
            A[i] = w->phi[i] * w->ux[i];
            B[i] = w->phi[i] * w->uy[i];
        }
        orc_grad(nx, ny, A, Ax, Ay);
        orc_grad(nx, ny, B, Bx, By);
        for (int i = 0; i < N; ++i) {
            w->C1[i] = Ax[i] + By[i];
            w->C7[i] = Ax[i] - By[i];
        }
    }
    free(r3); free(grx); free(gry); free(Ax); free(Ay); free(Bx); free(By); free(A); free(B);
}

/* Transpose of stages 1-7 at state w: given the adjoints of the node-level
 * quantities (rb = rho, jxb, jyb, uxb, uyb, Fxb, Fyb, mub, C1b, C7b; all are
 * consumed), add to lam_f[a][i] and to the parameter gradients. */
static void fields_vjp(const orc_case* c, const orc_fwd* w, double* rb, double* jxb, double* jyb, double* uxb,
                       double* uyb, double* Fxb, double* Fyb, double* mub, double* C1b, double* C7b,
                       double* lam_f, double* g_kappa, double* g_T)
{
    const int nx = c->nx, ny = c->ny, N = nx * ny;
    double* t1 = calloc(N, sizeof(double));
    double* t2 = calloc(N, sizeof(double));
    double* gmxb = calloc(N, sizeof(double));
    double* gmyb = calloc(N, sizeof(double));
    /* 7': C1 = Ax + By, C7 = Ax - By; A = phi ux, B = phi uy; phi = rho/3 - (c0 + mu)/3 */
    if (c->scheme == 1) {
        double* Axb = calloc(N, sizeof(double));
        double* Byb = calloc(N, sizeof(double));
        for (int i = 0; i < N; ++i) {
            Axb[i] = C1b[i] + C7b[i];
            Byb[i] = C1b[i] - C7b[i];
        }
        gradT(nx, ny, Axb, NULL, t1); /* A-bar */
        gradT(nx, ny, NULL, Byb, t2); /* B-bar */
        for (int i = 0; i < N; ++i) {
            double phib = t1[i] * w->ux[i] + t2[i] * w->uy[i];
            uxb[i] += w->phi[i] * t1[i];
            uyb[i] += w->phi[i] * t2[i];
            rb[i] += phib * CS2;
            mub[i] -= phib / 3.0;
        }
        free(Axb); free(Byb);
    }
    /* 6': u = (j + F/2) / rho */
    double half = (c->flags & 2) ? -0.5 : 0.5;
    for (int i = 0; i < N; ++i) {
        double r = w->rho[i];
        jxb[i] += uxb[i] / r;
        jyb[i] += uyb[i] / r;
        Fxb[i] += half * uxb[i] / r;
        Fyb[i] += half * uyb[i] / r;
        rb[i] -= (uxb[i] * w->ux[i] + uyb[i] * w->uy[i]) / r;
    }
    /* 5': force */
    for (int i = 0; i < N; ++i) {
        if (c->scheme == 0) {
            gmxb[i] = -w->rho[i] * Fxb[i];
            gmyb[i] = -w->rho[i] * Fyb[i];
        } else {
            gmxb[i] = (CS2 - w->rho[i]) * Fxb[i];
            gmyb[i] = (CS2 - w->rho[i]) * Fyb[i];
        }
        rb[i] -= w->gmx[i] * Fxb[i] + w->gmy[i] * Fyb[i];
    }
    if (c->scheme == 0) { /* F includes grad(rho/3) */
        gradT(nx, ny, Fxb, Fyb, t1);
        for (int i = 0; i < N; ++i) rb[i] += t1[i] * CS2;
    }
    /* 4': g = grad mu */
    gradT(nx, ny, gmxb, gmyb, t1);
    for (int i = 0; i < N; ++i) mub[i] += t1[i];
    /* 3': mu = E_f'(rho) - kappa lap */
    for (int i = 0; i < N; ++i) {
        rb[i] += d2Ef(c, w->rho[i]) * mub[i];
        *g_kappa -= mub[i] * w->lap[i];
        *g_T += mub[i] * dEf_dT(c, w->rho[i]);
        t2[i] = -c->kappa * mub[i];
    }
    /* 2': lap */
    lapT(nx, ny, t2, t1);
    for (int i = 0; i < N; ++i) rb[i] += t1[i];
    /* 1': rho = sum f, j = sum e f */
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < Q; ++a) lam_f[a * N + i] += rb[i] + EX[a] * jxb[i] + EY[a] * jyb[i];
    free(t1); free(t2); free(gmxb); free(gmyb);
}

/* d meq / d (rho, ux, uy, mu): rows k, columns (rho, ux, uy, mu) */
static void meq_jac(const orc_case* c, double rho, double ux, double uy, double mu, double J[Q][4])
{
    double u2 = ux * ux + uy * uy;
    for (int k = 0; k < Q; ++k) J[k][0] = J[k][1] = J[k][2] = J[k][3] = 0.0;
    J[0][0] = 1.0;
    if (c->scheme == 0) {
        J[1][0] = -2.0 + 3.0 * u2; J[1][1] = 6.0 * rho * ux; J[1][2] = 6.0 * rho * uy;
        J[2][0] = 1.0 - 3.0 * u2;  J[2][1] = -6.0 * rho * ux; J[2][2] = -6.0 * rho * uy;
        J[4][0] = -ux; J[4][1] = -rho;
        J[6][0] = -uy; J[6][2] = -rho;
    } else {
        double s = c->pm_c0 + mu; /* rho * gamma */
        J[1][0] = -4.0 + 3.0 * u2; J[1][1] = 6.0 * rho * ux; J[1][2] = 6.0 * rho * uy; J[1][3] = 2.0;
        J[2][0] = 4.0 - 3.0 * u2;  J[2][1] = -6.0 * rho * ux; J[2][2] = -6.0 * rho * uy; J[2][3] = -3.0;
        J[4][0] = -2.0 * ux; J[4][1] = s - 2.0 * rho; J[4][3] = ux;
        J[6][0] = -2.0 * uy; J[6][2] = s - 2.0 * rho; J[6][3] = uy;
    }
    J[3][0] = ux; J[3][1] = rho;
    J[5][0] = uy; J[5][2] = rho;
    J[7][0] = ux * ux - uy * uy; J[7][1] = 2.0 * rho * ux; J[7][2] = -2.0 * rho * uy;
    J[8][0] = ux * uy; J[8][1] = rho * uy; J[8][2] = rho * ux;
}

/* One reverse step: lam (in: adjoint of the state after the step, node
 * convention; out: adjoint of the state f before it, plus the u seeds at f).
 * u_seed != 0 adds the derivative of sum |u|^2 at state f. */
static void step_vjp(const orc_case* c, const double* f, double* lam, int u_seed, double* g_kappa, double* g_T)
{
    const int nx = c->nx, ny = c->ny, N = nx * ny;
    double Mi[Q * Q], lamr[Q];
    orc_Minv(Mi);
    relax_rates(c, c->tau_v, lamr);
    orc_fwd w;
    fwd_alloc(&w, N);
    fwd_fields(c, f, &w);
    double* ls = malloc((size_t)Q * N * sizeof(double));
    double* lf = calloc((size_t)Q * N, sizeof(double));
    double *rb = calloc(N, sizeof(double)), *jxb = calloc(N, sizeof(double)), *jyb = calloc(N, sizeof(double));
    double *uxb = calloc(N, sizeof(double)), *uyb = calloc(N, sizeof(double));
    double *Fxb = calloc(N, sizeof(double)), *Fyb = calloc(N, sizeof(double));
    double *mub = calloc(N, sizeof(double)), *C1b = calloc(N, sizeof(double)), *C7b = calloc(N, sizeof(double));
    /* 11': transpose of push streaming */
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int a = 0; a < Q; ++a)
                ls[a * N + y * nx + x] = lam[a * N + wrap(y + EY[a], ny) * nx + wrap(x + EX[a], nx)];
    for (int i = 0; i < N; ++i) {
        double msb[Q], mb[Q], meqb[Q], Sb[Q], Gb[Q], J[Q][4];
        /* 10': fs = Minv ms */
        for (int k = 0; k < Q; ++k) {
            double s = 0.0;
            for (int a = 0; a < Q; ++a) s += Mi[a * Q + k] * ls[a * N + i];
            msb[k] = s;
        }
        /* 9': ms = m - L (m - meq) + (1 - L/2)(S + C) */
        for (int k = 0; k < Q; ++k) {
            mb[k] = (1.0 - lamr[k]) * msb[k];
            meqb[k] = lamr[k] * msb[k];
            Sb[k] = (1.0 - 0.5 * lamr[k]) * msb[k];
        }
        if (c->scheme == 1 && !(c->flags & 1) && !(c->flags & 4)) {
            C1b[i] += 9.0 * Sb[1];
            C7b[i] += 3.0 * Sb[7];
        }
        /* 8': m = M f, S = M G, meq(rho, u, mu), G(u, F) */
        for (int a = 0; a < Q; ++a) {
            double s = 0.0, g = 0.0;
            for (int k = 0; k < Q; ++k) {
                s += MM[k][a] * mb[k];
                g += MM[k][a] * Sb[k];
            }
            lf[a * N + i] += s;
            Gb[a] = g;
        }
        meq_jac(c, w.rho[i], w.ux[i], w.uy[i], w.mu[i], J);
        for (int k = 0; k < Q; ++k) {
            rb[i] += J[k][0] * meqb[k];
            uxb[i] += J[k][1] * meqb[k];
            uyb[i] += J[k][2] * meqb[k];
            mub[i] += J[k][3] * meqb[k];
        }
        {
            double ux = w.ux[i], uy = w.uy[i], Fx = w.Fx[i], Fy = w.Fy[i];
            for (int a = 0; a < Q; ++a) {
                double eu = EX[a] * ux + EY[a] * uy, eF = EX[a] * Fx + EY[a] * Fy;
                double vx = (EX[a] - ux) / CS2 + eu * EX[a] / (CS2 * CS2);
                double vy = (EY[a] - uy) / CS2 + eu * EY[a] / (CS2 * CS2);
                Fxb[i] += Gb[a] * WA[a] * vx;
                Fyb[i] += Gb[a] * WA[a] * vy;
                uxb[i] += Gb[a] * WA[a] * (-Fx / CS2 + EX[a] * eF / (CS2 * CS2));
                uyb[i] += Gb[a] * WA[a] * (-Fy / CS2 + EY[a] * eF / (CS2 * CS2));
            }
        }
        if (u_seed) {
            uxb[i] += 2.0 * w.ux[i];
            uyb[i] += 2.0 * w.uy[i];
        }
    }
    fields_vjp(c, &w, rb, jxb, jyb, uxb, uyb, Fxb, Fyb, mub, C1b, C7b, lf, g_kappa, g_T);
    memcpy(lam, lf, (size_t)Q * N * sizeof(double));
    free(ls); free(lf); free(rb); free(jxb); free(jyb); free(uxb); free(uyb); free(Fxb); free(Fyb);
    free(mub); free(C1b); free(C7b);
    fwd_free(&w);
}

/* Adjoint of the initial populations f(0) = M^-1 m_eq(rho0, 0, mu(rho0)). */
static void init_vjp(const orc_case* c, const double* rho0, const double* lam0, double* g_rho0, double* g_kappa,
                     double* g_T)
{
    const int nx = c->nx, ny = c->ny, N = nx * ny;
    double Mi[Q * Q];
    orc_Minv(Mi);
    double* lap = calloc(N, sizeof(double));
    double* mub = calloc(N, sizeof(double));
    double* t = calloc(N, sizeof(double));
    orc_laplacian(nx, ny, rho0, lap);
    for (int i = 0; i < N; ++i) {
        double mu = orc_dEf(c, rho0[i]) - c->kappa * lap[i];
        double J[Q][4], meqb[Q];
        for (int k = 0; k < Q; ++k) {
            double s = 0.0;
            for (int a = 0; a < Q; ++a) s += Mi[a * Q + k] * lam0[a * N + i];
            meqb[k] = s;
        }
        meq_jac(c, rho0[i], 0.0, 0.0, mu, J);
        double rb = 0.0, mb = 0.0;
        for (int k = 0; k < Q; ++k) {
            rb += J[k][0] * meqb[k];
            mb += J[k][3] * meqb[k];
        }
        g_rho0[i] = rb + d2Ef(c, rho0[i]) * mb;
        mub[i] = mb;
        *g_kappa -= mb * lap[i];
        *g_T += mb * dEf_dT(c, rho0[i]);
        t[i] = -c->kappa * mb;
    }
    double* lt = calloc(N, sizeof(double));
    lapT(nx, ny, t, lt);
    for (int i = 0; i < N; ++i) g_rho0[i] += lt[i];
    free(lap); free(mub); free(t); free(lt);
}

/* Loss and gradients with respect to rho0, kappa and T (see the block
 * comment above). Returns 0, or -1 on a non-physical state or nu > 0. */
int orc_adjoint(const orc_case* c, const double* rho0, int64_t nsteps, int64_t u_from, const double* s_final,
                double* loss, double* g_rho0, double* g_kappa, double* g_T)
{
    const int nx = c->nx, ny = c->ny, N = nx * ny;
    if (c->nu > 0.0 || nsteps < 0 || c->scheme == 2 || c->scheme == 3 || c->scheme == 4 || c->walls)
        return -1; /* periodic, chemical-potential forms, Eq. 17 correction */
    int64_t K = 1;
    while (K * K < nsteps) ++K;
    const int64_t ncp = nsteps / K + 1;
    double* cp = malloc((size_t)ncp * Q * N * sizeof(double));
    double* f = malloc((size_t)Q * N * sizeof(double));
    if (orc_init(c, rho0, NULL, NULL, f) != 0) {
        free(cp);
        free(f);
        return -1;
    }
    /* forward: loss and checkpoints of the states 0, K, 2K, ... */
    double L = 0.0;
    orc_fwd w;
    fwd_alloc(&w, N);
    for (int64_t n = 0; n <= nsteps; ++n) {
        if (n % K == 0) memcpy(cp + (size_t)(n / K) * Q * N, f, (size_t)Q * N * sizeof(double));
        if (n >= u_from || n == nsteps) {
            fwd_fields(c, f, &w);
            for (int i = 0; i < N; ++i) {
                if (n >= u_from) L += w.ux[i] * w.ux[i] + w.uy[i] * w.uy[i];
                if (n == nsteps && s_final) L += s_final[i] * w.rho[i];
            }
        }
        if (n < nsteps && orc_step(c, f, 1) != 1) {
            fwd_free(&w); free(cp); free(f);
            return -1;
        }
    }
    fwd_free(&w);
    *loss = L;
    *g_kappa = 0.0;
    *g_T = 0.0;
    /* reverse sweep over segments [s, e] of at most K + 1 states, rebuilt
     * from the checkpoint at s; lam holds the adjoint of the state after n */
    double* lam = calloc((size_t)Q * N, sizeof(double));
    double* seg = malloc((size_t)(K + 1) * Q * N * sizeof(double));
    for (int64_t s = (nsteps / K) * K, e = nsteps; s >= 0; e = s - 1, s -= K) {
        memcpy(seg, cp + (size_t)(s / K) * Q * N, (size_t)Q * N * sizeof(double));
        for (int64_t n = s + 1; n <= e; ++n) {
            memcpy(seg + (size_t)(n - s) * Q * N, seg + (size_t)(n - s - 1) * Q * N, (size_t)Q * N * sizeof(double));
            orc_step(c, seg + (size_t)(n - s) * Q * N, 1);
        }
        for (int64_t n = e; n >= s; --n) {
            const double* fn = seg + (size_t)(n - s) * Q * N;
            if (n == nsteps) {
                /* final state: no later step; its u terms and the density term */
                memset(lam, 0, (size_t)Q * N * sizeof(double));
                if (nsteps >= u_from) step_vjp(c, fn, lam, 1, g_kappa, g_T);
                if (s_final)
                    for (int i = 0; i < N; ++i)
                        for (int a = 0; a < Q; ++a) lam[a * N + i] += s_final[i];
            } else {
                step_vjp(c, fn, lam, n >= u_from, g_kappa, g_T);
            }
        }
    }
    init_vjp(c, rho0, lam, g_rho0, g_kappa, g_T);
    free(lam); free(seg); free(cp); free(f);
    return 0;
}
