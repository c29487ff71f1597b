/*
 * FP64 CPU oracle for one time step of the coupled cascaded central-moment lattice Boltzmann
 * schemes of Hajabdollahi, Premnath & Welch, "Central Moment Lattice Boltzmann Method using a
 * Pressure-based Formulation for Multiphase Flows at High Density Ratios and including Effects
 * of Surface Tension and Marangoni Stresses" (arXiv:1909.04166).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct definition that the CUDA
 * library is checked against.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never calls it and shares no code with it.
 *
 * Scope (one time step, both D2Q9 lattices):
 *   - fluid lattice: pressure-based cascaded LB for the modified continuous Boltzmann equation,
 *     Sec. 4 (Eqs. cascadedLBEtwophaseflowexplicit, sourcetermcumulativetransformed,
 *     cumulativesourcetermcomponents, cascadedcollisionoperator, postcollisioncascadedLBscheme,
 *     hydrodynamicfields, fluidviscosity);
 *   - interface lattice: cascaded LB for the conservative Allen-Cahn equation, Sec. 5
 *     (Eqs. ACEcollisionLB, ACEstreamingLB and the g-hat / f-tilde expressions);
 *   - geometric surface tension with Marangoni stress, Sec. 2 Eq. surfacetensiongeometric and
 *     Sec. 6.7 Eqs. surfacetensiongeometricsurfactantsxcomp/ycomp, with sigma driven by a
 *     prescribed linear temperature field;
 *   - linear property interpolation, Sec. 2 Eq. sfluidpropertiesinterpolation.
 *
 * Readings taken where the paper is silent or misprinted (the CUDA library takes the same ones):
 *   R1  rho = rho_B + phi (rho_A - rho_B), mu likewise (Eq. sfluidpropertiesinterpolation prints
 *       (phi - phi_A), which would put rho_B in phase A; phi_A = 1, phi_B = 0).
 *   R2  m-hat^s'_8 uses +4 sigma'_00 (projection of S on K_8; the paper prints -8).
 *   R3  g-hat_7 uses -(3/2) u_x g-hat_3 (the paper prints u_y; the mirror of g-hat_6).
 *   R4  kappa-tilde = (3/2) sigma W (the coefficient that makes the integral of
 *       kappa-tilde |grad phi|^2 across the tanh profile equal sigma; Sec. 2).
 *   R5  curvature: |grad phi|^2 div n = |grad phi| (lap phi - n.H.n), H the Hessian of phi.
 *   R6  n = grad phi / (|grad phi| + 1e-6): Sec. 2 leaves n undefined where grad phi vanishes;
 *       the regularisation keeps rounding noise in the bulk phases (|grad phi| ~ 1e-7) from
 *       setting the direction of the sharpening flux M theta n and of F_s, and changes n by
 *       less than 1e-3 wherever |grad phi| > 1e-3.
 *   R7  F_p = -grad p* + c_s^2 (rho_A - rho_B) grad phi with p* = sum of the streamed g-bar
 *       (Sec. 3 Eq. netgradientpressureforce, Sec. 4 remark on grad rho).
 *   R8  no-slip walls: half-way bounce-back on both lattices; stencils use mirror ghosts.
 *   R9  omega_4 = omega_5 from the local viscosity, all other fluid omegas 1; omega^phi_1 =
 *       omega^phi_2 from M_phi, all other interface omegas 1 (Secs. 4 and 5).
 *   R10 initial populations are the equilibria (no -S/2 shift); the interface equilibrium at
 *       initialisation has its M_phi theta n term set to zero.
 *   R11 F_ext = (rho - rho_ref) g.
 *   R14 free-slip walls (Secs. 6.4-6.6): specular reflection half a node outside the last node;
 *       a population crossing such a wall keeps its tangential velocity, reverses the normal
 *       one and lands on the tangential neighbour inside; a population crossing a free-slip
 *       and a no-slip wall at a corner bounces back.  Stencils use mirror ghosts as in R8.
 *   R15 single relaxation time (Sec. 7): the cascaded operators of Secs. 4 and 5 with every
 *       relaxation rate equal to the shear rate (fluid) or to omega^phi_{1,2} (interface); with
 *       equal rates both reduce to relaxing all central moments at one rate.
 *   R16 Langmuir isotherm (Sec. 6.7): kappa-tilde(psi) = (3/2) W sigma0 [1 + beta ln(1 - psi)]
 *       for an imposed psi = psi0 + gradpsi . x, with the analytic gradient of kappa-tilde.
 *   R17 imposed shear flow (Sec. 6.1): the interface lattice alone, advected by the single-vortex
 *       field at node positions (x, y) = (i, j) with L0 = nx along x and ny along y, reversed for
 *       time levels t >= reverse_step; the fluid populations are carried unchanged.
 *
 * Pins of the force coupling (tests/test_oracle_pins.py, tests/test_oracle_physics.py): the
 * F != 0 terms of the fluid collision (R13) equal relaxation of the half-force-corrected
 * moments; the c_s^2 (rho_A - rho_B) grad phi part of F_p keeps a drop in a uniform stream
 * moving at the stream's speed; the -grad p* part advects p, so a pressure wave in a uniform
 * stream follows the linear modes of the paper's macroscopic equations.  Not separable by any
 * test: p* in place of the corrected p inside that gradient (R7); the two differ by
 * F_p . u / 2, second order in the flow.  That one reading is parity unpinned: the GPU path
 * takes it too and matches this file element by element, but no test would tell it from p.
 *
 * Layout: a population field is 9 planes [alpha][y][x], plane size nx*ny, row-major in x.
 * Node coordinates are (x, y) = (i, j), i in [0, nx), j in [0, ny).
 * Arithmetic: IEEE double, compiled without contraction (-ffp-contract=off).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 velocities in the paper's ordering, Sec. 4 Eq. particlevelocities. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

/* c_s^2 = c_sphi^2 = 1/3, Sec. 5. */
#define CS2 (1.0 / 3.0)

/* Regularisation of the interface normal (reading R6).  The tests may set another value
 * (orc_set_normal_eps) to check that the pins of R6 reject materially different ones. */
static double NORMAL_EPS = 1e-6;

/* Boundary kind of one side of the grid. */
#define BC_PERIODIC 0
#define BC_NOSLIP 1
#define BC_FREESLIP 2

typedef struct {
    int nx, ny;
    int bc_x0, bc_x1;          /* left (x = 0) and right (x = nx - 1) sides: BC_* */
    int bc_y0, bc_y1;          /* bottom (y = 0) and top (y = ny - 1) sides */
    double rho_a, rho_b;       /* phase A is phi = 1 */
    double mu_a, mu_b;         /* dynamic viscosities */
    double sigma0, dsigma_dT;  /* sigma(T) = sigma0 + dsigma_dT (T - T0) */
    double T0, gradT_x, gradT_y;   /* T(x, y) = T0 + gradT_x x + gradT_y y */
    double mobility, width;    /* M_phi, W */
    double gx, gy, rho_ref;    /* F_ext = (rho - rho_ref) (gx, gy) */
    int collision;             /* 0 cascaded (Secs. 4, 5); 1 single relaxation time (R15) */
    int sigma_model;           /* 0 sigma linear in T; 1 Langmuir isotherm in psi (R16) */
    double beta;               /* Gibbs elasticity number of the Langmuir isotherm */
    double psi0, gradpsi_x, gradpsi_y;   /* imposed psi = psi0 + gradpsi_x x + gradpsi_y y */
    int flow;                  /* 0 coupled lattices; 1 interface lattice in the imposed shear (R17) */
    int reverse_step;          /* imposed flow reversed for t >= reverse_step (<= 0: never) */
    double u0;                 /* imposed flow amplitude U_0 */
    int t;                     /* time level of the state (used by the imposed flow only) */
} orc_case;

/* Per-node macroscopic quantities of a step, exposed for the tests. */
typedef struct {
    double phi, rho, mu, omega_nu;
    double pstar, p, ux, uy;
    double dphix, dphiy, lap, hxx, hyy, hxy, dpx, dpy;
    double nx, ny, theta;
    double Fsx, Fsy, Ftx, Fty, Fpx, Fpy;
} orc_node;

/* ---------------------------------------------------------------------------------------------
 * Equilibria (initialisation, R10)
 * ------------------------------------------------------------------------------------------- */

/* Solve the 9x9 system sum_alpha ex^m ey^n pop_alpha = raw_mn for the populations, with the
 * moment order (00,10,01,20,02,11,21,12,22) of Sec. 4 Eq. discreterawmoments.  Plain Gaussian
 * elimination with partial pivoting. */
static void raw_to_populations(const double raw[9], double pop[9])
{
    static const int MX[9] = {0, 1, 0, 2, 0, 1, 2, 1, 2};
    static const int MY[9] = {0, 0, 1, 0, 2, 1, 1, 2, 2};
    double A[9][10];
    for (int r = 0; r < 9; ++r) {
        for (int a = 0; a < 9; ++a) A[r][a] = pow((double)EX[a], MX[r]) * pow((double)EY[a], MY[r]);
        A[r][9] = raw[r];
    }
    for (int c = 0; c < 9; ++c) {
        int piv = c;
        for (int r = c + 1; r < 9; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k < 10; ++k) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
        for (int r = 0; r < 9; ++r) {
            if (r == c) continue;
            double m = A[r][c] / A[c][c];
            for (int k = c; k < 10; ++k) A[r][k] -= m * A[c][k];
        }
    }
    for (int r = 0; r < 9; ++r) pop[r] = A[r][9] / A[r][r];
}

/* Central moments (order 00,10,01,20,02,11,21,12,22) about u -> raw moments, by the binomial
 * expansion of e^m e^n = ((e-u)+u)^m ((e-u)+u)^n. */
static void central_to_raw(const double c[9], double ux, double uy, double raw[9])
{
    /* position of the central moment (i, j), i, j <= 2, in the moment order above */
    static const int IDX[3][3] = {{0, 2, 4}, {1, 5, 7}, {3, 6, 8}};
    static const int MX[9] = {0, 1, 0, 2, 0, 1, 2, 1, 2};
    static const int MY[9] = {0, 0, 1, 0, 2, 1, 1, 2, 2};
    static const double BIN[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}};
    for (int r = 0; r < 9; ++r) {
        int m = MX[r], n = MY[r];
        double s = 0.0;
        for (int i = 0; i <= m; ++i)
            for (int j = 0; j <= n; ++j)
                s += BIN[m][i] * BIN[n][j] * pow(ux, m - i) * pow(uy, n - j) * c[IDX[i][j]];
        raw[r] = s;
    }
}

/* g^eq populations: discrete central moments matched to the continuous central moments of the
 * transformed Maxwellian, Sec. 3 Eq. centralmomentsgeqcomponents and Sec. 4 Eq. matchingmoments. */
void orc_geq(double p, double ux, double uy, double rho, double g[9])
{
    const double psi = p - rho * CS2;
    double c[9];
    c[0] = p;
    c[1] = -psi * ux;
    c[2] = -psi * uy;
    c[3] = p * CS2 + psi * ux * ux;
    c[4] = p * CS2 + psi * uy * uy;
    c[5] = psi * ux * uy;
    c[6] = -psi * (CS2 + ux * ux) * uy;
    c[7] = -psi * (CS2 + uy * uy) * ux;
    c[8] = CS2 * CS2 * CS2 * rho + psi * (ux * ux + CS2) * (uy * uy + CS2);
    double raw[9];
    central_to_raw(c, ux, uy, raw);
    raw_to_populations(raw, g);
}

/* f^eq populations from the matched central moments of Sec. 5 (kappa-hat^eq list); jx, jy are
 * the first-order central moments M_phi theta n (zero at initialisation, R10). */
void orc_feq(double phi, double ux, double uy, double jx, double jy, double f[9])
{
    double c[9];
    c[0] = phi;
    c[1] = jx;
    c[2] = jy;
    c[3] = CS2 * phi;
    c[4] = CS2 * phi;
    c[5] = 0.0;
    c[6] = 0.0;
    c[7] = 0.0;
    c[8] = CS2 * CS2 * phi;
    double raw[9];
    central_to_raw(c, ux, uy, raw);
    raw_to_populations(raw, f);
}

/* ---------------------------------------------------------------------------------------------
 * Collision kernels (one node)
 * ------------------------------------------------------------------------------------------- */

/* Raw moments of nine populations in the order (00,10,01,20,02,11,21,12,22),
 * Sec. 4 Eq. discreterawmoments / Sec. 5 Eq. discreterawmomentsACE. */
static void raw_moments(const double q[9], double r[9])
{
    for (int k = 0; k < 9; ++k) r[k] = 0.0;
    for (int a = 0; a < 9; ++a) {
        const double ex = EX[a], ey = EY[a];
        r[0] += q[a];
        r[1] += q[a] * ex;
        r[2] += q[a] * ey;
        r[3] += q[a] * ex * ex;
        r[4] += q[a] * ey * ey;
        r[5] += q[a] * ex * ey;
        r[6] += q[a] * ex * ex * ey;
        r[7] += q[a] * ex * ey * ey;
        r[8] += q[a] * ex * ex * ey * ey;
    }
}

/* Source raw moments sigma', projected source moments m-hat^s' and the cumulative source term
 * delta g^s of Sec. 4 (sigma' list, m-hat^s' list with reading R2, and Eq.
 * cumulativesourcetermcomponents).  omega: the nine fluid relaxation rates. */
void orc_fluid_source(double Ftx, double Fty, double Fpx, double Fpy, double ux, double uy,
                      const double omega[9], double sig[9], double mhat[9], double dg[9])
{
    const double G00 = Fpx * ux + Fpy * uy;   /* Gamma^p_00, Sec. 3 */
    sig[0] = G00;
    sig[1] = CS2 * Ftx;
    sig[2] = CS2 * Fty;
    sig[3] = 2.0 * CS2 * (Ftx * ux + Fpx * ux) + CS2 * G00;
    sig[4] = 2.0 * CS2 * (Fty * uy + Fpy * uy) + CS2 * G00;
    sig[5] = CS2 * (Ftx * uy + Fty * ux) + CS2 * (Fpx * uy + Fpy * ux);
    sig[6] = 0.0;
    sig[7] = 0.0;
    sig[8] = 0.0;
    /* order of sig: 00,10,01,20,02,11,21,12,22 */
    const double s00 = sig[0], s10 = sig[1], s01 = sig[2], s20 = sig[3], s02 = sig[4];
    const double s11 = sig[5], s21 = sig[6], s12 = sig[7], s22 = sig[8];
    mhat[0] = (1.0 - 0.5 * omega[0]) * s00;
    mhat[1] = (1.0 - 0.5 * omega[1]) * s10;
    mhat[2] = (1.0 - 0.5 * omega[2]) * s01;
    mhat[3] = (1.0 - 0.5 * omega[3]) * (3.0 * (s20 + s02) - 4.0 * s00);
    mhat[4] = (1.0 - 0.5 * omega[4]) * (s20 - s02);
    mhat[5] = (1.0 - 0.5 * omega[5]) * s11;
    mhat[6] = (1.0 - 0.5 * omega[6]) * (-3.0 * s21 + 2.0 * s01);
    mhat[7] = (1.0 - 0.5 * omega[7]) * (-3.0 * s12 + 2.0 * s10);
    mhat[8] = (1.0 - 0.5 * omega[8]) * (9.0 * s22 - 6.0 * (s20 + s02) + 4.0 * s00);   /* R2 */
    const double m0 = mhat[0], m1 = mhat[1], m2 = mhat[2], m3 = mhat[3], m4 = mhat[4];
    const double m5 = mhat[5], m6 = mhat[6], m7 = mhat[7], m8 = mhat[8];
    dg[0] = (m0 - m3 + m8) / 9.0;
    dg[1] = (4.0 * m0 + 6.0 * m1 - m3 + 9.0 * m4 + 6.0 * m7 - 2.0 * m8) / 36.0;
    dg[2] = (4.0 * m0 + 6.0 * m2 - m3 - 9.0 * m4 + 6.0 * m6 - 2.0 * m8) / 36.0;
    dg[3] = (4.0 * m0 - 6.0 * m1 - m3 + 9.0 * m4 - 6.0 * m7 - 2.0 * m8) / 36.0;
    dg[4] = (4.0 * m0 - 6.0 * m2 - m3 - 9.0 * m4 - 6.0 * m6 - 2.0 * m8) / 36.0;
    dg[5] = (4.0 * m0 + 6.0 * m1 + 6.0 * m2 + 2.0 * m3 + 9.0 * m5 - 3.0 * m6 - 3.0 * m7 + m8) / 36.0;
    dg[6] = (4.0 * m0 - 6.0 * m1 + 6.0 * m2 + 2.0 * m3 - 9.0 * m5 - 3.0 * m6 + 3.0 * m7 + m8) / 36.0;
    dg[7] = (4.0 * m0 - 6.0 * m1 - 6.0 * m2 + 2.0 * m3 + 9.0 * m5 + 3.0 * m6 + 3.0 * m7 + m8) / 36.0;
    dg[8] = (4.0 * m0 + 6.0 * m1 - 6.0 * m2 + 2.0 * m3 - 9.0 * m5 + 3.0 * m6 - 3.0 * m7 + m8) / 36.0;
}

/* Fluid-lattice cascaded collision of Sec. 4: h-hat from Eq. cascadedcollisionoperator (eta-bar'
 * are the raw moments of the streamed g-bar; p and u are the corrected fields of Eq.
 * hydrodynamicfields), then the post-collision g-bar-tilde of Eq. postcollisioncascadedLBscheme
 * including delta g^s.  Optionally returns h-hat. */
void orc_fluid_collide(const double gb[9], double p, double ux, double uy, double rho,
                       double Ftx, double Fty, double Fpx, double Fpy, const double omega[9],
                       double gout[9], double hout[9])
{
    double e[9];
    raw_moments(gb, e);
    const double e20 = e[3], e02 = e[4], e11 = e[5], e21 = e[6], e12 = e[7], e22 = e[8];
    const double psi = p - rho * CS2;
    const double G00 = Fpx * ux + Fpy * uy;
    const double ux2 = ux * ux, uy2 = uy * uy;
    double h[9];
    h[0] = 0.5 * omega[0] * G00 / 9.0;
    h[1] = 0.5 * omega[1] * CS2 * Ftx / 6.0;
    h[2] = 0.5 * omega[2] * CS2 * Fty / 6.0;
    h[3] = omega[3] / 12.0 * (2.0 * p * CS2 + rho * CS2 * (ux2 + uy2) - (e20 + e02));
    h[4] = omega[4] / 4.0 * (rho * CS2 * (ux2 - uy2) - (e20 - e02));
    h[5] = omega[5] / 4.0 * (rho * CS2 * ux * uy - e11);
    h[6] = omega[6] / 4.0 * (psi * (CS2 + ux2) * uy + e21 - uy * e20 - 2.0 * ux * e11
                             + 3.0 * CS2 * rho * ux2 * uy - ux2 * uy * p)
           - uy * (1.5 * h[3] + 0.5 * h[4]) - 2.0 * ux * h[5];
    h[7] = omega[7] / 4.0 * (psi * (CS2 + uy2) * ux + e12 - 2.0 * uy * e11 - ux * e02
                             + 3.0 * CS2 * rho * ux * uy2 - ux * uy2 * p)
           - ux * (1.5 * h[3] - 0.5 * h[4]) - 2.0 * uy * h[5];
    h[8] = omega[8] / 4.0 * (CS2 * CS2 * CS2 * rho + psi * (CS2 + ux2) * (CS2 + uy2) - e22
                             + 2.0 * (uy * e21 + ux * e12) - (uy2 * e20 + ux2 * e02)
                             - 4.0 * ux * uy * e11 + 4.0 * CS2 * rho * ux2 * uy2 - ux2 * uy2 * p)
           - 2.0 * h[3] - 0.5 * uy2 * (3.0 * h[3] + h[4]) - 0.5 * ux2 * (3.0 * h[3] - h[4])
           - 4.0 * ux * uy * h[5] - 2.0 * uy * h[6] - 2.0 * ux * h[7];

    double sig[9], mh[9], dg[9];
    orc_fluid_source(Ftx, Fty, Fpx, Fpy, ux, uy, omega, sig, mh, dg);

    gout[0] = gb[0] + (h[0] - 4.0 * (h[3] - h[8])) + dg[0];
    gout[1] = gb[1] + (h[0] + h[1] - h[3] + h[4] + 2.0 * (h[7] - h[8])) + dg[1];
    gout[2] = gb[2] + (h[0] + h[2] - h[3] - h[4] + 2.0 * (h[6] - h[8])) + dg[2];
    gout[3] = gb[3] + (h[0] - h[1] - h[3] + h[4] - 2.0 * (h[7] + h[8])) + dg[3];
    gout[4] = gb[4] + (h[0] - h[2] - h[3] - h[4] - 2.0 * (h[6] + h[8])) + dg[4];
    gout[5] = gb[5] + (h[0] + h[1] + h[2] + 2.0 * h[3] + h[5] - h[6] - h[7] + h[8]) + dg[5];
    gout[6] = gb[6] + (h[0] - h[1] + h[2] + 2.0 * h[3] - h[5] - h[6] + h[7] + h[8]) + dg[6];
    gout[7] = gb[7] + (h[0] - h[1] - h[2] + 2.0 * h[3] + h[5] + h[6] + h[7] + h[8]) + dg[7];
    gout[8] = gb[8] + (h[0] + h[1] - h[2] + 2.0 * h[3] - h[5] + h[6] - h[7] + h[8]) + dg[8];
    if (hout) for (int k = 0; k < 9; ++k) hout[k] = h[k];
}

/* Interface-lattice cascaded collision of Sec. 5: g-hat_0..g-hat_8 (with reading R3) and
 * f-tilde.  jx, jy = M_phi theta n_x, M_phi theta n_y; omega: the nine interface rates. */
void orc_ace_collide(const double f[9], double ux, double uy, double jx, double jy,
                     const double omega[9], double fout[9], double gout_hat[9])
{
    double k[9];
    raw_moments(f, k);
    const double phi = k[0];
    const double k10 = k[1], k01 = k[2], k20 = k[3], k02 = k[4], k11 = k[5];
    const double k21 = k[6], k12 = k[7], k22 = k[8];
    const double ux2 = ux * ux, uy2 = uy * uy;
    double g[9];
    g[0] = 0.0;
    g[1] = omega[1] / 6.0 * (phi * ux + jx - k10);
    g[2] = omega[2] / 6.0 * (phi * uy + jy - k01);
    g[3] = omega[3] / 12.0 * (2.0 * CS2 * phi - (ux2 + uy2) * phi - (k20 + k02)
                              + 2.0 * (ux * k10 + uy * k01)) + ux * g[1] + uy * g[2];
    g[4] = omega[4] / 4.0 * (-(ux2 - uy2) * phi - (k20 - k02) + 2.0 * (ux * k10 - uy * k01))
           + 3.0 * (ux * g[1] - uy * g[2]);
    g[5] = omega[5] / 4.0 * (-ux * uy * phi - k11 + (ux * k01 + uy * k10))
           + 1.5 * (ux * g[2] + uy * g[1]);
    g[6] = omega[6] / 4.0 * (-ux2 * uy * phi + k21 - uy * k20 - 2.0 * ux * k11
                             + 2.0 * ux * uy * k10 + ux2 * k01)
           + 3.0 * ux * uy * g[1] + (1.5 * ux2 + 1.0) * g[2] - 1.5 * uy * g[3] - 0.5 * uy * g[4]
           - 2.0 * ux * g[5];
    g[7] = omega[7] / 4.0 * (-ux * uy2 * phi + k12 - ux * k02 - 2.0 * uy * k11
                             + 2.0 * ux * uy * k01 + uy2 * k10)
           + (1.5 * uy2 + 1.0) * g[1] + 3.0 * ux * uy * g[2] - 1.5 * ux * g[3] /* R3 */
           + 0.5 * ux * g[4] - 2.0 * uy * g[5];
    g[8] = omega[8] / 4.0 * (CS2 * CS2 * phi - k22 + 2.0 * (ux * k12 + uy * k21)
                             - (uy2 * k20 + ux2 * k02) - 4.0 * ux * uy * k11
                             + 2.0 * (ux * uy2 * k10 + ux2 * uy * k01) - ux2 * uy2 * phi)
           + (2.0 * ux + 3.0 * ux * uy2) * g[1] + (2.0 * uy + 3.0 * ux2 * uy) * g[2]
           - (2.0 + 1.5 * (ux2 + uy2)) * g[3] + 0.5 * (ux2 - uy2) * g[4] - 4.0 * ux * uy * g[5]
           - 2.0 * uy * g[6] - 2.0 * ux * g[7];

    fout[0] = f[0] + (g[0] - 4.0 * (g[3] - g[8]));
    fout[1] = f[1] + (g[0] + g[1] - g[3] + g[4] + 2.0 * (g[7] - g[8]));
    fout[2] = f[2] + (g[0] + g[2] - g[3] - g[4] + 2.0 * (g[6] - g[8]));
    fout[3] = f[3] + (g[0] - g[1] - g[3] + g[4] - 2.0 * (g[7] + g[8]));
    fout[4] = f[4] + (g[0] - g[2] - g[3] - g[4] - 2.0 * (g[6] + g[8]));
    fout[5] = f[5] + (g[0] + g[1] + g[2] + 2.0 * g[3] + g[5] - g[6] - g[7] + g[8]);
    fout[6] = f[6] + (g[0] - g[1] + g[2] + 2.0 * g[3] - g[5] - g[6] + g[7] + g[8]);
    fout[7] = f[7] + (g[0] - g[1] - g[2] + 2.0 * g[3] + g[5] + g[6] + g[7] + g[8]);
    fout[8] = f[8] + (g[0] + g[1] - g[2] + 2.0 * g[3] - g[5] + g[6] - g[7] + g[8]);
    if (gout_hat) for (int q = 0; q < 9; ++q) gout_hat[q] = g[q];
}

/* ---------------------------------------------------------------------------------------------
 * Lattice helpers
 * ------------------------------------------------------------------------------------------- */

static inline int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }

/* Index of a column / row just outside the grid: periodic wrap, or at a wall (either kind) the
 * mirror ghost of R8 / R14, i.e. the first or last node. */
static int ghost_col(const orc_case* c, int xx)
{
    if (xx >= 0 && xx < c->nx) return xx;
    if (xx < 0) return c->bc_x0 == BC_PERIODIC ? wrap(xx, c->nx) : 0;
    return c->bc_x1 == BC_PERIODIC ? wrap(xx, c->nx) : c->nx - 1;
}

static int ghost_row(const orc_case* c, int yy)
{
    if (yy >= 0 && yy < c->ny) return yy;
    if (yy < 0) return c->bc_y0 == BC_PERIODIC ? wrap(yy, c->ny) : 0;
    return c->bc_y1 == BC_PERIODIC ? wrap(yy, c->ny) : c->ny - 1;
}

/* R17: the imposed single-vortex shear flow of Sec. 6.1 at node (x, y) and time level t,
 *   u_x = -U_0 pi cos(pi (x/L0 - 1/2)) sin(pi (y/L0 - 1/2)),
 *   u_y =  U_0 pi sin(pi (x/L0 - 1/2)) cos(pi (y/L0 - 1/2)),
 * with L0 = nx along x and ny along y, and the sign reversed for t >= reverse_step. */
#define ORC_PI 3.14159265358979323846
static void imposed_velocity(const orc_case* c, int x, int y, int t, double* ux, double* uy)
{
    const double s = (c->reverse_step > 0 && t >= c->reverse_step) ? -1.0 : 1.0;
    const double ax = ORC_PI * ((double)x / c->nx - 0.5);
    const double ay = ORC_PI * ((double)y / c->ny - 0.5);
    *ux = -s * c->u0 * ORC_PI * cos(ax) * sin(ay);
    *uy = s * c->u0 * ORC_PI * sin(ax) * cos(ay);
}

/* Nodal field value at (x+dx, y+dy). */
static double field_at(const orc_case* c, const double* a, int x, int y, int dx, int dy)
{
    return a[(size_t)ghost_row(c, y + dy) * c->nx + ghost_col(c, x + dx)];
}

/* Second-order isotropic finite differences on the D2Q9 stencil (Sec. 4, closing remark):
 *   grad a = (1/c_s^2) sum_alpha w_alpha e_alpha a(x + e_alpha),
 *   lap a  = (2/c_s^2) sum_alpha w_alpha (a(x + e_alpha) - a(x)),
 * and the Hessian (R5): d_xx a = [second x-difference of the row below + 10 x that of the own
 * row + that of the row above] / 12, d_yy transposed, d_xy the central cross difference.  Its
 * trace equals lap a. */
static const double W9[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static void stencil(const orc_case* c, const double* a, int x, int y, double* gx, double* gy,
                    double* lap, double* hxx, double* hyy, double* hxy)
{
    double sx = 0.0, sy = 0.0, sl = 0.0;
    const double ac = field_at(c, a, x, y, 0, 0);
    for (int q = 1; q < 9; ++q) {
        const double v = field_at(c, a, x, y, EX[q], EY[q]);
        sx += W9[q] * EX[q] * v;
        sy += W9[q] * EY[q] * v;
        sl += W9[q] * (v - ac);
    }
    *gx = sx / CS2;
    *gy = sy / CS2;
    if (lap) *lap = 2.0 * sl / CS2;
    if (hxx) {
        double s = 0.0;
        for (int j = -1; j <= 1; ++j) {
            const double wj = (j == 0) ? 10.0 : 1.0;
            s += wj * (field_at(c, a, x, y, 1, j) - 2.0 * field_at(c, a, x, y, 0, j)
                       + field_at(c, a, x, y, -1, j));
        }
        *hxx = s / 12.0;
    }
    if (hyy) {
        double s = 0.0;
        for (int i = -1; i <= 1; ++i) {
            const double wi = (i == 0) ? 10.0 : 1.0;
            s += wi * (field_at(c, a, x, y, i, 1) - 2.0 * field_at(c, a, x, y, i, 0)
                       + field_at(c, a, x, y, i, -1));
        }
        *hyy = s / 12.0;
    }
    if (hxy) {
        *hxy = (field_at(c, a, x, y, 1, 1) - field_at(c, a, x, y, -1, 1)
                - field_at(c, a, x, y, 1, -1) + field_at(c, a, x, y, -1, -1)) / 4.0;
    }
}

/* Whole-field stencils, exposed for the tests (exactness on quadratics). */
void orc_stencils(const orc_case* c, const double* a, double* gx, double* gy, double* lap,
                  double* hxx, double* hyy, double* hxy)
{
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            const size_t n = (size_t)y * c->nx + x;
            stencil(c, a, x, y, &gx[n], &gy[n], &lap[n], &hxx[n], &hyy[n], &hxy[n]);
        }
}

/* Fluid relaxation rate of the second-order shear moments from the local viscosity,
 * Sec. 4 Eq. fluidviscosity: mu = rho c_s^2 (1/omega - 1/2). */
static double omega_from_nu(double nu) { return 1.0 / (nu / CS2 + 0.5); }

/* All macroscopic quantities at node (x, y) from phi = sum f, p* = sum g-bar (whole fields) and
 * the node's streamed g-bar: properties (R1), stencils, normal, theta (Sec. 2 Eq.
 * thetavariable), forces (R4-R7, R11, Sec. 6.7 Marangoni components) and the corrected p, u of
 * Sec. 4 Eq. hydrodynamicfields. */
static void node_macros(const orc_case* c, const double* phi, const double* pst,
                        const double gb[9], int x, int y, orc_node* o)
{
    const size_t n = (size_t)y * c->nx + x;
    const double ph = phi[n];
    o->phi = ph;
    o->rho = c->rho_b + ph * (c->rho_a - c->rho_b);
    o->mu = c->mu_b + ph * (c->mu_a - c->mu_b);
    o->omega_nu = omega_from_nu(o->mu / o->rho);
    o->pstar = pst[n];

    stencil(c, phi, x, y, &o->dphix, &o->dphiy, &o->lap, &o->hxx, &o->hyy, &o->hxy);
    stencil(c, pst, x, y, &o->dpx, &o->dpy, NULL, NULL, NULL, NULL);

    const double g2 = o->dphix * o->dphix + o->dphiy * o->dphiy;
    o->theta = 4.0 * ph * (1.0 - ph) / c->width;
    {   /* R6: regularised normal */
        const double gm = sqrt(g2);
        o->nx = o->dphix / (gm + NORMAL_EPS);
        o->ny = o->dphiy / (gm + NORMAL_EPS);
        const double nHn = o->nx * o->nx * o->hxx + 2.0 * o->nx * o->ny * o->hxy
                           + o->ny * o->ny * o->hyy;
        double kt, dktx, dkty;   /* kappa-tilde = (3/2) sigma W (R4) and its gradient */
        if (c->sigma_model == 1) {
            /* R16: Langmuir isotherm sigma = sigma0 [1 + beta ln(1 - psi)], psi imposed */
            const double psi = c->psi0 + c->gradpsi_x * x + c->gradpsi_y * y;
            const double sigma = c->sigma0 * (1.0 + c->beta * log(1.0 - psi));
            const double dsigma_dpsi = -c->sigma0 * c->beta / (1.0 - psi);
            kt = 1.5 * sigma * c->width;
            dktx = 1.5 * c->width * dsigma_dpsi * c->gradpsi_x;
            dkty = 1.5 * c->width * dsigma_dpsi * c->gradpsi_y;
        } else {
            const double T = c->T0 + c->gradT_x * x + c->gradT_y * y;
            const double sigma = c->sigma0 + c->dsigma_dT * (T - c->T0);
            kt = 1.5 * sigma * c->width;
            dktx = 1.5 * c->width * c->dsigma_dT * c->gradT_x;
            dkty = 1.5 * c->width * c->dsigma_dT * c->gradT_y;
        }
        const double curv = gm * (o->lap - nHn);                       /* |grad phi|^2 div n */
        o->Fsx = -kt * curv * o->nx
                 + g2 * ((1.0 - o->nx * o->nx) * dktx - o->nx * o->ny * dkty);
        o->Fsy = -kt * curv * o->ny
                 + g2 * ((1.0 - o->ny * o->ny) * dkty - o->nx * o->ny * dktx);
    }
    o->Ftx = o->Fsx + (o->rho - c->rho_ref) * c->gx;
    o->Fty = o->Fsy + (o->rho - c->rho_ref) * c->gy;
    o->Fpx = -o->dpx + CS2 * (c->rho_a - c->rho_b) * o->dphix;          /* R7 */
    o->Fpy = -o->dpy + CS2 * (c->rho_a - c->rho_b) * o->dphiy;

    double jx = 0.0, jy = 0.0;
    for (int q = 0; q < 9; ++q) { jx += gb[q] * EX[q]; jy += gb[q] * EY[q]; }
    o->ux = (jx + 0.5 * CS2 * o->Ftx) / (o->rho * CS2);
    o->uy = (jy + 0.5 * CS2 * o->Fty) / (o->rho * CS2);
    o->p = o->pstar + 0.5 * (o->Fpx * o->ux + o->Fpy * o->uy);
}

/* phi = sum_alpha f_alpha (Sec. 5) and p* = sum_alpha g-bar_alpha (Sec. 4) at every node of
 * rows y0-1 .. y1 (wrapped or clamped to the grid), i.e. every row the stencils of rows
 * [y0, y1) read. */
static void zeroth_moments_rows(const orc_case* c, const double* g, const double* f, double* phi,
                                double* pst, int y0, int y1)
{
    const size_t N = (size_t)c->nx * c->ny;
    int lo = y0 - 1, hi = y1;
    if (hi - lo + 1 >= c->ny) { lo = 0; hi = c->ny - 1; }
    for (int yr = lo; yr <= hi; ++yr) {
        const int y = ghost_row(c, yr);
        for (int x = 0; x < c->nx; ++x) {
            const size_t n = (size_t)y * c->nx + x;
            double sp = 0.0, sg = 0.0;
            for (int q = 0; q < 9; ++q) { sp += f[q * N + n]; sg += g[q * N + n]; }
            phi[n] = sp;
            pst[n] = sg;
        }
    }
}

static void zeroth_moments(const orc_case* c, const double* g, const double* f, double* phi,
                           double* pst)
{
    zeroth_moments_rows(c, g, f, phi, pst, 0, c->ny);
}

/* ---------------------------------------------------------------------------------------------
 * Public entry points
 * ------------------------------------------------------------------------------------------- */

/* Equilibrium initialisation (R10) from nodal phi, p, ux, uy (row-major [ny][nx]). */
void orc_init(const orc_case* c, const double* phi, const double* p, const double* ux,
              const double* uy, double* g, double* f)
{
    const size_t N = (size_t)c->nx * c->ny;
    for (size_t n = 0; n < N; ++n) {
        const double rho = c->rho_b + phi[n] * (c->rho_a - c->rho_b);
        double gq[9], fq[9];
        orc_geq(p[n], ux[n], uy[n], rho, gq);
        orc_feq(phi[n], ux[n], uy[n], 0.0, 0.0, fq);
        for (int q = 0; q < 9; ++q) { g[q * N + n] = gq[q]; f[q * N + n] = fq[q]; }
    }
}

/* Macroscopic fields of a state (g-bar, f): phi, corrected p, u, rho; any output may be NULL. */
void orc_fields(const orc_case* c, const double* g, const double* f, double* phi_out,
                double* p_out, double* ux_out, double* uy_out, double* rho_out)
{
    const size_t N = (size_t)c->nx * c->ny;
    double* phi = (double*)malloc(N * sizeof(double));
    double* pst = (double*)malloc(N * sizeof(double));
    zeroth_moments(c, g, f, phi, pst);
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            const size_t n = (size_t)y * c->nx + x;
            double gb[9];
            for (int q = 0; q < 9; ++q) gb[q] = g[q * N + n];
            orc_node o;
            node_macros(c, phi, pst, gb, x, y, &o);
            if (c->flow == 1) {   /* R17: u imposed, no pressure field */
                imposed_velocity(c, x, y, c->t, &o.ux, &o.uy);
                o.p = 0.0;
            }
            if (phi_out) phi_out[n] = o.phi;
            if (p_out) p_out[n] = o.p;
            if (ux_out) ux_out[n] = o.ux;
            if (uy_out) uy_out[n] = o.uy;
            if (rho_out) rho_out[n] = o.rho;
        }
    free(phi);
    free(pst);
}

/* Per-node macroscopic record (tests): node (x, y) of a state. */
void orc_node_info(const orc_case* c, const double* g, const double* f, int x, int y,
                   orc_node* out)
{
    const size_t N = (size_t)c->nx * c->ny;
    double* phi = (double*)malloc(N * sizeof(double));
    double* pst = (double*)malloc(N * sizeof(double));
    zeroth_moments(c, g, f, phi, pst);
    const size_t n = (size_t)y * c->nx + x;
    double gb[9];
    for (int q = 0; q < 9; ++q) gb[q] = g[q * N + n];
    node_macros(c, phi, pst, gb, x, y, out);
    free(phi);
    free(pst);
}

/* Destination of the population leaving (x, y) along alpha: the neighbour x + e_alpha (periodic
 * wrap).  Where that crosses a no-slip wall, the same node in the opposite direction (half-way
 * bounce-back, R8); where it crosses only free-slip walls, the normal components crossing them
 * are reversed and the population stays on that side of the wall (specular reflection, R14).
 * Returns the flat index into the 9-plane field. */
static int direction_of(int ex, int ey)
{
    for (int q = 0; q < 9; ++q)
        if (EX[q] == ex && EY[q] == ey) return q;
    return -1;
}

static size_t stream_target(const orc_case* c, int q, int x, int y)
{
    static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    const size_t N = (size_t)c->nx * c->ny;
    int ex = EX[q], ey = EY[q];
    int xx = x + ex, yy = y + ey;
    int cross_x = 0, cross_y = 0, noslip = 0;
    if (xx < 0 || xx >= c->nx) {
        const int kind = xx < 0 ? c->bc_x0 : c->bc_x1;
        if (kind == BC_PERIODIC) xx = wrap(xx, c->nx);
        else { cross_x = 1; noslip |= kind == BC_NOSLIP; }
    }
    if (yy < 0 || yy >= c->ny) {
        const int kind = yy < 0 ? c->bc_y0 : c->bc_y1;
        if (kind == BC_PERIODIC) yy = wrap(yy, c->ny);
        else { cross_y = 1; noslip |= kind == BC_NOSLIP; }
    }
    if (noslip) return (size_t)OPP[q] * N + (size_t)y * c->nx + x;
    if (cross_x) { ex = -ex; xx = x; }
    if (cross_y) { ey = -ey; yy = y; }
    return (size_t)direction_of(ex, ey) * N + (size_t)yy * c->nx + xx;
}

/* Rows [y0, y1) of one time step: collide both lattices at every node of those rows (Secs. 4
 * and 5) and stream the post-collision populations, g-bar(x + e, t + 1) = g-bar-tilde(x, t) and
 * f likewise.  Restricting the rows serves only to time a bounded sample of a large grid.
 * Relaxation rates: R9 (cascaded) or all equal (R15).  With the imposed flow (R17) only the
 * interface lattice collides and streams; the fluid populations are copied unchanged. */
void orc_step_rows(const orc_case* c, const double* g, const double* f, double* g_new,
                   double* f_new, int y0, int y1)
{
    const size_t N = (size_t)c->nx * c->ny;
    double* phi = (double*)malloc(N * sizeof(double));
    double* pst = (double*)malloc(N * sizeof(double));
    zeroth_moments_rows(c, g, f, phi, pst, y0, y1);

    const int srt = c->collision == 1;
    const double omega_phi = 1.0 / (c->mobility / CS2 + 0.5);   /* Sec. 5: M_phi relation */
    const double o3 = srt ? omega_phi : 1.0;
    const double om_f[9] = {o3, omega_phi, omega_phi, o3, o3, o3, o3, o3, o3};

#pragma omp parallel for schedule(static)
    for (int y = y0; y < y1; ++y) {
        for (int x = 0; x < c->nx; ++x) {
            const size_t n = (size_t)y * c->nx + x;
            double gb[9], fq[9], go[9], fo[9];
            for (int q = 0; q < 9; ++q) { gb[q] = g[q * N + n]; fq[q] = f[q * N + n]; }
            if (c->flow == 1) {
                double dphx, dphy, ux, uy;
                stencil(c, phi, x, y, &dphx, &dphy, NULL, NULL, NULL, NULL);
                const double gm = sqrt(dphx * dphx + dphy * dphy);
                const double theta = 4.0 * phi[n] * (1.0 - phi[n]) / c->width;
                imposed_velocity(c, x, y, c->t, &ux, &uy);
                const double nx = dphx / (gm + NORMAL_EPS), ny = dphy / (gm + NORMAL_EPS);
                orc_ace_collide(fq, ux, uy, c->mobility * theta * nx, c->mobility * theta * ny,
                                om_f, fo, NULL);
                for (int q = 0; q < 9; ++q) {
                    f_new[stream_target(c, q, x, y)] = fo[q];
                    g_new[q * N + n] = gb[q];
                }
                continue;
            }
            orc_node o;
            node_macros(c, phi, pst, gb, x, y, &o);
            const double w = o.omega_nu, r = srt ? w : 1.0;
            const double om_g[9] = {r, r, r, r, w, w, r, r, r};
            orc_fluid_collide(gb, o.p, o.ux, o.uy, o.rho, o.Ftx, o.Fty, o.Fpx, o.Fpy, om_g, go,
                              NULL);
            const double jx = c->mobility * o.theta * o.nx;
            const double jy = c->mobility * o.theta * o.ny;
            orc_ace_collide(fq, o.ux, o.uy, jx, jy, om_f, fo, NULL);
            for (int q = 0; q < 9; ++q) {
                const size_t t = stream_target(c, q, x, y);
                g_new[t] = go[q];
                f_new[t] = fo[q];
            }
        }
    }
    free(phi);
    free(pst);
}

/* One time step over the whole grid.  g, f: current state (streamed populations); g_new, f_new:
 * next state (must not alias). */
void orc_step(const orc_case* c, const double* g, const double* f, double* g_new, double* f_new)
{
    orc_step_rows(c, g, f, g_new, f_new, 0, c->ny);
}

/* nsteps time steps in place on (g, f), using caller-provided scratch of the same size. */
void orc_run(const orc_case* c, double* g, double* f, double* g_tmp, double* f_tmp, int nsteps)
{
    const size_t bytes = (size_t)9 * c->nx * c->ny * sizeof(double);
    orc_case cs = *c;
    for (int s = 0; s < nsteps; ++s) {
        cs.t = c->t + s;
        orc_step(&cs, g, f, g_tmp, f_tmp);
        memcpy(g, g_tmp, bytes);
        memcpy(f, f_tmp, bytes);
    }
}

/* Round every population to the nearest IEEE binary32 value (round to nearest even). */
static void round_to_float(double* a, size_t n)
{
    for (size_t i = 0; i < n; ++i) a[i] = (double)(float)a[i];
}

/* As orc_run, with the state rounded to binary32 on entry and after every step: what storing the
 * populations in FP32 between steps does on its own, every operation of a step staying in FP64.
 * (Not a reading of the paper: it separates storage rounding from arithmetic rounding when the
 * tests weigh an FP32 implementation against this FP64 one.) */
void orc_run_float_storage(const orc_case* c, double* g, double* f, double* g_tmp,
                           double* f_tmp, int nsteps)
{
    const size_t n = (size_t)9 * c->nx * c->ny;
    round_to_float(g, n);
    round_to_float(f, n);
    orc_case cs = *c;
    for (int s = 0; s < nsteps; ++s) {
        cs.t = c->t + s;
        orc_step(&cs, g, f, g_tmp, f_tmp);
        memcpy(g, g_tmp, n * sizeof(double));
        memcpy(f, f_tmp, n * sizeof(double));
        round_to_float(g, n);
        round_to_float(f, n);
    }
}

void orc_set_normal_eps(double eps) { NORMAL_EPS = eps; }
double orc_get_normal_eps(void) { return NORMAL_EPS; }

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
