// Device-side arithmetic of the coupled cascaded central-moment LB step (arXiv:1909.04166) for
// sm_103a: per-case constants, storage conversion, the per-node update (forces, macroscopic
// fields, fluid and interface cascaded collisions) and the equilibrium initialisation.
//
// Conventions (shared with the C ABI in include/cmlbm.h):
//   D2Q9 ordering of Sec. 4 Eq. particlevelocities: e_x = (0,1,0,-1,0,1,-1,-1,1),
//   e_y = (0,0,1,0,-1,1,1,-1,-1).  A state holds 18 populations per node (9 fluid g-bar, then 9
//   interface f) in tiles of 32 columns: element (a, x, y) sits at
//   ((y * nstrips + x / 32) * 18 + a) * 32 + x % 32.  The state holds the streamed
//   (pre-collision) populations of the current time level.
//   c_s^2 = c_sphi^2 = 1/3 (Sec. 5).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace cmlbm {

// Per-case constants in the compute precision R.  Derived on the host from lbm_params.
template <typename R>
struct Consts {
    R rho_b, drho;       // rho = rho_b + phi drho                      (Sec. 2, linear interpolation)
    R mu_b, dmu;         // mu  = mu_b  + phi dmu
    R kt0, dktx, dkty;   // kappa-tilde(x, y) = kt0 + dktx x + dkty y   (kappa-tilde = 3/2 sigma W)
    R mob;               // M_phi
    R four_over_w;       // theta = (4/W) phi (1 - phi)                 (Sec. 2 Eq. thetavariable)
    R omega_phi_6;       // omega^phi_{1,2} / 6, from M_phi = c^2 (1/omega - 1/2)   (Sec. 5)
    R gx, gy, rho_ref;   // F_ext = (rho - rho_ref) g
    R cs2_drho;          // c_s^2 (rho_A - rho_B), the factor of grad rho in F_p
};

struct Geometry {
    int nx, ny;
    int nstrips;         // ceil(nx / 32): tiles of 32 columns per row
    int wall_x, wall_y;
};

// ---------------------------------------------------------------------------------------------
// Nine-point stencil window of a nodal field: value at (x + i, y + j), i, j in {-1, 0, 1}.
// ---------------------------------------------------------------------------------------------
template <typename R>
struct Win {
    R sw, s, se, w, c, e, nw, n, ne;
};

// Second-order isotropic differences on the D2Q9 neighbourhood (Sec. 4, closing remark):
// grad a = 3 sum_a w_a e_a a(x + e_a) and lap a = 6 sum_a w_a (a(x + e_a) - a(x)), with
// w = 1/9 (axis) and 1/36 (diagonal).  The Hessian is the 1-10-1 weighted second difference
// across the three rows (columns) of the window; its trace equals the Laplacian.
template <typename R>
__device__ __forceinline__ void grad_iso(const Win<R>& a, R& gx, R& gy)
{
    const R third = R(1) / R(3), twelfth = R(1) / R(12);
    gx = (a.e - a.w) * third + ((a.ne + a.se) - (a.nw + a.sw)) * twelfth;
    gy = (a.n - a.s) * third + ((a.ne + a.nw) - (a.se + a.sw)) * twelfth;
}

template <typename R>
__device__ __forceinline__ void lap_hess(const Win<R>& a, R& lap, R& hxx, R& hyy, R& hxy)
{
    const R sixth = R(1) / R(6), twelfth = R(1) / R(12);
    const R axis = (a.e + a.w) + (a.n + a.s);
    const R diag = (a.ne + a.nw) + (a.se + a.sw);
    lap = (R(4) * axis + diag - R(20) * a.c) * sixth;
    const R dxx_mid = a.e - R(2) * a.c + a.w;
    const R dyy_mid = a.n - R(2) * a.c + a.s;
    const R dxx_side = (a.ne - R(2) * a.n + a.nw) + (a.se - R(2) * a.s + a.sw);
    const R dyy_side = (a.ne - R(2) * a.e + a.se) + (a.nw - R(2) * a.w + a.sw);
    hxx = (R(10) * dxx_mid + dxx_side) * twelfth;
    hyy = (R(10) * dyy_mid + dyy_side) * twelfth;
    hxy = ((a.ne - a.nw) - (a.se - a.sw)) * R(0.25);
}

template <typename R> __device__ __forceinline__ R rcp_(R v) { return R(1) / v; }
template <> __device__ __forceinline__ float rcp_<float>(float v) { return __fdividef(1.0f, v); }
template <typename R> __device__ __forceinline__ R rsqrt_(R v) { return R(1) / sqrt(v); }
template <> __device__ __forceinline__ float rsqrt_<float>(float v) { return rsqrtf(v); }

// Macroscopic quantities of one node that the collisions need.
template <typename R>
struct Macro {
    R rho, omega;          // density, shear relaxation rate omega_4 = omega_5
    R ux, uy, p;           // corrected velocity and pressure (Sec. 4 Eq. hydrodynamicfields)
    R Ftx, Fty, Fpx, Fpy;  // total force and net gradient pressure force
    R jx, jy;              // M_phi theta n, the interface first-order equilibrium moment
};

// Forces and corrected fields of one node, from the phi and p* windows and the streamed g-bar
// first moments (Sec. 2 properties and surface tension, Sec. 6.7 Marangoni components, Sec. 3
// net gradient pressure force, Sec. 4 Eqs. hydrodynamicfields and fluidviscosity).
template <typename R>
__device__ __forceinline__ void node_macro(const Win<R>& ph, const Win<R>& ps, R jgx, R jgy,
                                           R xf, R yf, const Consts<R>& K, Macro<R>& m)
{
    const R phi = ph.c;
    m.rho = K.rho_b + phi * K.drho;
    const R mu = K.mu_b + phi * K.dmu;
    const R inv_rho = rcp_(m.rho);
    // omega = 1 / (nu / c_s^2 + 1/2), nu = mu / rho
    m.omega = rcp_(R(3) * mu * inv_rho + R(0.5));

    R dphx, dphy, lap, hxx, hyy, hxy, dpx, dpy;
    grad_iso(ph, dphx, dphy);
    lap_hess(ph, lap, hxx, hyy, hxy);
    grad_iso(ps, dpx, dpy);

    // where |grad phi|^2 <= 1e-24 the normal and the surface force are zero (branch-free)
    const R g2 = dphx * dphx + dphy * dphy;
    const bool has_n = g2 > R(1e-24);
    const R ig = has_n ? rsqrt_(g2) : R(0);
    const R g2m = has_n ? g2 : R(0);
    const R gm = g2m * ig;
    const R nx = dphx * ig, ny = dphy * ig;
    const R nHn = nx * nx * hxx + R(2) * nx * ny * hxy + ny * ny * hyy;
    const R kt = K.kt0 + K.dktx * xf + K.dkty * yf;
    const R cap = -kt * gm * (lap - nHn);          // -kappa-tilde |grad phi|^2 div n
    const R nd = nx * K.dktx + ny * K.dkty;         // n . grad kappa-tilde
    const R Fsx = cap * nx + g2m * (K.dktx - nx * nd);   // + |grad phi|^2 (I - n n) grad kappa-tilde
    const R Fsy = cap * ny + g2m * (K.dkty - ny * nd);
    const R dr = m.rho - K.rho_ref;
    m.Ftx = Fsx + dr * K.gx;
    m.Fty = Fsy + dr * K.gy;
    m.Fpx = K.cs2_drho * dphx - dpx;
    m.Fpy = K.cs2_drho * dphy - dpy;
    // rho c_s^2 u = sum g-bar e + c_s^2 F_t / 2
    m.ux = R(3) * inv_rho * (jgx + m.Ftx * R(1.0 / 6.0));
    m.uy = R(3) * inv_rho * (jgy + m.Fty * R(1.0 / 6.0));
    m.p = ps.c + R(0.5) * (m.Fpx * m.ux + m.Fpy * m.uy);
    const R theta_m = K.mob * K.four_over_w * phi * (R(1) - phi);
    m.jx = theta_m * nx;
    m.jy = theta_m * ny;
}

// Apply the moment-change vector c (coefficients of the orthogonal basis K_0..K_8 of Sec. 4
// Eq. orthogonalbasisvectors) to nine populations: q_a += sum_j K_j(a) c_j.
template <typename R>
__device__ __forceinline__ void apply_basis(R q[9], const R c[9])
{
    const R A = c[0] - c[3] - R(2) * c[8];
    const R B = c[0] + R(2) * c[3] + c[8];
    const R s1 = c[1] - c[7], s2 = c[2] - c[6];
    q[0] += c[0] - R(4) * c[3] + R(4) * c[8];
    q[1] += A + c[1] + c[4] + R(2) * c[7];
    q[3] += A - c[1] + c[4] - R(2) * c[7];
    q[2] += A + c[2] - c[4] + R(2) * c[6];
    q[4] += A - c[2] - c[4] - R(2) * c[6];
    q[5] += B + s1 + s2 + c[5];
    q[6] += B - s1 + s2 - c[5];
    q[7] += B - s1 - s2 + c[5];
    q[8] += B + s1 - s2 - c[5];
}

// Fluid-lattice collision (Sec. 4): h-hat of Eq. cascadedcollisionoperator plus the cumulative
// source delta g^s = K^-1 (I - Lambda/2) K S, combined into one moment-change vector.  All
// fluid relaxation rates are 1 except omega_4 = omega_5 = m.omega.
template <typename R>
__device__ __forceinline__ void collide_fluid(R g[9], const Macro<R>& m)
{
    const R third = R(1) / R(3);
    const R ux = m.ux, uy = m.uy, p = m.p, rho = m.rho, om = m.omega;
    const R ux2 = ux * ux, uy2 = uy * uy;
    // raw moments of the streamed g-bar
    const R d = (g[5] + g[6]) + (g[7] + g[8]);   // eta'_22
    const R e20 = g[1] + g[3] + d;
    const R e02 = g[2] + g[4] + d;
    const R e11 = (g[5] - g[6]) + (g[7] - g[8]);
    const R e21 = (g[5] + g[6]) - (g[7] + g[8]);
    const R e12 = (g[5] - g[6]) - (g[7] - g[8]);
    const R e22 = d;
    const R psi = p - rho * third;
    const R rc2 = rho * third;

    // source raw moments sigma' (Gamma^t, Gamma^p matched, second order and above of the
    // cumulative source truncated as in Sec. 4)
    const R G00 = m.Fpx * ux + m.Fpy * uy;
    const R s10 = m.Ftx * third, s01 = m.Fty * third;
    const R s20 = R(2) * third * (m.Ftx + m.Fpx) * ux + third * G00;
    const R s02 = R(2) * third * (m.Fty + m.Fpy) * uy + third * G00;
    const R s11 = third * ((m.Ftx + m.Fpx) * uy + (m.Fty + m.Fpy) * ux);
    const R half_om = R(1) - R(0.5) * om;

    R c[9];
    // h-hat_0..2 with omega = 1, plus m-hat^s'_j / |K_j|^2 (|K|^2 = 9, 6, 6, 36, 4, 4, 12, 12, 36)
    const R h0 = G00 * R(1.0 / 18.0);
    const R h1 = s10 * R(1.0 / 12.0);
    const R h2 = s01 * R(1.0 / 12.0);
    const R h3 = (R(2) * p * third + rc2 * (ux2 + uy2) - (e20 + e02)) * R(1.0 / 12.0);
    const R h4 = R(0.25) * om * (rc2 * (ux2 - uy2) - (e20 - e02));
    const R h5 = R(0.25) * om * (rc2 * ux * uy - e11);
    const R h6 = R(0.25) * (third * uy * (psi + R(2) * rho * ux2) + e21 - uy * e20 - R(2) * ux * e11)
                 - uy * (R(1.5) * h3 + R(0.5) * h4) - R(2) * ux * h5;
    const R h7 = R(0.25) * (third * ux * (psi + R(2) * rho * uy2) + e12 - R(2) * uy * e11 - ux * e02)
                 - ux * (R(1.5) * h3 - R(0.5) * h4) - R(2) * uy * h5;
    const R eq22 = third * third * p + third * psi * (ux2 + uy2) + R(3) * rc2 * ux2 * uy2;
    const R h8 = R(0.25) * (eq22 - e22 + R(2) * (uy * e21 + ux * e12) - (uy2 * e20 + ux2 * e02)
                            - R(4) * ux * uy * e11)
                 - R(2) * h3 - R(0.5) * uy2 * (R(3) * h3 + h4) - R(0.5) * ux2 * (R(3) * h3 - h4)
                 - R(4) * ux * uy * h5 - R(2) * uy * h6 - R(2) * ux * h7;

    const R m0 = R(0.5) * G00;
    const R m1 = R(0.5) * s10;
    const R m2 = R(0.5) * s01;
    const R m3 = R(0.5) * (R(3) * (s20 + s02) - R(4) * G00);
    const R m4 = half_om * (s20 - s02);
    const R m5 = half_om * s11;
    const R m6 = s01;   // (1 - 1/2)(2 sigma'_01), sigma'_21 = 0
    const R m7 = s10;
    const R m8 = R(0.5) * (R(4) * G00 - R(6) * (s20 + s02));
    c[0] = h0 + m0 * R(1.0 / 9.0);
    c[1] = h1 + m1 * R(1.0 / 6.0);
    c[2] = h2 + m2 * R(1.0 / 6.0);
    c[3] = h3 + m3 * R(1.0 / 36.0);
    c[4] = h4 + m4 * R(0.25);
    c[5] = h5 + m5 * R(0.25);
    c[6] = h6 + m6 * R(1.0 / 12.0);
    c[7] = h7 + m7 * R(1.0 / 12.0);
    c[8] = h8 + m8 * R(1.0 / 36.0);
    apply_basis(g, c);
}

// Interface-lattice collision (Sec. 5): g-hat_1..8 with the sharpening flux M_phi theta n in the
// first-order equilibria; omega^phi_{1,2} from M_phi, all other rates 1.  phi = sum f (the
// node's zeroth moment, already formed for the stencil window).
template <typename R>
__device__ __forceinline__ void collide_ace(R f[9], R phi, const Macro<R>& m, R omega_phi_6)
{
    const R third = R(1) / R(3);
    const R ux = m.ux, uy = m.uy;
    const R ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const R d = (f[5] + f[6]) + (f[7] + f[8]);
    const R k10 = (f[1] - f[3]) + (f[5] - f[6]) - (f[7] - f[8]);
    const R k01 = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const R k20 = f[1] + f[3] + d;
    const R k02 = f[2] + f[4] + d;
    const R k11 = (f[5] - f[6]) + (f[7] - f[8]);
    const R k21 = (f[5] + f[6]) - (f[7] + f[8]);
    const R k12 = (f[5] - f[6]) - (f[7] - f[8]);
    const R k22 = d;

    R g[9];
    g[0] = R(0);
    g[1] = omega_phi_6 * (phi * ux + m.jx - k10);
    g[2] = omega_phi_6 * (phi * uy + m.jy - k01);
    g[3] = (R(2) * third * phi - (ux2 + uy2) * phi - (k20 + k02) + R(2) * (ux * k10 + uy * k01))
               * R(1.0 / 12.0)
           + ux * g[1] + uy * g[2];
    g[4] = R(0.25) * (-(ux2 - uy2) * phi - (k20 - k02) + R(2) * (ux * k10 - uy * k01))
           + R(3) * (ux * g[1] - uy * g[2]);
    g[5] = R(0.25) * (-uxy * phi - k11 + ux * k01 + uy * k10) + R(1.5) * (ux * g[2] + uy * g[1]);
    g[6] = R(0.25) * (-ux * uxy * phi + k21 - uy * k20 - R(2) * ux * k11 + R(2) * uxy * k10
                      + ux2 * k01)
           + R(3) * uxy * g[1] + (R(1.5) * ux2 + R(1)) * g[2] - R(1.5) * uy * g[3]
           - R(0.5) * uy * g[4] - R(2) * ux * g[5];
    g[7] = R(0.25) * (-uxy * uy * phi + k12 - ux * k02 - R(2) * uy * k11 + R(2) * uxy * k01
                      + uy2 * k10)
           + (R(1.5) * uy2 + R(1)) * g[1] + R(3) * uxy * g[2] - R(1.5) * ux * g[3]
           + R(0.5) * ux * g[4] - R(2) * uy * g[5];
    g[8] = R(0.25) * (third * third * phi - k22 + R(2) * (ux * k12 + uy * k21)
                      - (uy2 * k20 + ux2 * k02) - R(4) * uxy * k11
                      + R(2) * uxy * (uy * k10 + ux * k01) - uxy * uxy * phi)
           + ux * (R(2) + R(3) * uy2) * g[1] + uy * (R(2) + R(3) * ux2) * g[2]
           - (R(2) + R(1.5) * (ux2 + uy2)) * g[3] + R(0.5) * (ux2 - uy2) * g[4]
           - R(4) * uxy * g[5] - R(2) * uy * g[6] - R(2) * ux * g[7];
    apply_basis(f, g);
}

// Populations from the nine raw moments (00,10,01,20,02,11,21,12,22) of D2Q9, closed form.
template <typename R>
__device__ __forceinline__ void raw_to_pop(const R r[9], R q[9])
{
    const R r00 = r[0], r10 = r[1], r01 = r[2], r20 = r[3], r02 = r[4];
    const R r11 = r[5], r21 = r[6], r12 = r[7], r22 = r[8];
    q[0] = r00 - r20 - r02 + r22;
    q[1] = R(0.5) * (r10 + r20 - r12 - r22);
    q[2] = R(0.5) * (r01 + r02 - r21 - r22);
    q[3] = R(0.5) * (-r10 + r20 + r12 - r22);
    q[4] = R(0.5) * (-r01 + r02 + r21 - r22);
    q[5] = R(0.25) * (r11 + r21 + r12 + r22);
    q[6] = R(0.25) * (-r11 + r21 - r12 + r22);
    q[7] = R(0.25) * (r11 - r21 - r12 + r22);
    q[8] = R(0.25) * (-r11 - r21 + r12 + r22);
}

// Raw moments from central moments about u (binomial shift), same moment order.
template <typename R>
__device__ __forceinline__ void central_to_raw(const R c[9], R ux, R uy, R r[9])
{
    const R c00 = c[0], c10 = c[1], c01 = c[2], c20 = c[3], c02 = c[4];
    const R c11 = c[5], c21 = c[6], c12 = c[7], c22 = c[8];
    const R ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    r[0] = c00;
    r[1] = c10 + ux * c00;
    r[2] = c01 + uy * c00;
    r[3] = c20 + R(2) * ux * c10 + ux2 * c00;
    r[4] = c02 + R(2) * uy * c01 + uy2 * c00;
    r[5] = c11 + ux * c01 + uy * c10 + uxy * c00;
    r[6] = c21 + uy * c20 + R(2) * ux * c11 + R(2) * uxy * c10 + ux2 * c01 + ux2 * uy * c00;
    r[7] = c12 + ux * c02 + R(2) * uy * c11 + R(2) * uxy * c01 + uy2 * c10 + ux * uy2 * c00;
    r[8] = c22 + R(2) * uy * c21 + R(2) * ux * c12 + uy2 * c20 + ux2 * c02 + R(4) * uxy * c11
           + R(2) * uxy * uy * c10 + R(2) * uxy * ux * c01 + uxy * uxy * c00;
}

// Equilibrium populations for initialisation: g^eq from the central moments of the transformed
// Maxwellian (Sec. 3 Eq. centralmomentsgeqcomponents), f^eq from the interface equilibria of
// Sec. 5 with the M_phi theta n term set to zero.
template <typename R>
__device__ __forceinline__ void equilibria(R phi, R p, R ux, R uy, R rho, R g[9], R f[9])
{
    const R third = R(1) / R(3);
    const R psi = p - rho * third;
    const R ux2 = ux * ux, uy2 = uy * uy;
    R c[9], r[9];
    c[0] = p;
    c[1] = -psi * ux;
    c[2] = -psi * uy;
    c[3] = p * third + psi * ux2;
    c[4] = p * third + psi * uy2;
    c[5] = psi * ux * uy;
    c[6] = -psi * (third + ux2) * uy;
    c[7] = -psi * (third + uy2) * ux;
    c[8] = third * third * third * rho + psi * (ux2 + third) * (uy2 + third);
    central_to_raw(c, ux, uy, r);
    raw_to_pop(r, g);
    c[0] = phi;
    c[1] = R(0);
    c[2] = R(0);
    c[3] = third * phi;
    c[4] = third * phi;
    c[5] = R(0);
    c[6] = R(0);
    c[7] = R(0);
    c[8] = third * third * phi;
    central_to_raw(c, ux, uy, r);
    raw_to_pop(r, f);
}

}  // namespace cmlbm
