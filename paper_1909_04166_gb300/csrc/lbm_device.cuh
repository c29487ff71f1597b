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
    R omega_phi;         // omega^phi_{1,2}, from M_phi = c^2 (1/omega - 1/2)   (Sec. 5)
    R gx, gy, rho_ref;   // F_ext = (rho - rho_ref) g
    R cs2_drho;          // c_s^2 (rho_A - rho_B), the factor of grad rho in F_p
    // Langmuir isotherm (Sec. 6.7): kappa-tilde = kt0 [1 + beta ln(1 - psi)], psi = psi0 +
    // gpsx x + gpsy y; replaces the linear kappa-tilde above when langmuir != 0 (the step
    // kernel's variant selects it at compile time)
    int langmuir;
    R beta, psi0, gpsx, gpsy;
    R u0pi;              // imposed shear flow (Sec. 6.1): U_0 pi
    R inv_nx, inv_ny;    // 1 / L0 along x and y for the imposed flow
    // 16-bit storage codec, lattice 0 = fluid g-bar, 1 = interface f: the stored number is
    // (q_a - w_a ref) * scale; unused for FP32 / FP64 storage
    R st_scale[2], st_inv[2], st_ref[2];
};

// D2Q9 weights (the populations of the rest state are w_a times the zeroth moment).
__host__ __device__ constexpr double d2q9_w(int a)
{
    return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// ---------------------------------------------------------------------------------------------
// Storage codec.  FP32 and FP64 states hold the populations themselves; FP16 / BF16 states
// hold scaled deviations from the rest-state weights times a per-lattice reference.
// ---------------------------------------------------------------------------------------------
template <typename S> struct Narrow { static constexpr bool value = sizeof(S) < 4; };

__device__ __forceinline__ float narrow_to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float narrow_to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename S> __device__ __forceinline__ S f_to_narrow(float v);
template <> __device__ __forceinline__ __half f_to_narrow<__half>(float v)
{
    return __float2half_rn(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 f_to_narrow<__nv_bfloat16>(float v)
{
    return __float2bfloat16_rn(v);
}

template <typename S, typename R>
__device__ __forceinline__ R decode(S v, int lat, int a, const Consts<R>& K)
{
    if constexpr (!Narrow<S>::value) {
        return static_cast<R>(v);
    } else {
        const R inv = lat ? K.st_inv[1] : K.st_inv[0];
        const R ref = lat ? K.st_ref[1] : K.st_ref[0];
        return narrow_to_f(v) * inv + R(d2q9_w(a)) * ref;
    }
}

template <typename S, typename R>
__device__ __forceinline__ S encode(R v, int lat, int a, const Consts<R>& K)
{
    if constexpr (!Narrow<S>::value) {
        return static_cast<S>(v);
    } else {
        const R scale = lat ? K.st_scale[1] : K.st_scale[0];
        const R ref = lat ? K.st_ref[1] : K.st_ref[0];
        return f_to_narrow<S>((v - R(d2q9_w(a)) * ref) * scale);
    }
}

// Sum of the nine decoded populations of one lattice from their stored values (the weights
// sum to one, so the reference enters once).
template <typename S, typename R>
__device__ __forceinline__ R decode_sum(const S* q, int stride, int lat, const Consts<R>& K)
{
    if constexpr (!Narrow<S>::value) {
        R s = R(0);
#pragma unroll
        for (int a = 0; a < 9; ++a) s += static_cast<R>(q[a * stride]);
        return s;
    } else {
        float s = 0.0f;
#pragma unroll
        for (int a = 0; a < 9; ++a) s += narrow_to_f(q[a * stride]);
        return s * (lat ? K.st_inv[1] : K.st_inv[0]) + (lat ? K.st_ref[1] : K.st_ref[0]);
    }
}

struct Geometry {
    int nx, ny;
    int nstrips;         // ceil(nx / 32): tiles of 32 columns per row
    int wall_x, wall_y;  // the axis has walls (either kind) instead of a period
    int slip;            // free-slip sides: bit 0 left, 1 right, 2 bottom, 3 top
};

// One case of a batch: its geometry and constants, the element offsets of its two state
// buffers inside the batch allocation, and its warp segmentation.
template <typename R>
struct BatchCase {
    Geometry G;
    int seg_h, nseg;
    long long off0, off1;
    Consts<R> K;
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

template <typename R> __device__ __forceinline__ R log_(R v) { return log(v); }
template <> __device__ __forceinline__ float log_<float>(float v) { return logf(v); }
template <typename R> __device__ __forceinline__ void sincospi_(R v, R* s, R* c)
{
    sincospi(v, s, c);
}
template <> __device__ __forceinline__ void sincospi_<float>(float v, float* s, float* c)
{
    sincospif(v, s, c);
}
template <typename R> __device__ __forceinline__ R rcp_(R v) { return R(1) / v; }
template <> __device__ __forceinline__ float rcp_<float>(float v) { return __fdividef(1.0f, v); }
template <typename R> __device__ __forceinline__ R rsqrt_(R v) { return R(1) / sqrt(v); }
template <> __device__ __forceinline__ float rsqrt_<float>(float v) { return rsqrtf(v); }
// sqrt(v) for v >= 0: exact in double; v * rsqrt(v) in float (0 for v = 0)
template <typename R> __device__ __forceinline__ R norm_(R v) { return sqrt(v); }
template <> __device__ __forceinline__ float norm_<float>(float v)
{
    return v * rsqrtf(fmaxf(v, 1e-37f));
}

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
template <typename R, bool LANGMUIR = false>
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

    // regularised normal n = grad phi / (|grad phi| + 1e-6): defined everywhere, and rounding
    // noise in the bulk phases cannot set its direction
    const R g2 = dphx * dphx + dphy * dphy;
    const R gm = norm_(g2);
    const R ig = rcp_(gm + R(1e-6));
    const R nx = dphx * ig, ny = dphy * ig;
    const R nHn = nx * nx * hxx + R(2) * nx * ny * hxy + ny * ny * hyy;
    R kt, dktx, dkty;   // kappa-tilde and its gradient at the node
    if constexpr (LANGMUIR) {
        const R om = R(1) - (K.psi0 + K.gpsx * xf + K.gpsy * yf);   // 1 - psi
        kt = K.kt0 * (R(1) + K.beta * log_(om));
        const R s = -K.kt0 * K.beta * rcp_(om);                      // d kappa-tilde / d psi
        dktx = s * K.gpsx;
        dkty = s * K.gpsy;
    } else {
        kt = K.kt0 + K.dktx * xf + K.dkty * yf;
        dktx = K.dktx;
        dkty = K.dkty;
    }
    const R cap = -kt * gm * (lap - nHn);          // -kappa-tilde |grad phi|^2 div n
    const R nd = nx * dktx + ny * dkty;             // n . grad kappa-tilde
    const R Fsx = cap * nx + g2 * (dktx - nx * nd);   // + |grad phi|^2 (I - n n) grad kappa-tilde
    const R Fsy = cap * ny + g2 * (dkty - ny * nd);
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

// Interface quantities of one node for the interface lattice alone (imposed flow): the
// sharpening flux M_phi theta n from the phi window, as in node_macro.
template <typename R>
__device__ __forceinline__ void interface_flux(const Win<R>& ph, const Consts<R>& K, R& jx, R& jy)
{
    R dphx, dphy;
    grad_iso(ph, dphx, dphy);
    const R gm = norm_(dphx * dphx + dphy * dphy);
    const R ig = rcp_(gm + R(1e-6));
    const R theta_m = K.mob * K.four_over_w * ph.c * (R(1) - ph.c);
    jx = theta_m * (dphx * ig);
    jy = theta_m * (dphy * ig);
}

// The imposed single-vortex shear of Sec. 6.1 from the precomputed sin / cos of
// pi (x / L0 - 1/2) (sx, cx) and pi (y / L0 - 1/2) (sy, cy); sign +1, or -1 once reversed.
template <typename R>
__device__ __forceinline__ void imposed_velocity(R sx, R cx, R sy, R cy, R sign,
                                                 const Consts<R>& K, R& ux, R& uy)
{
    const R a = sign * K.u0pi;
    ux = -a * cx * sy;
    uy = a * sx * cy;
}

// Populations from the nine raw moments (00,10,01,20,02,11,21,12,22) of D2Q9: the closed-form
// inverse of the moment matrix, with shared partial sums.
template <typename R>
__device__ __forceinline__ void raw_to_pop_fast(R r00, R r10, R r01, R r20, R r02, R r11, R r21,
                                                R r12, R r22, R q[9])
{
    const R a = r20 - r22, b = r02 - r22;
    const R sx = r10 - r12, sy = r01 - r21;
    q[0] = (r00 - a) - (b + r22);
    q[1] = R(0.5) * (a + sx);
    q[3] = R(0.5) * (a - sx);
    q[2] = R(0.5) * (b + sy);
    q[4] = R(0.5) * (b - sy);
    const R s = r22 + r21, t = r22 - r21, u = r11 + r12, v = r12 - r11;
    q[5] = R(0.25) * (s + u);
    q[6] = R(0.25) * (s - u);
    q[7] = R(0.25) * (t - v);
    q[8] = R(0.25) * (t + v);
}

// Fluid-lattice collision (Sec. 4), evaluated in raw-moment space.  The printed update
// g-bar-tilde = g-bar + K h-hat + delta g^s is rewritten exactly as follows:
//  * K (h-hat_3 .. h-hat_8) relaxes the central moments (about u) of the state V whose raw
//    moments are those of g-bar with the zeroth and first replaced by p and rho c^2 u (the
//    printed h-hat_3..8 use exactly these); with omega = 1 for the trace, 21, 12 and 22 moments
//    those become their equilibria (Sec. 3 Eq. centralmomentsgeqcomponents) and only the
//    deviator and the 11 moment keep a memory of g-bar, relaxed at omega_4 = omega_5;
//  * K (h-hat_0, h-hat_1, h-hat_2) and delta g^s = (1/2) S + (1/2 - omega/2)(K_4, K_5 parts of S)
//    (Sec. 4 Eqs. sourcetermcumulativetransformed, cumulativesourcetermcomponents) add known
//    raw moments;
//  * g-bar itself differs from V only in the zeroth and first raw moments.
// The nine raw moments of the result are assembled and inverted once.  Inputs: the streamed
// g-bar (overwritten with the post-collision populations) and p* = sum g-bar.
template <typename R>
__device__ __forceinline__ void collide_fluid(R g[9], R pstar, const Macro<R>& m)
{
    const R third = R(1) / R(3), ninth = R(1) / R(9);
    const R ux = m.ux, uy = m.uy, p = m.p, rho = m.rho, om = m.omega;
    const R ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const R rc2 = rho * third;                 // rho c^2
    const R psi = p - rc2;                     // p - rho c^2
    // second-order raw moments of g-bar that survive the collision (deviator and 11)
    const R dev = (g[1] + g[3]) - (g[2] + g[4]);
    const R e11 = (g[5] - g[6]) + (g[7] - g[8]);
    // central moments of V: deviator and 11, relaxed at omega
    const R a2 = p - R(2) * rc2;
    const R dV = dev + a2 * (ux2 - uy2);
    const R cV = e11 + a2 * uxy;
    const R dP = dV + om * (psi * (ux2 - uy2) - dV);
    const R cP = cV + om * (psi * uxy - cV);
    // post-collision central moments of order >= 2 (equilibria except dP, cP)
    const R tP = R(2) * p * third + psi * (ux2 + uy2);
    const R c20 = R(0.5) * (tP + dP), c02 = R(0.5) * (tP - dP);
    const R c21 = -psi * (third + ux2) * uy;
    const R c12 = -psi * (third + uy2) * ux;
    const R c22 = ninth * p + third * psi * (ux2 + uy2) + psi * ux2 * uy2;
    // back to raw moments about 0 (lower central moments: p, -psi u)
    const R b2 = p - R(2) * psi, b3 = p - R(3) * psi, b4 = p - R(4) * psi;
    R r20 = c20 + ux2 * b2;
    R r02 = c02 + uy2 * b2;
    R r11 = cP + uxy * b2;
    R r21 = c21 + uy * c20 + R(2) * ux * cP + ux2 * uy * b3;
    R r12 = c12 + ux * c02 + R(2) * uy * cP + ux * uy2 * b3;
    R r22 = c22 + R(2) * (uy * c21 + ux * c12) + uy2 * c20 + ux2 * c02 + R(4) * uxy * cP
            + ux2 * uy2 * b4;
    // sources: sigma' (Gamma^t + Gamma^p matched, truncated), h-hat_0..2 and delta g^s
    const R G00 = m.Fpx * ux + m.Fpy * uy;
    const R Ftx = m.Ftx, Fty = m.Fty;
    const R s20 = R(2) * third * (Ftx + m.Fpx) * ux + third * G00;
    const R s02 = R(2) * third * (Fty + m.Fpy) * uy + third * G00;
    const R s11 = third * ((Ftx + m.Fpx) * uy + (Fty + m.Fpy) * ux);
    const R kq = R(0.25) * (R(1) - om) * (s20 - s02);   // (1/2 - omega/2)(s20 - s02)/2
    r20 += third * G00 + R(0.5) * s20 + kq;
    r02 += third * G00 + R(0.5) * s02 - kq;
    r11 += (R(1) - R(0.5) * om) * s11;
    r21 += third * third * Fty;
    r12 += third * third * Ftx;
    r22 += R(2) * ninth * G00;
    const R r00 = pstar + G00;
    const R r10 = rc2 * ux + R(0.5) * third * Ftx;
    const R r01 = rc2 * uy + R(0.5) * third * Fty;
    raw_to_pop_fast(r00, r10, r01, r20, r02, r11, r21, r12, r22, g);
}

// Fluid-lattice operator of Sec. 4 with every relaxation rate equal to the shear rate omega
// (single relaxation time, Sec. 7), in raw-moment space.  As in collide_fluid, K (h-hat_3 ..
// h-hat_8) relaxes the central moments about u of the state V (raw moments of g-bar with the
// zeroth and first replaced by p and rho c^2 u), here all of orders >= 2 at omega; K (h-hat_0,
// h-hat_1, h-hat_2) adds omega G00 / 18 K_0 and omega c^2 F_t / 12 (K_1, K_2); with equal rates
// the cumulative source is (1 - omega/2) times the source itself, whose raw moments are sigma'.
template <typename R>
__device__ __forceinline__ void collide_fluid_srt(R g[9], R pstar, const Macro<R>& m)
{
    const R third = R(1) / R(3), ninth = R(1) / R(9);
    const R ux = m.ux, uy = m.uy, p = m.p, rho = m.rho, om = m.omega;
    const R ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const R rc2 = rho * third;
    const R psi = p - rc2;
    // raw moments of g-bar of orders >= 2
    const R s56 = g[5] + g[6], s78 = g[7] + g[8], d56 = g[5] - g[6], d78 = g[7] - g[8];
    const R e20 = (g[1] + g[3]) + (s56 + s78);
    const R e02 = (g[2] + g[4]) + (s56 + s78);
    const R e11 = d56 + d78, e21 = s56 - s78, e12 = d56 - d78, e22 = s56 + s78;
    // central moments of V about u
    const R a2 = p - R(2) * rc2, a3 = R(3) * rc2 - p, a4 = p - R(4) * rc2;
    const R v20 = e20 + ux2 * a2, v02 = e02 + uy2 * a2, v11 = e11 + uxy * a2;
    const R v21 = e21 - R(2) * ux * e11 - uy * e20 + ux2 * uy * a3;
    const R v12 = e12 - R(2) * uy * e11 - ux * e02 + ux * uy2 * a3;
    const R v22 = e22 - R(2) * (ux * e12 + uy * e21) + ux2 * e02 + uy2 * e20
                  + R(4) * uxy * e11 + ux2 * uy2 * a4;
    // relaxed towards the transformed Maxwellian's central moments
    const R c20 = v20 + om * (p * third + psi * ux2 - v20);
    const R c02 = v02 + om * (p * third + psi * uy2 - v02);
    const R c11 = v11 + om * (psi * uxy - v11);
    const R c21 = v21 + om * (-psi * (third + ux2) * uy - v21);
    const R c12 = v12 + om * (-psi * (third + uy2) * ux - v12);
    const R c22 = v22 + om * (ninth * p + third * psi * (ux2 + uy2) + psi * ux2 * uy2 - v22);
    // back to raw moments about 0 (lower central moments: p, -psi u)
    const R b2 = p - R(2) * psi, b3 = p - R(3) * psi, b4 = p - R(4) * psi;
    R r20 = c20 + ux2 * b2;
    R r02 = c02 + uy2 * b2;
    R r11 = c11 + uxy * b2;
    R r21 = c21 + uy * c20 + R(2) * ux * c11 + ux2 * uy * b3;
    R r12 = c12 + ux * c02 + R(2) * uy * c11 + ux * uy2 * b3;
    R r22 = c22 + R(2) * (uy * c21 + ux * c12) + uy2 * c20 + ux2 * c02 + R(4) * uxy * c11
            + ux2 * uy2 * b4;
    // h-hat_0..2 and (1 - omega/2) sigma'
    const R G00 = m.Fpx * ux + m.Fpy * uy;
    const R Ftx = m.Ftx, Fty = m.Fty;
    const R hs = R(1) - R(0.5) * om;
    const R s20 = R(2) * third * (Ftx + m.Fpx) * ux + third * G00;
    const R s02 = R(2) * third * (Fty + m.Fpy) * uy + third * G00;
    const R s11 = third * ((Ftx + m.Fpx) * uy + (Fty + m.Fpy) * ux);
    r20 += om * third * G00 + hs * s20;
    r02 += om * third * G00 + hs * s02;
    r11 += hs * s11;
    r21 += om * ninth * Fty;
    r12 += om * ninth * Ftx;
    r22 += R(2) * ninth * om * G00;
    const R r00 = pstar + G00;
    const R r10 = rc2 * ux + R(0.5) * third * Ftx;
    const R r01 = rc2 * uy + R(0.5) * third * Fty;
    raw_to_pop_fast(r00, r10, r01, r20, r02, r11, r21, r12, r22, g);
}

// Interface-lattice operator of Sec. 5 with every rate equal to omega^phi (Sec. 7): all central
// moments about u relax at omega^phi towards the equilibria (first order M_phi theta n,
// c20 = c02 = c^2 phi, c22 = c^4 phi, the others 0), in raw-moment space.
template <typename R>
__device__ __forceinline__ void collide_ace_srt(R f[9], R phi, const Macro<R>& m, R omega_phi)
{
    const R third = R(1) / R(3), ninth = R(1) / R(9);
    const R ux = m.ux, uy = m.uy, om = omega_phi;
    const R ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const R s56 = f[5] + f[6], s78 = f[7] + f[8], d56 = f[5] - f[6], d78 = f[7] - f[8];
    const R k10 = (f[1] - f[3]) + (d56 - d78);
    const R k01 = (f[2] - f[4]) + (s56 - s78);
    const R k20 = (f[1] + f[3]) + (s56 + s78);
    const R k02 = (f[2] + f[4]) + (s56 + s78);
    const R k11 = d56 + d78, k21 = s56 - s78, k12 = d56 - d78, k22 = s56 + s78;
    // central moments about u
    const R c10 = k10 - ux * phi, c01 = k01 - uy * phi;
    const R c20 = k20 - R(2) * ux * k10 + ux2 * phi;
    const R c02 = k02 - R(2) * uy * k01 + uy2 * phi;
    const R c11 = k11 - ux * k01 - uy * k10 + uxy * phi;
    const R c21 = k21 - R(2) * ux * k11 - uy * k20 + R(2) * uxy * k10 + ux2 * k01
                  - ux2 * uy * phi;
    const R c12 = k12 - R(2) * uy * k11 - ux * k02 + R(2) * uxy * k01 + uy2 * k10
                  - ux * uy2 * phi;
    const R c22 = k22 - R(2) * (ux * k12 + uy * k21) + ux2 * k02 + uy2 * k20 + R(4) * uxy * k11
                  - R(2) * uxy * (uy * k10 + ux * k01) + ux2 * uy2 * phi;
    // relaxation at one rate
    const R a = c10 + om * (m.jx - c10);
    const R b = c01 + om * (m.jy - c01);
    const R keep = R(1) - om;
    const R d20 = c20 + om * (third * phi - c20);
    const R d02 = c02 + om * (third * phi - c02);
    const R d11 = keep * c11, d21 = keep * c21, d12 = keep * c12;
    const R d22 = c22 + om * (ninth * phi - c22);
    // back to raw moments about 0
    const R r10 = a + ux * phi;
    const R r01 = b + uy * phi;
    const R r20 = d20 + R(2) * ux * a + ux2 * phi;
    const R r02 = d02 + R(2) * uy * b + uy2 * phi;
    const R r11 = d11 + ux * b + uy * a + uxy * phi;
    const R r21 = d21 + uy * d20 + R(2) * ux * d11 + R(2) * uxy * a + ux2 * b + ux2 * uy * phi;
    const R r12 = d12 + ux * d02 + R(2) * uy * d11 + R(2) * uxy * b + uy2 * a + ux * uy2 * phi;
    const R r22 = d22 + R(2) * (uy * d21 + ux * d12) + uy2 * d20 + ux2 * d02 + R(4) * uxy * d11
                  + R(2) * uxy * (uy * a + ux * b) + ux2 * uy2 * phi;
    raw_to_pop_fast(phi, r10, r01, r20, r02, r11, r21, r12, r22, f);
}

// Interface-lattice collision (Sec. 5), evaluated in raw-moment space: the cascaded operator
// relaxes the first-order central moments towards M_phi theta n at omega^phi_{1,2} and sets all
// higher central moments to their equilibria (rates 1): c20 = c02 = c^2 phi, c22 = c^4 phi,
// c11 = c21 = c12 = 0.  The closed-form g-hat of Sec. 5 is exactly this relaxation.  phi = sum f
// (the node's zeroth moment, already formed for the stencil window).
template <typename R>
__device__ __forceinline__ void collide_ace(R f[9], R phi, const Macro<R>& m, R omega_phi)
{
    const R third = R(1) / R(3), ninth = R(1) / R(9);
    const R ux = m.ux, uy = m.uy;
    const R ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const R k10 = (f[1] - f[3]) + (f[5] - f[6]) - (f[7] - f[8]);
    const R k01 = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const R c10 = k10 - ux * phi, c01 = k01 - uy * phi;
    const R a = c10 + omega_phi * (m.jx - c10);
    const R b = c01 + omega_phi * (m.jy - c01);
    const R cp = third * phi;
    const R r10 = a + ux * phi;
    const R r01 = b + uy * phi;
    const R r20 = cp + R(2) * ux * a + ux2 * phi;
    const R r02 = cp + R(2) * uy * b + uy2 * phi;
    const R r11 = ux * b + uy * a + uxy * phi;
    const R r21 = uy * cp + R(2) * uxy * a + ux2 * b + ux2 * uy * phi;
    const R r12 = ux * cp + R(2) * uxy * b + uy2 * a + ux * uy2 * phi;
    const R r22 = ninth * phi + (ux2 + uy2) * cp + R(2) * uxy * (uy * a + ux * b)
                  + ux2 * uy2 * phi;
    raw_to_pop_fast(phi, r10, r01, r20, r02, r11, r21, r12, r22, f);
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
