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
    // 16-bit storage, lattice 0 = fluid g-bar, 1 = interface f: deviation scale and its inverse
    // (unused for FP32 / FP64 storage)
    R st_scale[2], st_inv[2];
};

// Threads per block of the multi-step step kernel (lbm_step.cu, step_kernel_multi): 12 warps,
// one block per SM.
constexpr int kMultiBlock = 384;

// D2Q9 weights (the populations of the rest state are w_a times the zeroth moment).
__host__ __device__ constexpr double d2q9_w(int a)
{
    return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// ---------------------------------------------------------------------------------------------
// Storage.  FP32 and FP64 states hold the populations themselves.  The 16-bit states hold, per
// tile, two FP32 planes with every node's zeroth moments of the previous time level (Z_g = p*,
// Z_f = phi) and 18 planes of scaled deviations d_a = (q_a - w_a Z) s_L from the rest-state
// populations w_a Z of the node a population sits on (s_L per lattice).  Whoever writes a pushed
// population knows the destination's Z (it is in the writer's stencil window), so the reference
// costs no extra traffic, the pressure level and the phase fraction stay in FP32, and only the
// (small) departures from rest are rounded to 16 bits, with the floating exponent keeping the
// light phase's momentum significant.  sum_a q_a = Z + (sum_a d_a) / s_L.  The step stores a
// node's rest population last, with the rounding errors of its eight moving populations
// subtracted, so the 16-bit rounding does not accumulate in the lattice sums (lbm_step.cu,
// encode_err).
// ---------------------------------------------------------------------------------------------
template <typename S> struct Narrow { static constexpr bool value = sizeof(S) < 4; };

// Tile geometry in elements of S: population plane p (0..17) of column c of a tile is element
// P0 + 32 p + c; in the 16-bit form the FP32 planes Z_g, Z_f fill the first 256 bytes.
template <typename S>
struct Tile {
    static constexpr int ZBYTES = Narrow<S>::value ? 2 * 32 * 4 : 0;
    static constexpr int BYTES = ZBYTES + 18 * 32 * (int)sizeof(S);
    static constexpr int ELEMS = BYTES / (int)sizeof(S);
    static constexpr int P0 = ZBYTES / (int)sizeof(S);
};

__device__ __forceinline__ float narrow_to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float narrow_to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float narrow_to_f_or_self(__half v) { return __half2float(v); }
__device__ __forceinline__ float narrow_to_f_or_self(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float narrow_to_f_or_self(float v) { return v; }
template <typename S> __device__ __forceinline__ S f_to_narrow(float v);
template <> __device__ __forceinline__ __half f_to_narrow<__half>(float v)
{
    return __float2half_rn(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 f_to_narrow<__nv_bfloat16>(float v)
{
    return __float2bfloat16_rn(v);
}

// Population a of lattice lat from its stored value; z: the node's stored zeroth moment (16-bit
// forms only).
template <typename S, typename R>
__device__ __forceinline__ R decode(S v, R z, int lat, int a, const Consts<R>& K)
{
    if constexpr (!Narrow<S>::value) {
        return static_cast<R>(v);
    } else {
        const R inv = lat ? K.st_inv[1] : K.st_inv[0];
        return R(narrow_to_f(v)) * inv + R(d2q9_w(a)) * z;
    }
}

// Stored value of population a of lattice lat that will sit on a node whose zeroth moment (the
// reference the reader uses) is z.
template <typename S, typename R>
__device__ __forceinline__ S encode(R v, R z, int lat, int a, const Consts<R>& K)
{
    if constexpr (!Narrow<S>::value) {
        return static_cast<S>(v);
    } else {
        const R scale = lat ? K.st_scale[1] : K.st_scale[0];
        return f_to_narrow<S>(float((v - R(d2q9_w(a)) * z) * scale));
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
// Arithmetic types of the per-node update: float or double for one node, or F2 for two nodes at
// once (the two columns a lane owns in the paired FP32 step) on the packed FP32x2 instructions
// of sm_100+ (__ffma2_rn, __fadd2_rn, __fmul2_rn).  The formulas below are written once for all
// three; fmad(a, b, c) = a b + c marks the products that fuse (the packed instructions are not
// contracted by the compiler).  Transcendentals and reciprocals act on each half.
// ---------------------------------------------------------------------------------------------
struct F2 {
    float2 v;
    F2() = default;
    __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit F2(float2 p) : v(p) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
// a - b as one fused a + (-1) b
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    return F2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v));
}
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }

__device__ __forceinline__ float fmad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ F2 fmad(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

template <typename T> struct ScalarOf { using type = T; };
template <> struct ScalarOf<F2> { using type = float; };
template <typename T> using scalar_t = typename ScalarOf<T>::type;

template <typename R> __device__ __forceinline__ R log_(R v) { return log(v); }
template <> __device__ __forceinline__ float log_<float>(float v) { return logf(v); }
__device__ __forceinline__ F2 log_(F2 v) { return F2(logf(v.v.x), logf(v.v.y)); }
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
__device__ __forceinline__ F2 rcp_(F2 v)
{
    return F2(__fdividef(1.0f, v.v.x), __fdividef(1.0f, v.v.y));
}
// sqrt(v) for v >= 0: exact in double; v * rsqrt(v) in float (0 for v = 0)
template <typename R> __device__ __forceinline__ R norm_(R v) { return sqrt(v); }
template <> __device__ __forceinline__ float norm_<float>(float v)
{
    return v * rsqrtf(fmaxf(v, 1e-37f));
}
__device__ __forceinline__ F2 norm_(F2 v)
{
    return v * F2(rsqrtf(fmaxf(v.v.x, 1e-37f)), rsqrtf(fmaxf(v.v.y, 1e-37f)));
}

// ---------------------------------------------------------------------------------------------
// Nine-point stencil window of a nodal field: value at (x + i, y + j), i, j in {-1, 0, 1}.
// ---------------------------------------------------------------------------------------------
template <typename T>
struct Win {
    T sw, s, se, w, c, e, nw, n, ne;
};

// Second-order isotropic differences on the D2Q9 neighbourhood (Sec. 4, closing remark):
// grad a = 3 sum_a w_a e_a a(x + e_a) and lap a = 6 sum_a w_a (a(x + e_a) - a(x)), with
// w = 1/9 (axis) and 1/36 (diagonal).  The Hessian is the 1-10-1 weighted second difference
// across the three rows (columns) of the window; its trace equals the Laplacian.
template <typename T>
__device__ __forceinline__ void grad_iso(const Win<T>& a, T& gx, T& gy)
{
    using R = scalar_t<T>;
    const T third = T(R(1) / R(3)), twelfth = T(R(1) / R(12));
    gx = fmad(a.e - a.w, third, ((a.ne + a.se) - (a.nw + a.sw)) * twelfth);
    gy = fmad(a.n - a.s, third, ((a.ne + a.nw) - (a.se + a.sw)) * twelfth);
}

// Gradient, Laplacian and Hessian of one window, sharing the partial sums of its corners.
template <typename T>
__device__ __forceinline__ void stencils(const Win<T>& a, T& gx, T& gy, T& lap, T& hxx, T& hyy,
                                         T& hxy)
{
    using R = scalar_t<T>;
    const T third = T(R(1) / R(3)), sixth = T(R(1) / R(6)), twelfth = T(R(1) / R(12));
    const T m2 = T(R(-2));
    const T ee = a.ne + a.se, ww = a.nw + a.sw, nn = a.ne + a.nw, ss = a.se + a.sw;
    gx = fmad(a.e - a.w, third, (ee - ww) * twelfth);
    gy = fmad(a.n - a.s, third, (nn - ss) * twelfth);
    const T axis = (a.e + a.w) + (a.n + a.s);
    lap = fmad(T(R(4)), axis, fmad(T(R(-20)), a.c, nn + ss)) * sixth;
    const T mc = m2 * a.c;
    const T dxx_mid = (a.e + mc) + a.w;
    const T dyy_mid = (a.n + mc) + a.s;
    const T dxx_side = fmad(m2, a.n, nn) + fmad(m2, a.s, ss);
    const T dyy_side = fmad(m2, a.e, ee) + fmad(m2, a.w, ww);
    hxx = fmad(T(R(10)), dxx_mid, dxx_side) * twelfth;
    hyy = fmad(T(R(10)), dyy_mid, dyy_side) * twelfth;
    hxy = ((a.ne - a.nw) - (a.se - a.sw)) * T(R(0.25));
}

// Macroscopic quantities of one node that the collisions need.
template <typename T>
struct Macro {
    T rho, omega;          // density, shear relaxation rate omega_4 = omega_5
    T ux, uy, p;           // corrected velocity and pressure (Sec. 4 Eq. hydrodynamicfields)
    T Ftx, Fty, Fpx, Fpy;  // total force and net gradient pressure force
    T jx, jy;              // M_phi theta n, the interface first-order equilibrium moment
};

// Forces and corrected fields of one node, from the phi and p* windows and the streamed g-bar
// first moments (Sec. 2 properties and surface tension, Sec. 6.7 Marangoni components, Sec. 3
// net gradient pressure force, Sec. 4 Eqs. hydrodynamicfields and fluidviscosity).
template <typename T, bool LANGMUIR = false>
__device__ __forceinline__ void node_macro(const Win<T>& ph, const Win<T>& ps, T jgx, T jgy,
                                           T xf, T yf, const Consts<scalar_t<T>>& K, Macro<T>& m)
{
    using R = scalar_t<T>;
    const T one = T(R(1));
    const T phi = ph.c;
    m.rho = fmad(phi, T(K.drho), T(K.rho_b));
    const T mu = fmad(phi, T(K.dmu), T(K.mu_b));
    const T inv_rho = rcp_(m.rho);
    // omega = 1 / (nu / c_s^2 + 1/2), nu = mu / rho
    m.omega = rcp_(fmad(T(R(3)) * mu, inv_rho, T(R(0.5))));

    T dphx, dphy, lap, hxx, hyy, hxy, dpx, dpy;
    stencils(ph, dphx, dphy, lap, hxx, hyy, hxy);
    grad_iso(ps, dpx, dpy);

    // regularised normal n = grad phi / (|grad phi| + 1e-6): defined everywhere, and rounding
    // noise in the bulk phases cannot set its direction
    const T g2 = fmad(dphx, dphx, dphy * dphy);
    const T gm = norm_(g2);
    const T ig = rcp_(gm + T(R(1e-6)));
    const T nx = dphx * ig, ny = dphy * ig;
    const T nHn = fmad(nx * nx, hxx, fmad(T(R(2)) * nx * ny, hxy, ny * ny * hyy));
    T kt, dktx, dkty;   // kappa-tilde and its gradient at the node
    if constexpr (LANGMUIR) {
        const T om = one - fmad(T(K.gpsx), xf, fmad(T(K.gpsy), yf, T(K.psi0)));   // 1 - psi
        kt = T(K.kt0) * fmad(T(K.beta), log_(om), one);
        const T s = T(-K.kt0 * K.beta) * rcp_(om);                               // d kt / d psi
        dktx = s * T(K.gpsx);
        dkty = s * T(K.gpsy);
    } else {
        kt = fmad(T(K.dktx), xf, fmad(T(K.dkty), yf, T(K.kt0)));
        dktx = T(K.dktx);
        dkty = T(K.dkty);
    }
    const T cap = (kt * gm) * (nHn - lap);          // -kappa-tilde |grad phi|^2 div n
    const T mnd = T(R(0)) - fmad(nx, dktx, ny * dkty);   // -n . grad kappa-tilde
    // + |grad phi|^2 (I - n n) grad kappa-tilde
    const T Fsx = fmad(cap, nx, g2 * fmad(nx, mnd, dktx));
    const T Fsy = fmad(cap, ny, g2 * fmad(ny, mnd, dkty));
    const T dr = m.rho - T(K.rho_ref);
    m.Ftx = fmad(dr, T(K.gx), Fsx);
    m.Fty = fmad(dr, T(K.gy), Fsy);
    m.Fpx = T(K.cs2_drho) * dphx - dpx;
    m.Fpy = T(K.cs2_drho) * dphy - dpy;
    // rho c_s^2 u = sum g-bar e + c_s^2 F_t / 2
    const T three_inv_rho = T(R(3)) * inv_rho;
    m.ux = three_inv_rho * fmad(m.Ftx, T(R(1.0 / 6.0)), jgx);
    m.uy = three_inv_rho * fmad(m.Fty, T(R(1.0 / 6.0)), jgy);
    m.p = fmad(T(R(0.5)), fmad(m.Fpx, m.ux, m.Fpy * m.uy), ps.c);
    const T theta_m = T(K.mob * K.four_over_w) * (phi * (one - phi));
    m.jx = theta_m * nx;
    m.jy = theta_m * ny;
}

// Interface quantities of one node for the interface lattice alone (imposed flow): the
// sharpening flux M_phi theta n from the phi window, as in node_macro.
template <typename T>
__device__ __forceinline__ void interface_flux(const Win<T>& ph, const Consts<scalar_t<T>>& K,
                                               T& jx, T& jy)
{
    using R = scalar_t<T>;
    T dphx, dphy;
    grad_iso(ph, dphx, dphy);
    const T gm = norm_(fmad(dphx, dphx, dphy * dphy));
    const T ig = rcp_(gm + T(R(1e-6)));
    const T theta_m = T(K.mob * K.four_over_w) * (ph.c * (T(R(1)) - ph.c));
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
template <typename T>
__device__ __forceinline__ void raw_to_pop_fast(T r00, T r10, T r01, T r20, T r02, T r11, T r21,
                                                T r12, T r22, T q[9])
{
    using R = scalar_t<T>;
    const T half = T(R(0.5)), quarter = T(R(0.25));
    const T a = r20 - r22, b = r02 - r22;
    const T sx = r10 - r12, sy = r01 - r21;
    q[0] = (r00 - a) - (b + r22);
    q[1] = half * (a + sx);
    q[3] = half * (a - sx);
    q[2] = half * (b + sy);
    q[4] = half * (b - sy);
    const T s = r22 + r21, t = r22 - r21, u = r11 + r12, v = r12 - r11;
    q[5] = quarter * (s + u);
    q[6] = quarter * (s - u);
    q[7] = quarter * (t - v);
    q[8] = quarter * (t + v);
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
template <typename T>
__device__ __forceinline__ void collide_fluid(T g[9], T pstar, const Macro<T>& m)
{
    using R = scalar_t<T>;
    const T third = T(R(1) / R(3)), ninth = T(R(1) / R(9)), half = T(R(0.5));
    const T two = T(R(2));
    const T ux = m.ux, uy = m.uy, p = m.p, rho = m.rho, om = m.omega;
    const T ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const T rc2 = rho * third;                 // rho c^2
    const T psi = p - rc2;                     // p - rho c^2
    // second-order raw moments of g-bar that survive the collision (deviator and 11)
    const T dev = (g[1] + g[3]) - (g[2] + g[4]);
    const T e11 = (g[5] - g[6]) + (g[7] - g[8]);
    // central moments of V: deviator and 11, relaxed at omega
    const T a2 = fmad(T(R(-2)), rc2, p);
    const T dxy = ux2 - uy2, sxy = ux2 + uy2;
    const T keep = T(R(1)) - om, ompsi = om * psi;
    const T dP = fmad(keep, fmad(a2, dxy, dev), ompsi * dxy);
    const T cP = fmad(keep, fmad(a2, uxy, e11), ompsi * uxy);
    // post-collision central moments of order >= 2 (equilibria except dP, cP)
    const T tP = fmad(psi, sxy, T(R(2) / R(3)) * p);
    const T c20 = half * (tP + dP), c02 = half * (tP - dP);
    const T mpsi = T(R(0)) - psi;
    const T c21 = (mpsi * uy) * (third + ux2);
    const T c12 = (mpsi * ux) * (third + uy2);
    const T c22 = fmad(ninth, p, psi * fmad(third, sxy, ux2 * uy2));
    // back to raw moments about 0 (lower central moments: p, -psi u)
    const T b2 = fmad(T(R(-2)), psi, p), b3 = fmad(T(R(-3)), psi, p);
    const T b4 = fmad(T(R(-4)), psi, p);
    T r20 = fmad(ux2, b2, c20);
    T r02 = fmad(uy2, b2, c02);
    T r11 = fmad(uxy, b2, cP);
    T r21 = fmad(uy, c20, fmad(ux2 * uy, b3, fmad(two * ux, cP, c21)));
    T r12 = fmad(ux, c02, fmad(ux * uy2, b3, fmad(two * uy, cP, c12)));
    T r22 = fmad(two, fmad(uy, c21, ux * c12), c22);
    r22 = fmad(uy2, c20, fmad(ux2, c02, r22));
    r22 = fmad(T(R(4)) * uxy, cP, fmad(ux2 * uy2, b4, r22));
    // sources: sigma' (Gamma^t + Gamma^p matched, truncated), h-hat_0..2 and delta g^s
    const T G00 = fmad(m.Fpx, ux, m.Fpy * uy);
    const T Ftx = m.Ftx, Fty = m.Fty;
    const T FTx = Ftx + m.Fpx, FTy = Fty + m.Fpy;
    const T G3 = third * G00;
    const T s20 = fmad(T(R(2) / R(3)) * FTx, ux, G3);
    const T s02 = fmad(T(R(2) / R(3)) * FTy, uy, G3);
    const T s11 = third * fmad(FTx, uy, FTy * ux);
    const T kq = (T(R(0.25)) * keep) * (s20 - s02);   // (1/2 - omega/2)(s20 - s02)/2
    r20 = r20 + fmad(half, s20, G3 + kq);
    r02 = r02 + fmad(half, s02, G3 - kq);
    r11 = fmad(fmad(T(R(-0.5)), om, T(R(1))), s11, r11);
    r21 = fmad(ninth, Fty, r21);
    r12 = fmad(ninth, Ftx, r12);
    r22 = fmad(T(R(2) / R(9)), G00, r22);
    const T r00 = pstar + G00;
    const T r10 = fmad(rc2, ux, T(R(1) / R(6)) * Ftx);
    const T r01 = fmad(rc2, uy, T(R(1) / R(6)) * Fty);
    raw_to_pop_fast(r00, r10, r01, r20, r02, r11, r21, r12, r22, g);
}

// Fluid-lattice operator of Sec. 4 with every relaxation rate equal to the shear rate omega
// (single relaxation time, Sec. 7), in raw-moment space.  As in collide_fluid, K (h-hat_3 ..
// h-hat_8) relaxes the central moments about u of the state V (raw moments of g-bar with the
// zeroth and first replaced by p and rho c^2 u), here all of orders >= 2 at omega; K (h-hat_0,
// h-hat_1, h-hat_2) adds omega G00 / 18 K_0 and omega c^2 F_t / 12 (K_1, K_2); with equal rates
// the cumulative source is (1 - omega/2) times the source itself, whose raw moments are sigma'.
template <typename T>
__device__ __forceinline__ void collide_fluid_srt(T g[9], T pstar, const Macro<T>& m)
{
    using R = scalar_t<T>;
    const T third = T(R(1) / R(3)), ninth = T(R(1) / R(9));
    const T two = T(R(2)), m2 = T(R(-2));
    const T ux = m.ux, uy = m.uy, p = m.p, rho = m.rho, om = m.omega;
    const T ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const T rc2 = rho * third;
    const T psi = p - rc2;
    // raw moments of g-bar of orders >= 2
    const T s56 = g[5] + g[6], s78 = g[7] + g[8], d56 = g[5] - g[6], d78 = g[7] - g[8];
    const T e20 = (g[1] + g[3]) + (s56 + s78);
    const T e02 = (g[2] + g[4]) + (s56 + s78);
    const T e11 = d56 + d78, e21 = s56 - s78, e12 = d56 - d78, e22 = s56 + s78;
    // central moments of V about u
    const T a2 = fmad(m2, rc2, p), a3 = fmad(T(R(3)), rc2, T(R(0)) - p);
    const T a4 = fmad(T(R(-4)), rc2, p);
    const T v20 = fmad(ux2, a2, e20), v02 = fmad(uy2, a2, e02), v11 = fmad(uxy, a2, e11);
    const T v21 = fmad(m2 * ux, e11, fmad(T(R(0)) - uy, e20, fmad(ux2 * uy, a3, e21)));
    const T v12 = fmad(m2 * uy, e11, fmad(T(R(0)) - ux, e02, fmad(ux * uy2, a3, e12)));
    T v22 = fmad(m2, fmad(ux, e12, uy * e21), e22);
    v22 = fmad(ux2, e02, fmad(uy2, e20, v22));
    v22 = fmad(T(R(4)) * uxy, e11, fmad(ux2 * uy2, a4, v22));
    // relaxed towards the transformed Maxwellian's central moments
    const T keep = T(R(1)) - om;
    const T c20 = fmad(keep, v20, om * fmad(psi, ux2, third * p));
    const T c02 = fmad(keep, v02, om * fmad(psi, uy2, third * p));
    const T c11 = fmad(keep, v11, om * (psi * uxy));
    const T mpsi = T(R(0)) - psi;
    const T c21 = fmad(keep, v21, om * ((mpsi * uy) * (third + ux2)));
    const T c12 = fmad(keep, v12, om * ((mpsi * ux) * (third + uy2)));
    const T c22 = fmad(keep, v22, om * fmad(ninth, p, psi * fmad(third, ux2 + uy2, ux2 * uy2)));
    // back to raw moments about 0 (lower central moments: p, -psi u)
    const T b2 = fmad(m2, psi, p), b3 = fmad(T(R(-3)), psi, p), b4 = fmad(T(R(-4)), psi, p);
    T r20 = fmad(ux2, b2, c20);
    T r02 = fmad(uy2, b2, c02);
    T r11 = fmad(uxy, b2, c11);
    T r21 = fmad(uy, c20, fmad(ux2 * uy, b3, fmad(two * ux, c11, c21)));
    T r12 = fmad(ux, c02, fmad(ux * uy2, b3, fmad(two * uy, c11, c12)));
    T r22 = fmad(two, fmad(uy, c21, ux * c12), c22);
    r22 = fmad(uy2, c20, fmad(ux2, c02, r22));
    r22 = fmad(T(R(4)) * uxy, c11, fmad(ux2 * uy2, b4, r22));
    // h-hat_0..2 and (1 - omega/2) sigma'
    const T G00 = fmad(m.Fpx, ux, m.Fpy * uy);
    const T Ftx = m.Ftx, Fty = m.Fty;
    const T hs = fmad(T(R(-0.5)), om, T(R(1)));
    const T FTx = Ftx + m.Fpx, FTy = Fty + m.Fpy;
    const T G3 = third * G00;
    const T s20 = fmad(T(R(2) / R(3)) * FTx, ux, G3);
    const T s02 = fmad(T(R(2) / R(3)) * FTy, uy, G3);
    const T s11 = third * fmad(FTx, uy, FTy * ux);
    const T omG3 = om * G3;
    r20 = fmad(hs, s20, r20 + omG3);
    r02 = fmad(hs, s02, r02 + omG3);
    r11 = fmad(hs, s11, r11);
    r21 = fmad(om * ninth, Fty, r21);
    r12 = fmad(om * ninth, Ftx, r12);
    r22 = fmad(T(R(2) / R(9)) * om, G00, r22);
    const T r00 = pstar + G00;
    const T r10 = fmad(rc2, ux, T(R(1) / R(6)) * Ftx);
    const T r01 = fmad(rc2, uy, T(R(1) / R(6)) * Fty);
    raw_to_pop_fast(r00, r10, r01, r20, r02, r11, r21, r12, r22, g);
}

// Interface-lattice operator of Sec. 5 with every rate equal to omega^phi (Sec. 7): all central
// moments about u relax at omega^phi towards the equilibria (first order M_phi theta n,
// c20 = c02 = c^2 phi, c22 = c^4 phi, the others 0), in raw-moment space.
template <typename T>
__device__ __forceinline__ void collide_ace_srt(T f[9], T phi, const Macro<T>& m, T omega_phi)
{
    using R = scalar_t<T>;
    const T third = T(R(1) / R(3)), ninth = T(R(1) / R(9));
    const T two = T(R(2)), m2 = T(R(-2)), zero = T(R(0));
    const T ux = m.ux, uy = m.uy, om = omega_phi;
    const T ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const T s56 = f[5] + f[6], s78 = f[7] + f[8], d56 = f[5] - f[6], d78 = f[7] - f[8];
    const T k10 = (f[1] - f[3]) + (d56 - d78);
    const T k01 = (f[2] - f[4]) + (s56 - s78);
    const T k20 = (f[1] + f[3]) + (s56 + s78);
    const T k02 = (f[2] + f[4]) + (s56 + s78);
    const T k11 = d56 + d78, k21 = s56 - s78, k12 = d56 - d78, k22 = s56 + s78;
    // central moments about u
    const T mux = zero - ux, muy = zero - uy;
    const T c10 = fmad(mux, phi, k10), c01 = fmad(muy, phi, k01);
    const T c20 = fmad(m2 * ux, k10, fmad(ux2, phi, k20));
    const T c02 = fmad(m2 * uy, k01, fmad(uy2, phi, k02));
    const T c11 = fmad(mux, k01, fmad(muy, k10, fmad(uxy, phi, k11)));
    const T c21 = fmad(m2 * ux, k11, fmad(muy, k20, fmad(two * uxy, k10,
                       fmad(ux2, k01, fmad(ux2 * muy, phi, k21)))));
    const T c12 = fmad(m2 * uy, k11, fmad(mux, k02, fmad(two * uxy, k01,
                       fmad(uy2, k10, fmad(uy2 * mux, phi, k12)))));
    T c22 = fmad(m2, fmad(ux, k12, uy * k21), k22);
    c22 = fmad(ux2, k02, fmad(uy2, k20, c22));
    c22 = fmad(T(R(4)) * uxy, k11, fmad(m2 * uxy, fmad(uy, k10, ux * k01),
                                          fmad(ux2 * uy2, phi, c22)));
    // relaxation at one rate
    const T keep = T(R(1)) - om;
    const T a = fmad(keep, c10, om * m.jx);
    const T b = fmad(keep, c01, om * m.jy);
    const T d20 = fmad(keep, c20, om * (third * phi));
    const T d02 = fmad(keep, c02, om * (third * phi));
    const T d11 = keep * c11, d21 = keep * c21, d12 = keep * c12;
    const T d22 = fmad(keep, c22, om * (ninth * phi));
    // back to raw moments about 0
    const T r10 = fmad(ux, phi, a);
    const T r01 = fmad(uy, phi, b);
    const T r20 = fmad(two * ux, a, fmad(ux2, phi, d20));
    const T r02 = fmad(two * uy, b, fmad(uy2, phi, d02));
    const T r11 = fmad(ux, b, fmad(uy, a, fmad(uxy, phi, d11)));
    const T r21 = fmad(uy, d20, fmad(two * ux, d11, fmad(two * uxy, a,
                       fmad(ux2, b, fmad(ux2 * uy, phi, d21)))));
    const T r12 = fmad(ux, d02, fmad(two * uy, d11, fmad(two * uxy, b,
                       fmad(uy2, a, fmad(ux * uy2, phi, d12)))));
    T r22 = fmad(two, fmad(uy, d21, ux * d12), d22);
    r22 = fmad(uy2, d20, fmad(ux2, d02, r22));
    r22 = fmad(T(R(4)) * uxy, d11, fmad(two * uxy, fmad(uy, a, ux * b),
                                          fmad(ux2 * uy2, phi, r22)));
    raw_to_pop_fast(phi, r10, r01, r20, r02, r11, r21, r12, r22, f);
}

// Interface-lattice collision (Sec. 5), evaluated in raw-moment space: the cascaded operator
// relaxes the first-order central moments towards M_phi theta n at omega^phi_{1,2} and sets all
// higher central moments to their equilibria (rates 1): c20 = c02 = c^2 phi, c22 = c^4 phi,
// c11 = c21 = c12 = 0.  The closed-form g-hat of Sec. 5 is exactly this relaxation.  phi = sum f
// (the node's zeroth moment, already formed for the stencil window).
template <typename T>
__device__ __forceinline__ void collide_ace(T f[9], T phi, const Macro<T>& m, T omega_phi)
{
    using R = scalar_t<T>;
    const T third = T(R(1) / R(3)), ninth = T(R(1) / R(9)), two = T(R(2));
    const T ux = m.ux, uy = m.uy;
    const T ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const T k10 = ((f[1] - f[3]) + (f[5] - f[6])) - (f[7] - f[8]);
    const T k01 = ((f[2] - f[4]) + (f[5] + f[6])) - (f[7] + f[8]);
    const T keep = T(R(1)) - omega_phi;
    const T mux = T(R(0)) - ux, muy = T(R(0)) - uy;
    // a = c10 + omega (jx - c10) with c10 = k10 - ux phi
    const T a = fmad(keep, fmad(mux, phi, k10), omega_phi * m.jx);
    const T b = fmad(keep, fmad(muy, phi, k01), omega_phi * m.jy);
    const T cp = third * phi;
    const T r10 = fmad(ux, phi, a);
    const T r01 = fmad(uy, phi, b);
    const T r20 = fmad(two * ux, a, fmad(ux2, phi, cp));
    const T r02 = fmad(two * uy, b, fmad(uy2, phi, cp));
    const T r11 = fmad(ux, b, fmad(uy, a, uxy * phi));
    const T r21 = fmad(uy, cp, fmad(two * uxy, a, fmad(ux2, b, (ux2 * uy) * phi)));
    const T r12 = fmad(ux, cp, fmad(two * uxy, b, fmad(uy2, a, (ux * uy2) * phi)));
    const T r22 = fmad(ninth, phi, fmad(ux2 + uy2, cp, fmad(two * uxy, fmad(uy, a, ux * b),
                                                             (ux2 * uy2) * phi)));
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
