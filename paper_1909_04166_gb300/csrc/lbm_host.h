// Host-side helpers shared by the C ABI translation units: parameter validation, per-case
// constants, storage sizes and the dispatch from lbm_precision to the kernel instantiations.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "../../include/cmlbm.h"
#include "lbm_device.cuh"

namespace cmlbm {

// Kernel launchers (lbm_step.cu), one instantiation per (compute R, storage S) pair and, for
// the step, per variant V (bit 0 single relaxation time, bit 1 interface lattice alone in the
// imposed flow).
template <typename R, typename S, int V>
cudaError_t launch_step(const void*, void*, const Geometry&, const Consts<R>&, int, int, int*,
                        int flow_sign, int cut_first_wait, cudaStream_t);
template <typename R, typename S, int V>
cudaError_t configure_step(int block);
template <typename R, typename S, int V>
int step_blocks_per_sm(int block);
template <typename R, typename S, int V>
int step_warp_strips(int nstrips);
template <typename R, typename S, int V>
cudaError_t build_step_graph(const void*, const void*, const Geometry&, const Consts<R>&, int,
                             int, int*, int, int, cudaGraphExec_t*);
// Several steps in one cooperative launch, each warp waiting only for its neighbours between
// steps (lbm_step.cu, multi_body); multi_blocks_per_sm is its residency (0 if unknown).
template <typename R, typename S, int V>
cudaError_t configure_multi(int block);
template <typename R, typename S, int V>
int multi_blocks_per_sm(int block);
template <typename R, typename S, int V>
cudaError_t launch_multi(void* a, void* b, const Geometry&, const Consts<R>&, int seg_h,
                         int block, int* err, int flow_sign, int nsteps, unsigned* prog,
                         int far_wait, cudaStream_t);
// The bounds-checked step (cascaded coupled form only): every global load, store and bulk copy
// of a step is range-checked against the two state buffers; an access outside is skipped and
// the error word gets bit 1 (LBM_ERR_INDEX).
template <typename R, typename S>
cudaError_t configure_step_checked(int block);
template <typename R, typename S>
cudaError_t launch_step_checked(const void*, void*, const Geometry&, const Consts<R>&, int, int,
                                int*, int shrink_rows, cudaStream_t);
template <typename R, typename S>
cudaError_t launch_init(const double*, const double*, const double*, const double*, void*,
                        const Geometry&, const Consts<R>&, cudaStream_t);
template <typename R, typename S>
cudaError_t launch_fields(const void*, const Geometry&, const Consts<R>&, int, double*, double*,
                          double*, double*, double*, cudaStream_t);
template <typename R, typename S>
cudaError_t launch_pack(const void*, double*, const Geometry&, const Consts<R>&, cudaStream_t);
template <typename R, typename S>
cudaError_t launch_unpack(const double*, void*, const Geometry&, const Consts<R>&,
                          cudaStream_t);
// The batched step of variant V (0 cascaded, 1 SRT, 4 Langmuir, 5 both; no imposed flow; the
// 16-bit storage modes 0 only).
template <typename R, typename S, int V>
cudaError_t configure_batch(int block);
// Several batched steps in one cooperative launch (lbm_step.cu, batch_multi_body): the tasks
// order[wbeg[w] .. wbeg[w + 1]) go to warp w, one progress word per task.
template <typename R, typename S, int V>
cudaError_t configure_batch_multi();
template <typename R, typename S, int V>
int batch_multi_blocks_per_sm();
template <typename R, typename S, int V>
cudaError_t launch_batch_multi(void* base, const BatchCase<R>*, const int2* tasks,
                               const int* order, const int* wbeg, unsigned* prog, int ntasks,
                               int nwarps, int nsteps, int parity0, int far_wait, int* err,
                               cudaStream_t);
template <typename R, typename S, int V>
cudaError_t launch_batch_step(void*, const BatchCase<R>*, const int2*, int, int, int, int*,
                              cudaStream_t);
template <typename R, typename S, int V>
cudaError_t build_batch_graph(void*, const BatchCase<R>*, const int2*, int, int, int, int*, int,
                              cudaGraphExec_t*);

inline bool valid_precision(int p)
{
    return p == LBM_FP64 || p == LBM_FP32 || p == LBM_FP32_FP16 || p == LBM_FP32_BF16;
}

inline bool valid_bc(int b) { return b == LBM_PERIODIC || b == LBM_WALL || b == LBM_FREESLIP; }

// Boundary kinds of the low and high side of one axis (the high side defaults to the low one; a
// periodic axis is periodic on both sides); false if invalid.
inline bool side_kinds(int lo, int hi_override, int* lo_out, int* hi_out)
{
    const int hi = hi_override == 0 ? lo : hi_override;
    if (!valid_bc(lo) || !valid_bc(hi) || ((lo == LBM_PERIODIC) != (hi == LBM_PERIODIC)))
        return false;
    *lo_out = lo;
    *hi_out = hi;
    return true;
}

// Step variant of a case (see launch_step): bit 0 single relaxation time, bit 1 imposed flow
// (interface lattice alone: no surface tension enters), bit 2 Langmuir isotherm.
inline int step_variant(const lbm_params& P)
{
    if (P.flow == LBM_FLOW_SHEAR) return 2 | (P.collision == LBM_SRT ? 1 : 0);
    return (P.collision == LBM_SRT ? 1 : 0) | (P.sigma_model == LBM_SIGMA_LANGMUIR ? 4 : 0);
}

inline int validate_params(const lbm_params* P)
{
    if (!P) return LBM_ERR_ARG;
    if (P->nx < 1 || P->ny < 1 || P->nx > 65536 || P->ny > 65536) return LBM_ERR_ARG;
    int k0, k1;
    if (!side_kinds(P->bc_x, P->bc_x_hi, &k0, &k1) || !side_kinds(P->bc_y, P->bc_y_hi, &k0, &k1))
        return LBM_ERR_ARG;
    if ((P->collision != LBM_CASCADED && P->collision != LBM_SRT) ||
        (P->sigma_model != LBM_SIGMA_LINEAR_T && P->sigma_model != LBM_SIGMA_LANGMUIR) ||
        (P->flow != LBM_FLOW_COUPLED && P->flow != LBM_FLOW_SHEAR))
        return LBM_ERR_ARG;
    if (!valid_precision(P->precision)) return LBM_ERR_UNSUPPORTED;
    if (step_variant(*P) != 0 && P->precision != LBM_FP64 && P->precision != LBM_FP32)
        return LBM_ERR_UNSUPPORTED;
    const double v[] = {P->rho_a, P->rho_b, P->mu_a, P->mu_b, P->sigma0, P->dsigma_dT, P->T0,
                        P->gradT_x, P->gradT_y, P->mobility, P->width, P->gx, P->gy,
                        P->rho_ref, P->store_scale_g, P->store_scale_f,
                        P->beta, P->psi0, P->gradpsi_x, P->gradpsi_y, P->u0};
    for (double d : v)
        if (!std::isfinite(d)) return LBM_ERR_PARAM;
    if (P->rho_a <= 0 || P->rho_b <= 0 || P->mu_a <= 0 || P->mu_b <= 0) return LBM_ERR_PARAM;
    if (P->width <= 0 || P->mobility <= 0) return LBM_ERR_PARAM;
    if (P->store_scale_g < 0 || P->store_scale_f < 0) return LBM_ERR_PARAM;
    if (P->sigma_model == LBM_SIGMA_LANGMUIR) {
        // psi is linear, so its maximum over the grid sits at a corner; ln(1 - psi) needs psi < 1
        for (int cx = 0; cx < 2; ++cx)
            for (int cy = 0; cy < 2; ++cy) {
                const double psi = P->psi0 + P->gradpsi_x * (cx ? P->nx - 1 : 0) +
                                   P->gradpsi_y * (cy ? P->ny - 1 : 0);
                if (!(psi < 1.0)) return LBM_ERR_PARAM;
            }
    }
    return LBM_OK;
}

// Geometry of a case: tiles, walls and free-slip sides.
inline Geometry make_geometry(const lbm_params& P)
{
    Geometry G;
    G.nx = P.nx;
    G.ny = P.ny;
    G.nstrips = (P.nx + 31) / 32;
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    side_kinds(P.bc_x, P.bc_x_hi, &x0, &x1);
    side_kinds(P.bc_y, P.bc_y_hi, &y0, &y1);
    G.wall_x = x0 != LBM_PERIODIC;
    G.wall_y = y0 != LBM_PERIODIC;
    G.slip = (x0 == LBM_FREESLIP ? 1 : 0) | (x1 == LBM_FREESLIP ? 2 : 0) |
             (y0 == LBM_FREESLIP ? 4 : 0) | (y1 == LBM_FREESLIP ? 8 : 0);
    return G;
}

inline size_t elem_bytes(int precision)
{
    switch (precision) {
    case LBM_FP64: return sizeof(double);
    case LBM_FP32: return sizeof(float);
    default: return 2;
    }
}

inline int strips_of(int nx) { return (nx + 31) / 32; }

// Bytes of one tile (32 columns of one row) of a state: 18 population planes, and in the 16-bit
// forms two FP32 zeroth-moment planes in front (Tile<S> in the device header).
inline size_t tile_bytes(int precision)
{
    switch (precision) {
    case LBM_FP64: return (size_t)Tile<double>::BYTES;
    case LBM_FP32: return (size_t)Tile<float>::BYTES;
    default: return (size_t)Tile<__half>::BYTES;
    }
}

// Elements (of the storage type) of one state buffer.
inline size_t buffer_elems(int nx, int ny, int precision)
{
    return (size_t)ny * strips_of(nx) * tile_bytes(precision) / elem_bytes(precision);
}

// Per-case constants (definitions in include/cmlbm.h and the device header).
template <typename R>
Consts<R> make_consts(const lbm_params& P)
{
    Consts<R> K;
    K.rho_b = R(P.rho_b);
    K.drho = R(P.rho_a - P.rho_b);
    K.mu_b = R(P.mu_b);
    K.dmu = R(P.mu_a - P.mu_b);
    // kappa-tilde = 3/2 sigma W with sigma = sigma0 + dsigma_dT (gradT . x)
    K.kt0 = R(1.5 * P.width * P.sigma0);
    K.dktx = R(1.5 * P.width * P.dsigma_dT * P.gradT_x);
    K.dkty = R(1.5 * P.width * P.dsigma_dT * P.gradT_y);
    K.mob = R(P.mobility);
    K.four_over_w = R(4.0 / P.width);
    // M_phi = c^2 (1/omega - 1/2) -> omega = 1 / (3 M_phi + 1/2)
    K.omega_phi = R(1.0 / (3.0 * P.mobility + 0.5));
    K.gx = R(P.gx);
    K.gy = R(P.gy);
    K.rho_ref = R(P.rho_ref);
    K.cs2_drho = R((P.rho_a - P.rho_b) / 3.0);
    // 16-bit storage: deviations from the rest state of the node, scaled (defaults per format:
    // FP16 keeps the light phase's deviations, ~1e-6 and up, in its normal range)
    double sg = 1.0, sf = 1.0;
    if (P.precision == LBM_FP32_FP16) {
        sg = P.store_scale_g > 0 ? P.store_scale_g : 16384.0;
        sf = P.store_scale_f > 0 ? P.store_scale_f : 4096.0;
    } else if (P.precision == LBM_FP32_BF16) {
        sg = P.store_scale_g > 0 ? P.store_scale_g : 1.0;
        sf = P.store_scale_f > 0 ? P.store_scale_f : 1.0;
    }
    K.st_scale[0] = R(sg);
    K.st_scale[1] = R(sf);
    K.st_inv[0] = R(1.0 / sg);
    K.st_inv[1] = R(1.0 / sf);
    K.langmuir = P.sigma_model == LBM_SIGMA_LANGMUIR ? 1 : 0;
    K.beta = R(P.beta);
    K.psi0 = R(P.psi0);
    K.gpsx = R(P.gradpsi_x);
    K.gpsy = R(P.gradpsi_y);
    K.u0pi = R(P.u0 * 3.14159265358979323846);
    K.inv_nx = R(1.0 / P.nx);
    K.inv_ny = R(1.0 / P.ny);
    return K;
}

// Call f(R{}, S{}, std::integral_constant<int, V>{}) with the compute and storage types of a
// precision mode and the step variant V (variants other than 0 exist for FP64 and FP32 only;
// validate_params rejects the other combinations).
template <class F>
auto with_variant(int precision, int variant, F&& f)
{
    using V0 = std::integral_constant<int, 0>;
    using V1 = std::integral_constant<int, 1>;
    using V2 = std::integral_constant<int, 2>;
    using V3 = std::integral_constant<int, 3>;
    using V4 = std::integral_constant<int, 4>;
    using V5 = std::integral_constant<int, 5>;
    switch (precision) {
    case LBM_FP64:
        switch (variant) {
        case 1: return f(double(), double(), V1());
        case 2: return f(double(), double(), V2());
        case 3: return f(double(), double(), V3());
        case 4: return f(double(), double(), V4());
        case 5: return f(double(), double(), V5());
        default: return f(double(), double(), V0());
        }
    case LBM_FP32_FP16: return f(float(), __half(), V0());
    case LBM_FP32_BF16: return f(float(), __nv_bfloat16(), V0());
    default:
        switch (variant) {
        case 1: return f(float(), float(), V1());
        case 2: return f(float(), float(), V2());
        case 3: return f(float(), float(), V3());
        case 4: return f(float(), float(), V4());
        case 5: return f(float(), float(), V5());
        default: return f(float(), float(), V0());
        }
    }
}

// Call f(R{}, S{}) with the compute and storage types of a precision mode.
template <class F>
auto with_types(int precision, F&& f)
{
    switch (precision) {
    case LBM_FP64: return f(double(), double());
    case LBM_FP32_FP16: return f(float(), __half());
    case LBM_FP32_BF16: return f(float(), __nv_bfloat16());
    default: return f(float(), float());
    }
}

}  // namespace cmlbm
