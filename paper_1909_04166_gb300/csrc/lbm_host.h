// Host-side helpers shared by the C ABI translation units: parameter validation, per-case
// constants, storage sizes and the dispatch from lbm_precision to the kernel instantiations.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "../../include/cmlbm.h"
#include "lbm_device.cuh"

namespace cmlbm {

// Kernel launchers (lbm_step.cu), one instantiation per (compute R, storage S) pair.
template <typename R, typename S>
cudaError_t launch_step(const void*, void*, const Geometry&, const Consts<R>&, int, int, int*,
                        cudaStream_t);
template <typename R, typename S>
cudaError_t configure_step(int block);
template <typename R, typename S>
int step_blocks_per_sm(int block);
template <typename R, typename S>
cudaError_t build_step_graph(const void*, const void*, const Geometry&, const Consts<R>&, int,
                             int, int*, int, cudaGraphExec_t*);
template <typename R, typename S>
cudaError_t launch_init(const double*, const double*, const double*, const double*, void*,
                        const Geometry&, const Consts<R>&, cudaStream_t);
template <typename R, typename S>
cudaError_t launch_fields(const void*, const Geometry&, const Consts<R>&, double*, double*,
                          double*, double*, double*, cudaStream_t);
template <typename R, typename S>
cudaError_t launch_pack(const void*, double*, const Geometry&, const Consts<R>&, cudaStream_t);
template <typename R, typename S>
cudaError_t launch_unpack(const double*, void*, const Geometry&, const Consts<R>&,
                          cudaStream_t);
template <typename R, typename S>
cudaError_t configure_batch(int block);
template <typename R, typename S>
cudaError_t launch_batch_step(void*, const BatchCase<R>*, const int2*, int, int, int, int*,
                              cudaStream_t);
template <typename R, typename S>
cudaError_t build_batch_graph(void*, const BatchCase<R>*, const int2*, int, int, int, int*, int,
                              cudaGraphExec_t*);

inline bool valid_precision(int p)
{
    return p == LBM_FP64 || p == LBM_FP32 || p == LBM_FP32_FP16 || p == LBM_FP32_BF16;
}

inline int validate_params(const lbm_params* P)
{
    if (!P) return LBM_ERR_ARG;
    if (P->nx < 1 || P->ny < 1 || P->nx > 65536 || P->ny > 65536) return LBM_ERR_ARG;
    if ((P->bc_x != LBM_PERIODIC && P->bc_x != LBM_WALL) ||
        (P->bc_y != LBM_PERIODIC && P->bc_y != LBM_WALL))
        return LBM_ERR_ARG;
    if (!valid_precision(P->precision)) return LBM_ERR_UNSUPPORTED;
    const double v[] = {P->rho_a, P->rho_b, P->mu_a, P->mu_b, P->sigma0, P->dsigma_dT, P->T0,
                        P->gradT_x, P->gradT_y, P->mobility, P->width, P->gx, P->gy,
                        P->rho_ref, P->store_scale_g, P->store_scale_f, P->store_ref_g};
    for (double d : v)
        if (!std::isfinite(d)) return LBM_ERR_PARAM;
    if (P->rho_a <= 0 || P->rho_b <= 0 || P->mu_a <= 0 || P->mu_b <= 0) return LBM_ERR_PARAM;
    if (P->width <= 0 || P->mobility <= 0) return LBM_ERR_PARAM;
    if (P->store_scale_g < 0 || P->store_scale_f < 0) return LBM_ERR_PARAM;
    return LBM_OK;
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

inline size_t buffer_elems(int nx, int ny) { return (size_t)ny * strips_of(nx) * 18 * 32; }

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
    // 16-bit storage: deviations from w_a * ref, scaled (defaults per format)
    double sg = 1.0, sf = 1.0;
    if (P.precision == LBM_FP32_FP16) {
        sg = P.store_scale_g > 0 ? P.store_scale_g : 16384.0;
        sf = P.store_scale_f > 0 ? P.store_scale_f : 256.0;
    } else if (P.precision == LBM_FP32_BF16) {
        sg = P.store_scale_g > 0 ? P.store_scale_g : 1.0;
        sf = P.store_scale_f > 0 ? P.store_scale_f : 1.0;
    }
    K.st_scale[0] = R(sg);
    K.st_scale[1] = R(sf);
    K.st_inv[0] = R(1.0 / sg);
    K.st_inv[1] = R(1.0 / sf);
    K.st_ref[0] = R(P.store_ref_g);
    K.st_ref[1] = R(0.5);
    return K;
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
