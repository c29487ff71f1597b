// C ABI of the library (declared in include/cmlbm.h): parameter validation, per-case constants,
// device buffers, launches and diagnostics.  All device work goes through the kernels of
// lbm_step.cu and the reductions below; nothing here computes physics on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/cmlbm.h"
#include "lbm_device.cuh"
#include "lbm_host.h"

using namespace cmlbm;

struct lbm_ctx {
    lbm_params P;
    Geometry G;
    Consts<double> Kd;
    Consts<float> Kf;
    size_t elem;           // bytes per stored population
    size_t state_bytes;    // one buffer (18 populations per node, tiles of 32 columns)
    char* buf;             // two buffers back to back
    bool own;
    int cur;               // buffer holding the current state
    bool initialised;
    long long steps;
    int seg_h, block;
    cudaStream_t st;
    double* scratch;       // nodal fields for diagnostics / field extraction (5 N doubles)
    double* partials;      // reduction partials
    int* err;              // device error word of the step kernel (bounded waits)
    int variant;           // step variant (lbm_host.h step_variant)
    // graphs of 2 (k + 1) steps (k < kGraphSizes) from buffer 0 / 1, flow sign + / -
    cudaGraphExec_t graph[2][2][16];
    int use_graph;
    int cut_first_wait;    // lbm_inject_timeout (1: first shared-memory wait, 2: neighbour wait)
    unsigned* prog;        // progress words of the multi-step kernel, one per warp
    int use_multi;         // lbm_set_persistent
    int multi_bps;         // resident blocks per SM of the multi-step kernel (0: not usable)
    int checked;           // steps run through the bounds-checked kernel (lbm_set_checked)
    int nsm;
    int last_cuda;
};

namespace {

constexpr int kReduceSlots = 8;
// Runs of n >= 2 steps replay graphs of an even number of steps, 2 .. 32 (even: the buffer
// parity returns): 32-step graphs while at least 32 steps are left, then one graph for the even
// rest; a last odd step is a single launch.
constexpr int kGraphSizes = 16;
// Runs of n >= 2 steps go to the multi-step kernel instead where it is enabled and its grid is
// co-resident, in launches of at most this many steps.
constexpr int kMultiMaxSteps = 1 << 16;
// Progress words allocated per SM (an SM holds at most 64 resident warps).
constexpr int kMaxWarpsPerSm = 64;
// lbm_set_persistent 2 (the default with FP32 storage): the multi-step kernel where it fits and
// the segments have at least this many rows (measured on one GB300, FP32, us per step against
// graph replays: drop impact 2048 x 1024, 18-row segments, 48.7 against 54.4; 1024 x 1024,
// 9 rows, 24.5 against 26.9; Rayleigh-Taylor 256 x 1024, 3 rows, 11.0 against 11.6; Marangoni
// 512 x 256, 2 rows, 8.9 against 7.1; Laplace 64 x 64, 1 row, 5.9 against 3.7).
constexpr int kMultiAuto = 2;
constexpr int kMultiAutoMinRows = 3;

template <typename R> const Consts<R>& kref(const lbm_ctx* c);
template <> const Consts<double>& kref<double>(const lbm_ctx* c) { return c->Kd; }
template <> const Consts<float>& kref<float>(const lbm_ctx* c) { return c->Kf; }

int validate(const lbm_params* P) { return validate_params(P); }

int cuda_fail(lbm_ctx* c, cudaError_t e)
{
    if (c) c->last_cuda = (int)e;
    if (e == cudaErrorMemoryAllocation) return LBM_ERR_NOMEM;
    return LBM_ERR_CUDA;
}

void* cur_state(lbm_ctx* c) { return c->buf + (size_t)c->cur * c->state_bytes; }

// Rows per warp segment: the warps of one launch fill the resident slots of every SM a whole
// number of times (waves), with segments of about kSegRows rows.  One wave while its segments
// are no taller than that; taller grids take more waves of shorter segments, which the block
// scheduler balances across SMs (measured on the drop impact at 2048 columns: 4096 rows in one
// wave of 72-row segments 36.8 GLUPS, in four waves of 18 rows 41.7; 2048 rows 38.1 against 39.4
// in two waves; a partial wave is slower than one full wave).
constexpr int kSegRows = 16;

int default_seg_rows(const lbm_ctx* c)
{
    int strips_per_row = 1;
    const int bps = with_variant(c->P.precision, c->variant, [&](auto r, auto s, auto v) {
        using R = decltype(r);
        using S = decltype(s);
        strips_per_row = step_warp_strips<R, S, decltype(v)::value>(c->G.nstrips);
        return step_blocks_per_sm<R, S, decltype(v)::value>(c->block);
    });
    const long long resident = (long long)c->nsm * bps * (c->block / 32);
    const long long strips = strips_per_row;
    long long nseg = resident / strips;
    if (nseg < 1) nseg = 1;
    long long h = (c->G.ny + nseg - 1) / nseg;
    const long long waves = (h + kSegRows / 2) / kSegRows;
    if (waves > 1) {
        nseg *= waves;
        h = (c->G.ny + nseg - 1) / nseg;
    }
    if (h < 1) h = 1;
    if (h > c->G.ny) h = c->G.ny;
    return (int)h;
}

cudaError_t configure(lbm_ctx* c)
{
    return with_variant(c->P.precision, c->variant, [&](auto r, auto s, auto v) {
        using R = decltype(r);
        using S = decltype(s);
        constexpr int V = decltype(v)::value;
        cudaError_t e = configure_step<R, S, V>(c->block);
        if (e != cudaSuccess) return e;
        // the multi-step kernel is optional: without it runs go to the graphs
        c->multi_bps = configure_multi<R, S, V>(kMultiBlock) == cudaSuccess
                           ? multi_blocks_per_sm<R, S, V>(kMultiBlock)
                           : 0;
        cudaGetLastError();
        return cudaSuccess;
    });
}

// The multi-step kernel can take runs of this context: enabled, not in a test or debugging mode
// that needs single launches, and its grid (the current segmentation) co-resident on the device.
bool multi_fits(const lbm_ctx* c)
{
    if (!c->use_multi || c->multi_bps <= 0 || c->checked || c->cut_first_wait == 1) return false;
    // automatic: only with segments tall enough that a step outlasts the waits between steps
    if (c->use_multi == kMultiAuto && c->seg_h < kMultiAutoMinRows) return false;
    const int strips = with_variant(c->P.precision, c->variant, [&](auto r, auto s, auto v) {
        return step_warp_strips<decltype(r), decltype(s), decltype(v)::value>(c->G.nstrips);
    });
    const long long nseg = (c->G.ny + c->seg_h - 1) / c->seg_h;
    const long long warps = (long long)strips * nseg;
    const int wpb = kMultiBlock / 32;
    const long long blocks = (warps + wpb - 1) / wpb;
    return blocks <= (long long)c->nsm * c->multi_bps && warps <= (long long)c->nsm * kMaxWarpsPerSm;
}

cudaError_t launch_multi_run(lbm_ctx* c, int nsteps, int sign)
{
    void* a = cur_state(c);
    void* b = c->buf + (size_t)(1 - c->cur) * c->state_bytes;
    return with_variant(c->P.precision, c->variant, [&](auto r, auto s, auto v) {
        using R = decltype(r);
        return launch_multi<R, decltype(s), decltype(v)::value>(
            a, b, c->G, kref<R>(c), c->seg_h, kMultiBlock, c->err, sign ? sign : 1, nsteps,
            c->prog, c->cut_first_wait == 2 ? 1 : 0, c->st);
    });
}

void drop_graphs(lbm_ctx* c)
{
    for (int k = 0; k < 2; ++k)
        for (int d = 0; d < 2; ++d)
            for (int n = 0; n < kGraphSizes; ++n)
                if (c->graph[k][d][n]) {
                    cudaGraphExecDestroy(c->graph[k][d][n]);
                    c->graph[k][d][n] = nullptr;
                }
}

// Sign of the imposed flow for the step from time level t (+1 before the reversal, -1 from it
// on); 0 when the case advances the coupled lattices.
int flow_sign_at(const lbm_ctx* c, long long t)
{
    if (c->P.flow != LBM_FLOW_SHEAR) return 0;
    return (c->P.reverse_step > 0 && t >= c->P.reverse_step) ? -1 : 1;
}

cudaError_t launch_one(lbm_ctx* c, const void* src, void* dst, int sign)
{
    if (c->checked) {
        return with_variant(c->P.precision, 0, [&](auto r, auto s, auto) {
            using R = decltype(r);
            return launch_step_checked<R, decltype(s)>(src, dst, c->G, kref<R>(c), c->seg_h,
                                                       c->block, c->err,
                                                       c->checked == 2 ? 1 : 0, c->st);
        });
    }
    return with_variant(c->P.precision, c->variant, [&](auto r, auto s, auto v) {
        using R = decltype(r);
        return launch_step<R, decltype(s), decltype(v)::value>(
            src, dst, c->G, kref<R>(c), c->seg_h, c->block, c->err, sign ? sign : 1,
            c->cut_first_wait, c->st);
    });
}

// The graph of 2 (k + 1) steps from buffer `start` with flow sign `sign`.
cudaError_t build_graph(lbm_ctx* c, int start, int sign, int k)
{
    cudaGraphExec_t* slot = &c->graph[start][sign < 0 ? 1 : 0][k];
    if (*slot) return cudaSuccess;
    const void* a = c->buf + (size_t)start * c->state_bytes;
    const void* b = c->buf + (size_t)(1 - start) * c->state_bytes;
    return with_variant(c->P.precision, c->variant, [&](auto r, auto s, auto v) {
        using R = decltype(r);
        return build_step_graph<R, decltype(s), decltype(v)::value>(
            a, b, c->G, kref<R>(c), c->seg_h, c->block, c->err, sign ? sign : 1, 2 * (k + 1),
            slot);
    });
}

// A new state replaces the one a recorded device error made invalid: clear the error word.
cudaError_t clear_device_error(lbm_ctx* c)
{
    return cudaMemsetAsync(c->err, 0, sizeof(int), c->st);
}

// Every graph size from both start buffers for flow sign `sign`, built together the first time
// any of them is needed and uploaded to the device at once (a graph is otherwise uploaded at its
// first launch, which then starts late), so that later runs of any length (and parity) launch
// without building or uploading.
cudaError_t ensure_graphs(lbm_ctx* c, int sign)
{
    cudaError_t e = cudaSuccess;
    for (int start = 0; start < 2 && e == cudaSuccess; ++start)
        for (int k = 0; k < kGraphSizes && e == cudaSuccess; ++k) {
            cudaGraphExec_t& slot = c->graph[start][sign < 0 ? 1 : 0][k];
            if (slot) continue;
            e = build_graph(c, start, sign, k);
            if (e == cudaSuccess) e = cudaGraphUpload(slot, c->st);
        }
    return e;
}

// Read the step kernel's error word (synchronises the stream).
int check_device_error(lbm_ctx* c)
{
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e);
    if (h & 2) return LBM_ERR_INDEX;
    return h ? LBM_ERR_TIMEOUT : LBM_OK;
}

int make_ctx(const lbm_params* params, void* ext, size_t ext_bytes, lbm_ctx** out)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    int s = validate(params);
    if (s) return s;
    cudaError_t e = cudaSetDevice(params->device);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_NOMEM;
    c->P = *params;
    c->G = make_geometry(*params);
    c->variant = step_variant(*params);
    c->Kd = make_consts<double>(*params);
    c->Kf = make_consts<float>(*params);
    c->elem = elem_bytes(params->precision);
    c->state_bytes = buffer_elems(params->nx, params->ny, params->precision) * c->elem;
    c->st = static_cast<cudaStream_t>(params->stream);
    int dev = params->device, nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    c->nsm = nsm > 0 ? nsm : 1;
    c->block = 128;
    c->use_graph = 1;
    // the multi-step kernel automatically for FP32 storage (measured faster than graph replays
    // there on grids of tall segments; slower with FP64 and 16-bit storage)
    c->use_multi = params->precision == LBM_FP32 ? kMultiAuto : 0;
    if (ext) {
        if (ext_bytes < 2 * c->state_bytes || (reinterpret_cast<uintptr_t>(ext) & 15)) {
            delete c;
            return LBM_ERR_ARG;
        }
        c->buf = static_cast<char*>(ext);
        c->own = false;
    } else {
        e = cudaMalloc(&c->buf, 2 * c->state_bytes);
        if (e != cudaSuccess) {
            delete c;
            return e == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA;
        }
        c->own = true;
    }
    // zero the padding columns once so that every byte of the state is defined
    e = cudaMemsetAsync(c->buf, 0, 2 * c->state_bytes, c->st);
    if (e == cudaSuccess) e = cudaMalloc(&c->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), c->st);
    if (e == cudaSuccess)
        e = cudaMalloc(&c->prog, (size_t)c->nsm * kMaxWarpsPerSm * sizeof(unsigned));
    if (e == cudaSuccess) e = configure(c);
    if (e == cudaSuccess) c->seg_h = default_seg_rows(c);
    if (e != cudaSuccess) {
        int r = cuda_fail(c, e);
        if (c->own) cudaFree(c->buf);
        if (c->err) cudaFree(c->err);
        if (c->prog) cudaFree(c->prog);
        delete c;
        return r;
    }
    *out = c;
    return LBM_OK;
}

int ensure_scratch(lbm_ctx* c)
{
    if (c->scratch) return LBM_OK;
    const size_t N = (size_t)c->G.nx * c->G.ny;
    cudaError_t e = cudaMalloc(&c->scratch, 5 * N * sizeof(double));
    if (e != cudaSuccess) { c->scratch = nullptr; return cuda_fail(c, e); }
    e = cudaMalloc(&c->partials, (size_t)(4 * c->nsm + 1) * kReduceSlots * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(c->scratch);
        c->scratch = nullptr;
        c->partials = nullptr;
        return cuda_fail(c, e);
    }
    return LBM_OK;
}

int run_fields(lbm_ctx* c, double* phi, double* p, double* ux, double* uy, double* rho)
{
    cudaError_t e = with_types(c->P.precision, [&](auto r, auto s) {
        using R = decltype(r);
        return launch_fields<R, decltype(s)>(cur_state(c), c->G, kref<R>(c),
                                             flow_sign_at(c, c->steps), phi, p, ux, uy, rho,
                                             c->st);
    });
    return e == cudaSuccess ? LBM_OK : cuda_fail(c, e);
}

// ---------------------------------------------------------------------------------------------
// FP64 reductions of the diagnostics (block partials, then one block in a fixed order)
// ---------------------------------------------------------------------------------------------
struct DiagArgs {
    int nx, ny, wall_x, wall_y;
    double xc, yc, r_in, r_out;   // regions r < r_in, r > r_out (r_in < 0: none)
};

// Threads of the final reduction: kReduceSlots slots x kFinalLanes fixed-order partial sums.
constexpr int kFinalLanes = 32;

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// slots: 0 sum phi, 1 sum p, 2 max |u|^2, 3 sum p inside, 4 count inside, 5 sum p outside,
// 6 count outside, 7 non-finite count.  The regions compare squared distances with r_in^2 and
// r_out^2 and the speed is squared (square root of the maximum at the end): no FP64 square root
// per node.
__global__ void diag_partial_kernel(const double* __restrict__ phi, const double* __restrict__ p,
                                    const double* __restrict__ ux, const double* __restrict__ uy,
                                    DiagArgs A, double* __restrict__ part)
{
    double acc[kReduceSlots] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long N = (long long)A.nx * A.ny;
    const double rin2 = A.r_in * A.r_in, rout2 = A.r_out < 0 ? -1.0 : A.r_out * A.r_out;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const double ph = phi[n], pp = p[n], u = ux[n], v = uy[n];
        if (!(isfinite(ph) && isfinite(pp) && isfinite(u) && isfinite(v))) {
            acc[7] += 1.0;
            continue;
        }
        acc[0] += ph;
        acc[1] += pp;
        acc[2] = fmax(acc[2], u * u + v * v);
        if (A.r_in >= 0) {
            const int y = (int)(n / A.nx), x = (int)(n % A.nx);
            double dx = fabs(x - A.xc), dy = fabs(y - A.yc);
            if (!A.wall_x) dx = fmin(dx, A.nx - dx);
            if (!A.wall_y) dy = fmin(dy, A.ny - dy);
            const double r2 = dx * dx + dy * dy;
            if (r2 < rin2) { acc[3] += pp; acc[4] += 1.0; }
            if (r2 > rout2) { acc[5] += pp; acc[6] += 1.0; }
        }
    }
    __shared__ double sh[32][kReduceSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < kReduceSlots; ++k) {
        const double r = (k == 2) ? warp_max(acc[k]) : warp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = r;
    }
    __syncthreads();
    if (wid == 0) {
        for (int k = 0; k < kReduceSlots; ++k) {
            double r = lane < nw ? sh[lane][k] : 0.0;
            r = (k == 2) ? warp_max(r) : warp_sum(r);
            if (lane == 0) part[(size_t)blockIdx.x * kReduceSlots + k] = r;
        }
    }
}

// The block partials of diag_partial_kernel combined in a fixed order (one block of
// kReduceSlots x kFinalLanes threads): thread (j, k) folds blocks j, j + 32, j + 64, ... of
// slot k, then one thread per slot folds the 32 results in lane order.  Deterministic for a
// given block count.
__device__ __forceinline__ void fold_partials(const double* __restrict__ part, int nblocks,
                                              double r[kReduceSlots])
{
    __shared__ double sh[kFinalLanes][kReduceSlots];
    const int k = threadIdx.x % kReduceSlots, j = threadIdx.x / kReduceSlots;
    double a = 0.0;
    for (int b = j; b < nblocks; b += kFinalLanes) {
        const double v = part[(size_t)b * kReduceSlots + k];
        a = (k == 2) ? fmax(a, v) : a + v;
    }
    sh[j][k] = a;
    __syncthreads();
    if (threadIdx.x < kReduceSlots) {
        double t = 0.0;
        for (int i = 0; i < kFinalLanes; ++i) t = (k == 2) ? fmax(t, sh[i][k]) : t + sh[i][k];
        r[k] = t;
    }
}

__global__ void __launch_bounds__(kReduceSlots * kFinalLanes)
diag_final_kernel(double* __restrict__ part, int nblocks)
{
    double r[kReduceSlots];
    fold_partials(part, nblocks, r);
    if (threadIdx.x < kReduceSlots) part[(size_t)nblocks * kReduceSlots + threadIdx.x] = r[threadIdx.x];
}

// ---------------------------------------------------------------------------------------------
// Allocation-free diagnostics: the block partials live in a fixed device array instead of
// context scratch.  The array is part of the library image, so every GPU that loads the library
// holds it until the process exits.
// ---------------------------------------------------------------------------------------------
constexpr int kNoAllocMaxBlocks = 4096;          // partial-sum slots in the fixed array
constexpr int kNoAllocThreads = 256;
constexpr long long kNoAllocNodesPerBlock = 2048; // 8 nodes per thread
static __device__ __align__(256) double g_noalloc_partials[(kNoAllocMaxBlocks + 1) * kReduceSlots];

// Device address of g_noalloc_partials per device ordinal, looked up once per device and CUDA
// context (a device reset unloads the library image and the array moves).  The context identity
// comes from the driver's cuCtxGetCurrent / cuCtxGetId, reached through the runtime's entry-point
// query so that the library keeps no link-time dependency on the driver library.
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[64] = {};
unsigned long long g_noalloc_ctx[64] = {};

using CtxGetCurrentFn = int (*)(void**);                    // CUresult (CUcontext*)
using CtxGetIdFn = int (*)(void*, unsigned long long*);     // CUresult (CUcontext, id*)

// Identity of the calling thread's current CUDA context; false if it cannot be determined.
bool current_context_id(unsigned long long* id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {   // under g_noalloc_mutex
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound;
        cudaDriverEntryPointQueryResult q2 = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                             &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
                cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        looked_up = true;
    }
    if (!get_current || !get_id) return false;
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

__global__ void __launch_bounds__(kReduceSlots * kFinalLanes)
diag_store_kernel(const double* __restrict__ part, int nblocks, lbm_diag* out)
{
    __shared__ double r[kReduceSlots];
    double mine[kReduceSlots];
    fold_partials(part, nblocks, mine);
    if (threadIdx.x < kReduceSlots) r[threadIdx.x] = mine[threadIdx.x];
    __syncthreads();
    if (threadIdx.x != 0) return;
    out->sum_phi = r[0];
    out->sum_p = r[1];
    out->max_speed = sqrt(r[2]);
    out->dp_laplace = (r[4] > 0 && r[6] > 0) ? r[3] / r[4] - r[5] / r[6] : 0.0;
    out->nonfinite = (int64_t)r[7];
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------------------------
extern "C" {

int lbm_state_bytes(const lbm_params* params, size_t* bytes)
{
    if (!bytes) return LBM_ERR_ARG;
    int s = validate(params);
    if (s) return s;
    *bytes = 2 * buffer_elems(params->nx, params->ny, params->precision) *
             elem_bytes(params->precision);
    return LBM_OK;
}

int lbm_create(const lbm_params* params, lbm_ctx** out)
{
    return make_ctx(params, nullptr, 0, out);
}

int lbm_create_with_buffer(const lbm_params* params, void* device_buffer, size_t bytes,
                           lbm_ctx** out)
{
    if (!device_buffer) {
        if (out) *out = nullptr;
        return LBM_ERR_ARG;
    }
    return make_ctx(params, device_buffer, bytes, out);
}

int lbm_init_fields_device(lbm_ctx* c, const double* phi, const double* p, const double* ux,
                           const double* uy)
{
    if (!c || !phi || !p || !ux || !uy) return LBM_ERR_ARG;
    cudaSetDevice(c->P.device);
    c->cur = 0;
    cudaError_t e = clear_device_error(c);
    if (e == cudaSuccess)
        e = with_types(c->P.precision, [&](auto r, auto s) {
            using R = decltype(r);
            return launch_init<R, decltype(s)>(phi, p, ux, uy, cur_state(c), c->G, kref<R>(c),
                                               c->st);
        });
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->initialised = true;
    c->steps = 0;
    return LBM_OK;
}

int lbm_init_fields(lbm_ctx* c, const double* phi, const double* p, const double* ux,
                    const double* uy)
{
    if (!c || !phi || !p || !ux || !uy) return LBM_ERR_ARG;
    cudaSetDevice(c->P.device);
    int s = ensure_scratch(c);
    if (s) return s;
    const size_t N = (size_t)c->G.nx * c->G.ny, B = N * sizeof(double);
    const double* src[4] = {phi, p, ux, uy};
    for (int k = 0; k < 4; ++k) {
        cudaError_t e = cudaMemcpyAsync(c->scratch + k * N, src[k], B, cudaMemcpyHostToDevice,
                                        c->st);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    s = lbm_init_fields_device(c, c->scratch, c->scratch + N, c->scratch + 2 * N,
                               c->scratch + 3 * N);
    if (s) return s;
    cudaError_t e = cudaStreamSynchronize(c->st);
    return e == cudaSuccess ? LBM_OK : cuda_fail(c, e);
}

int lbm_step(lbm_ctx* c, int32_t nsteps)
{
    if (!c || nsteps < 0) return LBM_ERR_ARG;
    if (!c->initialised) return LBM_ERR_STATE;
    int32_t k = 0;
    while (k < nsteps) {
        // steps until the imposed flow reverses (the sign is constant within a run)
        const int sign = flow_sign_at(c, c->steps);
        long long run = nsteps - k;
        if (sign > 0 && c->P.reverse_step > 0)
            run = std::min<long long>(run, c->P.reverse_step - c->steps);
        // runs of two or more steps: one multi-step launch, or replays of prebuilt graphs of
        // 2 .. 32 launches
        if (run >= 2 && multi_fits(c)) {
            while (run >= 2) {
                const int chunk = (int)std::min<long long>(run, kMultiMaxSteps);
                cudaError_t e = launch_multi_run(c, chunk, sign);
                if (e != cudaSuccess) return cuda_fail(c, e);
                if (chunk & 1) c->cur = 1 - c->cur;
                k += chunk;
                run -= chunk;
                c->steps += chunk;
            }
        }
        while (c->use_graph && !c->checked && !c->cut_first_wait && run >= 2) {
            const int chunk = (int)std::min<long long>(run & ~1LL, 2 * kGraphSizes);
            cudaError_t e = ensure_graphs(c, sign);
            if (e == cudaSuccess)
                e = cudaGraphLaunch(c->graph[c->cur][sign < 0 ? 1 : 0][chunk / 2 - 1], c->st);
            if (e != cudaSuccess) return cuda_fail(c, e);
            k += chunk;
            run -= chunk;
            c->steps += chunk;   // even chunk: the current buffer is unchanged
        }
        for (; run > 0; --run, ++k) {
            void* src = cur_state(c);
            void* dst = c->buf + (size_t)(1 - c->cur) * c->state_bytes;
            cudaError_t e = launch_one(c, src, dst, sign);
            if (e != cudaSuccess) return cuda_fail(c, e);
            c->cur = 1 - c->cur;
            ++c->steps;
        }
    }
    return LBM_OK;
}

int lbm_set_graphs(lbm_ctx* c, int32_t enable)
{
    if (!c) return LBM_ERR_ARG;
    c->use_graph = enable ? 1 : 0;
    return LBM_OK;
}

int lbm_set_persistent(lbm_ctx* c, int32_t enable)
{
    if (!c || enable < 0 || enable > 2) return LBM_ERR_ARG;
    c->use_multi = enable;
    return LBM_OK;
}

int lbm_get_step_path(lbm_ctx* c, int32_t* path)
{
    if (!c || !path) return LBM_ERR_ARG;
    if (multi_fits(c)) *path = LBM_PATH_MULTI;
    else if (c->use_graph && !c->checked && !c->cut_first_wait) *path = LBM_PATH_GRAPHS;
    else *path = LBM_PATH_SINGLE;
    return LBM_OK;
}

int lbm_inject_timeout(lbm_ctx* c, int32_t enable)
{
    if (!c || enable < 0 || enable > 2) return LBM_ERR_ARG;
    c->cut_first_wait = enable;
    return LBM_OK;
}

int lbm_set_checked(lbm_ctx* c, int32_t enable)
{
    if (!c || enable < 0 || enable > 2) return LBM_ERR_ARG;
    if (enable && c->variant != 0) return LBM_ERR_UNSUPPORTED;
    if (enable) {
        cudaSetDevice(c->P.device);
        cudaError_t e = with_variant(c->P.precision, 0, [&](auto r, auto s, auto) {
            return configure_step_checked<decltype(r), decltype(s)>(c->block);
        });
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    c->checked = enable;
    return LBM_OK;
}

int lbm_get_fields(lbm_ctx* c, double* phi, double* p, double* ux, double* uy, double* rho)
{
    if (!c) return LBM_ERR_ARG;
    if (!c->initialised) return LBM_ERR_STATE;
    cudaSetDevice(c->P.device);
    int s = ensure_scratch(c);
    if (s) return s;
    const size_t N = (size_t)c->G.nx * c->G.ny, B = N * sizeof(double);
    double* d[5];
    for (int k = 0; k < 5; ++k) d[k] = c->scratch + k * N;
    s = run_fields(c, d[0], d[1], d[2], d[3], d[4]);
    if (s) return s;
    double* h[5] = {phi, p, ux, uy, rho};
    for (int k = 0; k < 5; ++k) {
        if (!h[k]) continue;
        cudaError_t e = cudaMemcpyAsync(h[k], d[k], B, cudaMemcpyDeviceToHost, c->st);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return check_device_error(c);
}

int lbm_get_populations(lbm_ctx* c, double* g, double* f)
{
    if (!c || !g || !f) return LBM_ERR_ARG;
    if (!c->initialised) return LBM_ERR_STATE;
    cudaSetDevice(c->P.device);
    const size_t N = (size_t)c->G.nx * c->G.ny;
    double* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, 18 * N * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(c, e);
    e = with_types(c->P.precision, [&](auto r, auto s) {
        return launch_pack<double, decltype(s)>(cur_state(c), tmp, c->G, c->Kd, c->st);
    });
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g, tmp, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f, tmp + 9 * N, 9 * N * sizeof(double), cudaMemcpyDeviceToHost,
                            c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return check_device_error(c);
}

int lbm_set_populations(lbm_ctx* c, const double* g, const double* f)
{
    if (!c || !g || !f) return LBM_ERR_ARG;
    cudaSetDevice(c->P.device);
    const size_t N = (size_t)c->G.nx * c->G.ny;
    double* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, 18 * N * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(c, e);
    e = cudaMemcpyAsync(tmp, g, 9 * N * sizeof(double), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tmp + 9 * N, f, 9 * N * sizeof(double), cudaMemcpyHostToDevice,
                            c->st);
    c->cur = 0;
    if (e == cudaSuccess) e = clear_device_error(c);
    if (e == cudaSuccess)
        e = with_types(c->P.precision, [&](auto r, auto s) {
            return launch_unpack<double, decltype(s)>(tmp, cur_state(c), c->G, c->Kd, c->st);
        });
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->initialised = true;
    return LBM_OK;
}

int lbm_save_state(lbm_ctx* c, void* host, size_t bytes, int64_t* steps)
{
    if (!c || !host || bytes != c->state_bytes) return LBM_ERR_ARG;
    if (!c->initialised) return LBM_ERR_STATE;
    cudaSetDevice(c->P.device);
    cudaError_t e = cudaMemcpyAsync(host, cur_state(c), bytes, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e);
    if (steps) *steps = c->steps;
    return check_device_error(c);
}

int lbm_load_state(lbm_ctx* c, const void* host, size_t bytes, int64_t steps)
{
    if (!c || !host || bytes != c->state_bytes || steps < 0) return LBM_ERR_ARG;
    cudaSetDevice(c->P.device);
    c->cur = 0;
    cudaError_t e = clear_device_error(c);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cur_state(c), host, bytes, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->initialised = true;
    c->steps = steps;
    return LBM_OK;
}

int lbm_state_device(lbm_ctx* c, void** state, int32_t* nstrips, int64_t* elements)
{
    if (!c || !state) return LBM_ERR_ARG;
    if (!c->initialised) return LBM_ERR_STATE;
    *state = cur_state(c);
    if (nstrips) *nstrips = c->G.nstrips;
    if (elements) *elements = (int64_t)buffer_elems(c->G.nx, c->G.ny, c->P.precision);
    return LBM_OK;
}

int lbm_check(lbm_ctx* c)
{
    if (!c) return LBM_ERR_ARG;
    cudaSetDevice(c->P.device);
    return check_device_error(c);
}

int lbm_diagnostics(lbm_ctx* c, double xc, double yc, double r_in, double r_out, lbm_diag* out)
{
    if (!c || !out) return LBM_ERR_ARG;
    if (!c->initialised) return LBM_ERR_STATE;
    cudaSetDevice(c->P.device);
    int s = ensure_scratch(c);
    if (s) return s;
    const size_t N = (size_t)c->G.nx * c->G.ny;
    s = run_fields(c, c->scratch, c->scratch + N, c->scratch + 2 * N, c->scratch + 3 * N,
                   c->scratch + 4 * N);
    if (s) return s;
    DiagArgs A{c->G.nx, c->G.ny, c->G.wall_x, c->G.wall_y, xc, yc, r_in, r_out};
    const int nb = 4 * c->nsm;
    diag_partial_kernel<<<nb, 256, 0, c->st>>>(c->scratch, c->scratch + N, c->scratch + 2 * N,
                                               c->scratch + 3 * N, A, c->partials);
    diag_final_kernel<<<1, kReduceSlots * kFinalLanes, 0, c->st>>>(c->partials, nb);
    double r[kReduceSlots];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r, c->partials + (size_t)nb * kReduceSlots, sizeof(r),
                            cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e);
    out->sum_phi = r[0];
    out->sum_p = r[1];
    out->max_speed = std::sqrt(r[2]);
    out->dp_laplace = (r[4] > 0 && r[6] > 0) ? r[3] / r[4] - r[5] / r[6] : 0.0;
    out->nonfinite = (int64_t)r[7];
    int s2 = check_device_error(c);
    if (s2) return s2;
    return out->nonfinite ? LBM_ERR_NONFINITE : LBM_OK;
}

int lbm_set_launch(lbm_ctx* c, int32_t seg_rows, int32_t block_threads)
{
    if (!c || seg_rows < 0 || block_threads < 0) return LBM_ERR_ARG;
    if (block_threads && (block_threads % 32 || block_threads > 256)) return LBM_ERR_ARG;
    drop_graphs(c);
    if (seg_rows) c->seg_h = seg_rows;
    if (block_threads) {
        c->block = block_threads;
        cudaSetDevice(c->P.device);
        cudaError_t e = configure(c);
        if (e == cudaSuccess && c->checked)
            e = with_variant(c->P.precision, 0, [&](auto r, auto s, auto) {
                return configure_step_checked<decltype(r), decltype(s)>(c->block);
            });
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    return LBM_OK;
}

int lbm_get_launch(lbm_ctx* c, int32_t* seg_rows, int32_t* block_threads)
{
    if (!c) return LBM_ERR_ARG;
    if (seg_rows) *seg_rows = c->seg_h;
    if (block_threads) *block_threads = c->block;
    return LBM_OK;
}

int64_t lbm_steps_done(const lbm_ctx* c) { return c ? c->steps : -1; }

void lbm_destroy(lbm_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->P.device);
    cudaStreamSynchronize(c->st);
    if (c->own) cudaFree(c->buf);
    if (c->scratch) cudaFree(c->scratch);
    if (c->partials) cudaFree(c->partials);
    if (c->err) cudaFree(c->err);
    if (c->prog) cudaFree(c->prog);
    drop_graphs(c);
    delete c;
}

const char* lbm_strerror(int s)
{
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_PARAM: return "invalid physical parameter";
    case LBM_ERR_CUDA: return "CUDA runtime error";
    case LBM_ERR_NOMEM: return "device allocation failed";
    case LBM_ERR_STATE: return "state not initialised";
    case LBM_ERR_NONFINITE: return "non-finite values in the fields";
    case LBM_ERR_UNSUPPORTED: return "unsupported precision mode";
    case LBM_ERR_TIMEOUT: return "a bounded device wait timed out (state invalid)";
    case LBM_ERR_INDEX: return "the checked step kernel found an access outside the state buffers";
    default: return "unknown status";
    }
}

int lbm_last_cuda_error(const lbm_ctx* c) { return c ? c->last_cuda : 0; }

int lbm_diagnostics_noalloc(const double* phi, const double* p, const double* ux,
                            const double* uy, int32_t nx, int32_t ny, int32_t bc_x, int32_t bc_y,
                            double xc, double yc, double r_in, double r_out, lbm_diag* out,
                            void* stream)
{
    if (!phi || !p || !ux || !uy || !out || nx < 1 || ny < 1) return LBM_ERR_ARG;
    if (!valid_bc(bc_x) || !valid_bc(bc_y)) return LBM_ERR_ARG;
    const long long N = (long long)nx * ny;
    if (N > (long long)kNoAllocMaxBlocks * kNoAllocNodesPerBlock) return LBM_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LBM_ERR_CUDA;
    double* part = nullptr;
    {
        // set-up, once per device and context, with that device current
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        unsigned long long ctx_id = 0;
        const bool have_id = current_context_id(&ctx_id);
        if (!g_noalloc_ptr[dev] || !have_id || ctx_id != g_noalloc_ctx[dev]) {
            void* addr = nullptr;
            if (cudaGetSymbolAddress(&addr, g_noalloc_partials) != cudaSuccess || !addr)
                return LBM_ERR_CUDA;
            g_noalloc_ptr[dev] = static_cast<double*>(addr);
            g_noalloc_ctx[dev] = have_id ? ctx_id : 0;
        }
        part = g_noalloc_ptr[dev];
    }
    const int nb = (int)((N + kNoAllocNodesPerBlock - 1) / kNoAllocNodesPerBlock);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DiagArgs A{nx, ny, bc_x != LBM_PERIODIC, bc_y != LBM_PERIODIC, xc, yc, r_in, r_out};
    // launched through cudaLaunchKernel so that each launch's own status is checked: a CUDA
    // error the caller left pending is not taken for ours, nor cleared
    void* a1[] = {(void*)&phi, (void*)&p, (void*)&ux, (void*)&uy, (void*)&A, (void*)&part};
    cudaError_t e = cudaLaunchKernel((const void*)diag_partial_kernel, dim3(nb),
                                     dim3(kNoAllocThreads), a1, 0, st);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    int nblocks = nb;
    void* a2[] = {(void*)&part, (void*)&nblocks, (void*)&out};
    e = cudaLaunchKernel((const void*)diag_store_kernel, dim3(1), dim3(kReduceSlots * kFinalLanes),
                         a2, 0, st);
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // extern "C"
