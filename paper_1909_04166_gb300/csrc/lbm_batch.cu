// Batched C ABI (declared in include/cmlbm.h): many independent cases of uneven grid sizes
// advanced together, one launch of the batched step kernel per time step (replayed from a CUDA
// graph), with an autotuner that picks the segment height and block size on the live batch.
//
// Orientation.  A warp owns whole strips of 32 (FP64) or 64 (FP32 arithmetic) columns, so a
// case whose width is not a multiple of that leaves lanes idle in its last strip.  Under the
// fewest-columns layout each case is stored in the orientation whose padded strips cover fewer
// nodes: a case whose transpose wins is stepped as the problem reflected across the diagonal
// (x <-> y for the grid, the boundary kinds, the temperature and surfactant gradients and the
// body force; populations 1 <-> 2, 3 <-> 4, 6 <-> 8), which the D2Q9 scheme of Secs. 3 and 5
// maps onto the reflected solution.  Fields and populations cross the boundary in the case's
// own orientation; the transposes run on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <utility>
#include <vector>

#include "../../include/cmlbm.h"
#include "lbm_device.cuh"
#include "lbm_host.h"

using namespace cmlbm;

namespace {

// runs of n >= 2 steps replay graphs of an even number of steps, 2 .. 32 (32-step graphs while at
// least 32 steps are left, then one for the even rest; the parity returns after each)
constexpr int kBatchGraphSizes = 16;

struct HostCase {
    lbm_params P;           // as stored: the reflected problem when tr
    bool tr;                // stored transposed
    Geometry G;
    Consts<double> Kd;
    Consts<float> Kf;
    long long off0, off1;   // element offsets of the two buffers
    long long nodes;
};

// Population index under the reflection x <-> y (e_a -> (e_y, e_x)).
constexpr int kDiagonal[9] = {0, 2, 1, 4, 3, 5, 8, 7, 6};

// The problem reflected across the diagonal: every x quantity becomes the y one.
lbm_params reflected(const lbm_params& p)
{
    lbm_params q = p;
    std::swap(q.nx, q.ny);
    std::swap(q.bc_x, q.bc_y);
    std::swap(q.bc_x_hi, q.bc_y_hi);
    std::swap(q.gradT_x, q.gradT_y);
    std::swap(q.gx, q.gy);
    std::swap(q.gradpsi_x, q.gradpsi_y);
    return q;
}

// t = the transpose of a, a row-major [ny][nx] host array (t is [nx][ny]).
void transpose(const double* a, int nx, int ny, double* t)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) t[(size_t)x * ny + y] = a[(size_t)y * nx + x];
}

}  // namespace

struct lbm_batch {
    std::vector<HostCase> cases;
    int precision, device;
    size_t elem;
    cudaStream_t st;
    char* base;             // all state buffers
    size_t base_bytes;
    void* dcases;           // BatchCase<R>[ncases] on the device
    int2* dtasks;
    int ntasks;
    int* err;
    double* scratch;        // 5 * max nodes doubles (init / fields)
    long long max_nodes, total_nodes;
    int variant;            // step variant shared by all cases (lbm_host.h step_variant)
    int cur;                // shared buffer parity
    int seg_h, block;
    cudaGraphExec_t graph[2][16];  // 2 (k + 1) steps from parity 0 / 1
    int last_cuda;
    // the batched multi-step kernel (lbm_batch_set_persistent): the warps' task lists and one
    // progress word per task
    int nsm;
    int use_multi, multi_bps, nwarps_multi;
    int* dorder;
    int* dwbeg;
    unsigned* dprog;
};

namespace {

int fail_cuda(lbm_batch* b, cudaError_t e)
{
    if (b) b->last_cuda = (int)e;
    return e == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA;
}

void drop_batch_graphs(lbm_batch* b)
{
    for (int k = 0; k < 2; ++k)
        for (int n = 0; n < kBatchGraphSizes; ++n)
            if (b->graph[k][n]) {
                cudaGraphExecDestroy(b->graph[k][n]);
                b->graph[k][n] = nullptr;
            }
}

// Task lists of the batched multi-step kernel: the tasks go to the warps of one 12-warp block
// per SM by the longest-first rule on their nodes (each task also reloads the two rows around
// its segment), and every warp takes its tasks in the order of their indices.
cudaError_t build_assignment(lbm_batch* b, const std::vector<int2>& tasks,
                             const std::vector<int>& seg_rows, const std::vector<int>& width)
{
    const int ntasks = (int)tasks.size();
    const int nwarps = std::max(1, std::min(ntasks, b->nsm * (kMultiBlock / 32)));
    std::vector<long long> cost(ntasks);
    for (int i = 0; i < ntasks; ++i) cost[i] = (long long)(seg_rows[i] + 2) * width[i];
    std::vector<int> idx(ntasks);
    for (int i = 0; i < ntasks; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    std::vector<std::pair<long long, int>> heap;   // (load, warp), smallest load on top
    for (int w = 0; w < nwarps; ++w) heap.push_back({0, w});
    auto later = [](const std::pair<long long, int>& a, const std::pair<long long, int>& c) {
        return a.first != c.first ? a.first > c.first : a.second > c.second;
    };
    std::make_heap(heap.begin(), heap.end(), later);
    std::vector<std::vector<int>> lists(nwarps);
    for (int i : idx) {
        std::pop_heap(heap.begin(), heap.end(), later);
        heap.back().first += cost[i];
        lists[heap.back().second].push_back(i);
        std::push_heap(heap.begin(), heap.end(), later);
    }
    std::vector<int> order, wbeg(nwarps + 1, 0);
    order.reserve(ntasks);
    for (int w = 0; w < nwarps; ++w) {
        std::sort(lists[w].begin(), lists[w].end());
        wbeg[w] = (int)order.size();
        order.insert(order.end(), lists[w].begin(), lists[w].end());
    }
    wbeg[nwarps] = (int)order.size();
    if (b->dorder) cudaFree(b->dorder);
    if (b->dwbeg) cudaFree(b->dwbeg);
    if (b->dprog) cudaFree(b->dprog);
    b->dorder = nullptr;
    b->dwbeg = nullptr;
    b->dprog = nullptr;
    cudaError_t e = cudaMalloc(&b->dorder, ntasks * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->dwbeg, (nwarps + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->dprog, ntasks * sizeof(unsigned));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->dorder, order.data(), ntasks * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->dwbeg, wbeg.data(), (nwarps + 1) * sizeof(int), cudaMemcpyHostToDevice);
    b->nwarps_multi = e == cudaSuccess ? nwarps : 0;
    return e;
}

// (Re)build the per-case descriptors and the flattened warp-task list for segment height h.
int build_tasks(lbm_batch* b, int h)
{
    const int n = (int)b->cases.size();
    std::vector<int2> tasks;
    std::vector<int> seg_rows, width;   // rows and columns of each task
    std::vector<BatchCase<double>> cd(b->precision == LBM_FP64 ? n : 0);
    std::vector<BatchCase<float>> cf(b->precision != LBM_FP64 ? n : 0);
    for (int c = 0; c < n; ++c) {
        const HostCase& hc = b->cases[c];
        const int nseg = (hc.G.ny + h - 1) / h;
        const int wstrips = with_types(b->precision, [&](auto r, auto s) {
            return step_warp_strips<decltype(r), decltype(s), 0>(hc.G.nstrips);
        });
        const int nw = wstrips * nseg;
        const int cols = hc.G.nstrips == wstrips ? 32 : 64;   // columns per warp strip
        for (int k = 0; k < nw; ++k) {
            tasks.push_back(make_int2(c, k));
            const int strip = k % wstrips, seg = k / wstrips;
            seg_rows.push_back(std::min(h, hc.G.ny - seg * h));
            width.push_back(std::min(cols, hc.G.nx - strip * cols));
        }
        if (b->precision == LBM_FP64)
            cd[c] = BatchCase<double>{hc.G, h, nseg, hc.off0, hc.off1, hc.Kd};
        else
            cf[c] = BatchCase<float>{hc.G, h, nseg, hc.off0, hc.off1, hc.Kf};
    }
    if (tasks.size() > (size_t)0x7fffffff / 32) return LBM_ERR_ARG;
    cudaStreamSynchronize(b->st);   // no launch may still read the old task list
    drop_batch_graphs(b);
    if (b->dtasks) cudaFree(b->dtasks);
    b->dtasks = nullptr;
    cudaError_t e = cudaMalloc(&b->dtasks, tasks.size() * sizeof(int2));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->dtasks, tasks.data(), tasks.size() * sizeof(int2),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        if (b->precision == LBM_FP64)
            e = cudaMemcpy(b->dcases, cd.data(), n * sizeof(BatchCase<double>),
                           cudaMemcpyHostToDevice);
        else
            e = cudaMemcpy(b->dcases, cf.data(), n * sizeof(BatchCase<float>),
                           cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = build_assignment(b, tasks, seg_rows, width);
    if (e != cudaSuccess) return fail_cuda(b, e);
    b->ntasks = (int)tasks.size();
    b->seg_h = h;
    return LBM_OK;
}

// Call f(R{}, S{}, V{}) for the batch's precision and step variant (the imposed-flow variants
// are refused at creation and never reach a kernel).
template <class F>
cudaError_t with_batch_kernel(const lbm_batch* b, F&& f)
{
    return with_variant(b->precision, b->variant, [&](auto r, auto s, auto v) -> cudaError_t {
        if constexpr ((decltype(v)::value & 2) != 0) return cudaErrorInvalidValue;
        else return f(r, s, v);
    });
}

cudaError_t configure(lbm_batch* b)
{
    return with_batch_kernel(b, [&](auto r, auto s, auto v) {
        using R = decltype(r);
        using S = decltype(s);
        constexpr int V = decltype(v)::value;
        cudaError_t e = configure_batch<R, S, V>(b->block);
        if (e != cudaSuccess) return e;
        // the multi-step kernel is optional: without it runs go to the graphs
        b->multi_bps = configure_batch_multi<R, S, V>() == cudaSuccess
                           ? batch_multi_blocks_per_sm<R, S, V>()
                           : 0;
        cudaGetLastError();
        return cudaSuccess;
    });
}

// The batched multi-step kernel takes runs of this batch: enabled, and its warps resident at
// once.
bool multi_fits(const lbm_batch* b)
{
    if (!b->use_multi || b->multi_bps <= 0 || b->nwarps_multi <= 0) return false;
    const int wpb = kMultiBlock / 32;
    return (b->nwarps_multi + wpb - 1) / wpb <= b->nsm * b->multi_bps;
}

cudaError_t launch_multi_run(lbm_batch* b, int nsteps)
{
    return with_batch_kernel(b, [&](auto r, auto s, auto v) {
        using R = decltype(r);
        return launch_batch_multi<R, decltype(s), decltype(v)::value>(
            b->base, static_cast<BatchCase<R>*>(b->dcases), b->dtasks, b->dorder, b->dwbeg,
            b->dprog, b->ntasks, b->nwarps_multi, nsteps, b->cur, 0, b->err, b->st);
    });
}

cudaError_t launch_one(lbm_batch* b)
{
    return with_batch_kernel(b, [&](auto r, auto s, auto v) {
        using R = decltype(r);
        return launch_batch_step<R, decltype(s), decltype(v)::value>(
            b->base, static_cast<BatchCase<R>*>(b->dcases), b->dtasks, b->ntasks, b->cur,
            b->block, b->err, b->st);
    });
}

// Every graph size from both buffer parities, built together the first time any is needed and
// uploaded to the device at once (as in lbm_api.cu).
cudaError_t ensure_graphs(lbm_batch* b)
{
    cudaError_t e = cudaSuccess;
    for (int par = 0; par < 2 && e == cudaSuccess; ++par)
        for (int k = 0; k < kBatchGraphSizes && e == cudaSuccess; ++k) {
            if (b->graph[par][k]) continue;
            e = with_batch_kernel(b, [&](auto r, auto s, auto v) {
                using R = decltype(r);
                return build_batch_graph<R, decltype(s), decltype(v)::value>(
                    b->base, static_cast<BatchCase<R>*>(b->dcases), b->dtasks, b->ntasks, par,
                    b->block, b->err, 2 * (k + 1), &b->graph[par][k]);
            });
            if (e == cudaSuccess) e = cudaGraphUpload(b->graph[par][k], b->st);
        }
    return e;
}

template <typename R> const Consts<R>& kref(const HostCase& hc);
template <> const Consts<double>& kref<double>(const HostCase& hc) { return hc.Kd; }
template <> const Consts<float>& kref<float>(const HostCase& hc) { return hc.Kf; }

void* case_state(lbm_batch* b, int c)
{
    const HostCase& hc = b->cases[c];
    return b->base + (size_t)(b->cur ? hc.off1 : hc.off0) * b->elem;
}

int check_err(lbm_batch* b)
{
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return fail_cuda(b, e);
    return h ? LBM_ERR_TIMEOUT : LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_params* params, int32_t ncases, lbm_batch** out)
{
    return lbm_batch_create_ex(params, ncases, LBM_BATCH_FEWEST_COLUMNS, out);
}

int lbm_batch_create_ex(const lbm_params* params, int32_t ncases, int32_t layout,
                        lbm_batch** out)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!params || ncases < 1) return LBM_ERR_ARG;
    if (layout != LBM_BATCH_AS_GIVEN && layout != LBM_BATCH_FEWEST_COLUMNS) return LBM_ERR_ARG;
    for (int c = 0; c < ncases; ++c) {
        int s = validate_params(&params[c]);
        if (s) return s;
        if (params[c].precision != params[0].precision || params[c].device != params[0].device ||
            params[c].stream != params[0].stream)
            return LBM_ERR_ARG;
        if ((step_variant(params[c]) & 2) != 0) return LBM_ERR_UNSUPPORTED;   // imposed flow
        if (step_variant(params[c]) != step_variant(params[0])) return LBM_ERR_ARG;
    }
    if (cudaSetDevice(params[0].device) != cudaSuccess) return LBM_ERR_CUDA;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_NOMEM;
    b->precision = params[0].precision;
    b->variant = step_variant(params[0]);
    b->device = params[0].device;
    b->elem = elem_bytes(b->precision);
    b->st = static_cast<cudaStream_t>(params[0].stream);
    b->block = 128;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
    b->nsm = nsm > 0 ? nsm : 1;
    long long off = 0;
    for (int c = 0; c < ncases; ++c) {
        HostCase hc;
        hc.P = params[c];
        hc.tr = false;
        if (layout == LBM_BATCH_FEWEST_COLUMNS) {
            // nodes covered by the padded strips of either orientation
            const auto covered = [&](int w, int h) {
                const int wstrips = with_types(b->precision, [&](auto r, auto s) {
                    return step_warp_strips<decltype(r), decltype(s), 0>((w + 31) / 32);
                });
                return (long long)wstrips * h;
            };
            hc.tr = covered(hc.P.ny, hc.P.nx) < covered(hc.P.nx, hc.P.ny);
            if (hc.tr) hc.P = reflected(hc.P);
        }
        hc.G = make_geometry(hc.P);
        hc.Kd = make_consts<double>(hc.P);
        hc.Kf = make_consts<float>(hc.P);
        const long long elems = (long long)buffer_elems(hc.G.nx, hc.G.ny, b->precision);
        hc.off0 = off;
        hc.off1 = off + elems;
        off += 2 * elems;      // whole tiles (multiples of 16 bytes) keep every buffer aligned
        hc.nodes = (long long)hc.G.nx * hc.G.ny;
        b->max_nodes = std::max(b->max_nodes, hc.nodes);
        b->total_nodes += hc.nodes;
        b->cases.push_back(hc);
    }
    b->base_bytes = (size_t)off * b->elem;
    cudaError_t e = cudaMalloc(&b->base, b->base_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->base, 0, b->base_bytes, b->st);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->dcases, ncases * (b->precision == LBM_FP64 ? sizeof(BatchCase<double>)
                                                                      : sizeof(BatchCase<float>)));
    if (e == cudaSuccess) e = cudaMalloc(&b->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->err, 0, sizeof(int), b->st);
    if (e == cudaSuccess) e = cudaMalloc(&b->scratch, 5 * (size_t)b->max_nodes * sizeof(double));
    if (e == cudaSuccess) e = configure(b);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    int s = e == cudaSuccess ? build_tasks(b, 16) : fail_cuda(b, e);
    if (s) {
        lbm_batch_destroy(b);
        return s;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_init_fields(lbm_batch* b, int32_t c, const double* phi, const double* p,
                          const double* ux, const double* uy)
{
    if (!b || c < 0 || c >= (int)b->cases.size() || !phi || !p || !ux || !uy) return LBM_ERR_ARG;
    cudaSetDevice(b->device);
    const HostCase& hc = b->cases[c];
    const size_t N = (size_t)hc.nodes, B = N * sizeof(double);
    const double* src[4] = {phi, p, ux, uy};
    std::vector<double> t;
    if (hc.tr) {   // the reflected fields: phi, p and the swapped velocity components
        const int nx = hc.P.ny, ny = hc.P.nx;   // the case's own grid
        t.resize(4 * N);
        const double* own[4] = {phi, p, uy, ux};
        for (int k = 0; k < 4; ++k) {
            transpose(own[k], nx, ny, t.data() + k * N);
            src[k] = t.data() + k * N;
        }
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(b->scratch + k * N, src[k], B, cudaMemcpyHostToDevice, b->st);
    double* d = b->scratch;
    if (e == cudaSuccess)
        e = with_types(b->precision, [&](auto r, auto s) {
            using R = decltype(r);
            return launch_init<R, decltype(s)>(d, d + N, d + 2 * N, d + 3 * N, case_state(b, c),
                                               hc.G, kref<R>(hc), b->st);
        });
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    return e == cudaSuccess ? LBM_OK : fail_cuda(b, e);
}

int lbm_batch_step(lbm_batch* b, int32_t nsteps)
{
    if (!b || nsteps < 0) return LBM_ERR_ARG;
    cudaSetDevice(b->device);
    int32_t k = 0;
    while (nsteps - k >= 2 && multi_fits(b)) {   // one multi-step launch per 65536 steps
        const int chunk = std::min(nsteps - k, 1 << 16);
        cudaError_t e = launch_multi_run(b, chunk);
        if (e != cudaSuccess) return fail_cuda(b, e);
        k += chunk;
        b->cur ^= chunk & 1;
    }
    while (nsteps - k >= 2) {
        const int chunk = std::min((nsteps - k) & ~1, 2 * kBatchGraphSizes);
        cudaError_t e = ensure_graphs(b);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->graph[b->cur][chunk / 2 - 1], b->st);
        if (e != cudaSuccess) return fail_cuda(b, e);
        k += chunk;                        // even chunk: parity unchanged
    }
    for (; k < nsteps; ++k) {
        cudaError_t e = launch_one(b);
        if (e != cudaSuccess) return fail_cuda(b, e);
        b->cur ^= 1;
    }
    return LBM_OK;
}

int lbm_batch_get_fields(lbm_batch* b, int32_t c, double* phi, double* p, double* ux,
                         double* uy, double* rho)
{
    if (!b || c < 0 || c >= (int)b->cases.size()) return LBM_ERR_ARG;
    cudaSetDevice(b->device);
    const HostCase& hc = b->cases[c];
    const size_t N = (size_t)hc.nodes, B = N * sizeof(double);
    double* d = b->scratch;
    cudaError_t e = with_types(b->precision, [&](auto r, auto s) {
        using R = decltype(r);
        return launch_fields<R, decltype(s)>(case_state(b, c), hc.G, kref<R>(hc), 0, d, d + N,
                                             d + 2 * N, d + 3 * N, d + 4 * N, b->st);
    });
    // destination of stored field k (phi, p, u_x, u_y, rho of the stored grid): a transposed
    // case's stored u_x is its own u_y
    double* own[5] = {phi, p, hc.tr ? uy : ux, hc.tr ? ux : uy, rho};
    double* h[5] = {own[0], own[1], own[2], own[3], own[4]};
    std::vector<double> t;
    if (hc.tr) {   // fetch the stored fields, then transpose each into the case's orientation
        t.resize(5 * N);
        for (int k = 0; k < 5; ++k) h[k] = own[k] ? t.data() + k * N : nullptr;
    }
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
        if (h[k]) e = cudaMemcpyAsync(h[k], d + k * N, B, cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return fail_cuda(b, e);
    if (hc.tr)
        for (int k = 0; k < 5; ++k)
            if (own[k]) transpose(t.data() + k * N, hc.P.nx, hc.P.ny, own[k]);
    return check_err(b);
}

int lbm_batch_get_populations(lbm_batch* b, int32_t c, double* g, double* f)
{
    if (!b || c < 0 || c >= (int)b->cases.size() || !g || !f) return LBM_ERR_ARG;
    cudaSetDevice(b->device);
    const HostCase& hc = b->cases[c];
    const size_t N = (size_t)hc.nodes;
    double* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, 18 * N * sizeof(double));
    if (e == cudaSuccess)
        e = with_types(b->precision, [&](auto r, auto s) {
            return launch_pack<double, decltype(s)>(case_state(b, c), tmp, hc.G, hc.Kd, b->st);
        });
    std::vector<double> t(hc.tr ? 18 * N : 0);
    double* hg = hc.tr ? t.data() : g;
    double* hf = hc.tr ? t.data() + 9 * N : f;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hg, tmp, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hf, tmp + 9 * N, 9 * N * sizeof(double), cudaMemcpyDeviceToHost,
                            b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return fail_cuda(b, e);
    if (hc.tr)   // population a of the case is the stored population kDiagonal[a], transposed
        for (int a = 0; a < 9; ++a) {
            transpose(hg + kDiagonal[a] * N, hc.P.nx, hc.P.ny, g + a * N);
            transpose(hf + kDiagonal[a] * N, hc.P.nx, hc.P.ny, f + a * N);
        }
    return check_err(b);
}

int lbm_batch_set_launch(lbm_batch* b, int32_t seg_rows, int32_t block_threads)
{
    if (!b || seg_rows < 0 || block_threads < 0) return LBM_ERR_ARG;
    if (block_threads && (block_threads % 32 || block_threads > 256)) return LBM_ERR_ARG;
    cudaSetDevice(b->device);
    if (block_threads) {
        b->block = block_threads;
        drop_batch_graphs(b);
        cudaError_t e = configure(b);
        if (e != cudaSuccess) return fail_cuda(b, e);
    }
    return seg_rows ? build_tasks(b, seg_rows) : LBM_OK;
}

int lbm_batch_set_persistent(lbm_batch* b, int32_t enable)
{
    if (!b || enable < 0 || enable > 1) return LBM_ERR_ARG;
    b->use_multi = enable;
    return LBM_OK;
}

int lbm_batch_get_step_path(const lbm_batch* b, int32_t* path)
{
    if (!b || !path) return LBM_ERR_ARG;
    *path = multi_fits(b) ? LBM_PATH_MULTI : LBM_PATH_GRAPHS;
    return LBM_OK;
}

int lbm_batch_get_launch(const lbm_batch* b, int32_t* seg_rows, int32_t* block_threads)
{
    if (!b) return LBM_ERR_ARG;
    if (seg_rows) *seg_rows = b->seg_h;
    if (block_threads) *block_threads = b->block;
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch* b, int32_t trial_steps, int32_t* seg_rows, int32_t* block_threads)
{
    if (!b || trial_steps < 1) return LBM_ERR_ARG;
    cudaSetDevice(b->device);
    // keep the state: trials run on it and it is restored afterwards
    void* backup = nullptr;
    cudaError_t e = cudaMalloc(&backup, b->base_bytes);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(backup, b->base, b->base_bytes, cudaMemcpyDeviceToDevice, b->st);
    if (e != cudaSuccess) {
        if (backup) cudaFree(backup);
        return fail_cuda(b, e);
    }
    const int cur0 = b->cur;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int segs[] = {8, 12, 16, 24, 32, 48, 64};
    const int blocks[] = {64, 128};
    float best = 1e30f;
    int best_seg = b->seg_h, best_block = b->block;
    int status = LBM_OK;
    for (int bl : blocks) {
        for (int sg : segs) {
            status = lbm_batch_set_launch(b, sg, bl);
            if (status) break;
            for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
                e = launch_one(b);
                b->cur ^= 1;
            }
            cudaEventRecord(e0, b->st);
            for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) {
                e = launch_one(b);
                b->cur ^= 1;
            }
            cudaEventRecord(e1, b->st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_seg = sg;
                best_block = bl;
            }
        }
        if (status || e != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cur = cur0;
    cudaError_t e2 =
        cudaMemcpyAsync(b->base, backup, b->base_bytes, cudaMemcpyDeviceToDevice, b->st);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(b->st);
    cudaFree(backup);
    if (e != cudaSuccess) return fail_cuda(b, e);
    if (e2 != cudaSuccess) return fail_cuda(b, e2);
    if (status) return status;
    status = lbm_batch_set_launch(b, best_seg, best_block);
    if (status) return status;
    if (seg_rows) *seg_rows = best_seg;
    if (block_threads) *block_threads = best_block;
    return check_err(b);
}

int64_t lbm_batch_nodes(const lbm_batch* b) { return b ? b->total_nodes : -1; }

int lbm_batch_case_transposed(const lbm_batch* b, int32_t c)
{
    if (!b || c < 0 || c >= (int)b->cases.size()) return LBM_ERR_ARG;
    return b->cases[c].tr ? 1 : 0;
}

int lbm_batch_check(lbm_batch* b)
{
    if (!b) return LBM_ERR_ARG;
    cudaSetDevice(b->device);
    return check_err(b);
}

void lbm_batch_destroy(lbm_batch* b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->st);
    drop_batch_graphs(b);
    if (b->base) cudaFree(b->base);
    if (b->dcases) cudaFree(b->dcases);
    if (b->dtasks) cudaFree(b->dtasks);
    if (b->err) cudaFree(b->err);
    if (b->scratch) cudaFree(b->scratch);
    if (b->dorder) cudaFree(b->dorder);
    if (b->dwbeg) cudaFree(b->dwbeg);
    if (b->dprog) cudaFree(b->dprog);
    delete b;
}

}  // extern "C"
