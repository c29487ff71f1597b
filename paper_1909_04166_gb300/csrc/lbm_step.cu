// Fused time-step kernel, equilibrium initialisation and field extraction for the coupled
// cascaded central-moment LB schemes of arXiv:1909.04166 on sm_103a.
//
// Step kernel design (one launch = one time step of both lattices over the whole grid):
//   * Each warp owns a strip of 32 columns and a segment of rows, and marches along the rows.
//     A lane owns one column: it loads the 18 streamed populations of its node with coalesced
//     loads (SoA planes), forms phi = sum f and p* = sum g-bar, and keeps a rolling 3x3 window of
//     (phi, p*) in registers; the east/west neighbours come from warp shuffles and the two halo
//     columns of the strip from one distributed load + half-warp reduction per row.  No shared
//     memory and no block-level synchronisation.
//   * Row y is updated once phi and p* of row y+1 are known: stencils, forces, corrected p and
//     u, fluid and interface collisions in registers, then the 18 post-collision populations
//     are pushed to the neighbours in the other buffer (x + e_a), with half-way bounce-back at
//     walls.  The state therefore always holds streamed (pre-collision) populations.
//   * Segments alternate their marching direction so that the two warps sharing a segment
//     boundary read its halo rows at about the same time (halo re-reads hit L2).
#include "lbm_device.cuh"

namespace cmlbm {

static constexpr unsigned FULL = 0xffffffffu;

struct StepLaunch {
    int seg_h;     // rows per segment
    int nstrips;   // ceil(nx / 32)
    int nseg;      // ceil(ny / seg_h)
};

template <typename R>
__device__ __forceinline__ R shfl_up(R v) { return __shfl_up_sync(FULL, v, 1); }
template <typename R>
__device__ __forceinline__ R shfl_dn(R v) { return __shfl_down_sync(FULL, v, 1); }

__device__ __forceinline__ int map_row(int y, const Geometry& G)
{
    if (y < 0) return G.wall_y ? 0 : y + G.ny;
    if (y >= G.ny) return G.wall_y ? G.ny - 1 : y - G.ny;
    return y;
}

// One (phi, p*) row of the window for this lane: own column, west and east neighbours.
template <typename R>
struct Row3 {
    R phw, phc, phe, psw, psc, pse;
};

// Load the 18 populations of column x in row yy, sum them, and assemble the lane's row of the
// window including the strip's halo columns xl, xr.
template <typename R, typename S>
__device__ __forceinline__ void load_row(const S* __restrict__ src, const Geometry& G, int yy,
                                         int x, int xl, int xr, int lane, int wlast, R gq[9],
                                         R fq[9], Row3<R>& row)
{
    const S* base = src + (long long)yy * G.pitch + x;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        gq[a] = load_pop<S, R>(base + a * G.plane);
        fq[a] = load_pop<S, R>(base + (9 + a) * G.plane);
    }
    // halo: lanes 0..8 read g-bar planes, lanes 16..24 read f planes, at columns xl and xr
    const int q = lane & 15;
    R hl = R(0), hr = R(0);
    if (q < 9) {
        const S* hb = src + (long long)((lane >> 4) * 9 + q) * G.plane + (long long)yy * G.pitch;
        hl = load_pop<S, R>(hb + xl);
        hr = load_pop<S, R>(hb + xr);
    }
    const R phc = ((fq[0] + fq[1]) + (fq[2] + fq[3])) + ((fq[4] + fq[5]) + (fq[6] + fq[7])) + fq[8];
    const R psc = ((gq[0] + gq[1]) + (gq[2] + gq[3])) + ((gq[4] + gq[5]) + (gq[6] + gq[7])) + gq[8];
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
        hl += __shfl_xor_sync(FULL, hl, off);
        hr += __shfl_xor_sync(FULL, hr, off);
    }
    const R psl = __shfl_sync(FULL, hl, 0), phl = __shfl_sync(FULL, hl, 16);
    const R psr = __shfl_sync(FULL, hr, 0), phr = __shfl_sync(FULL, hr, 16);
    row.phc = phc;
    row.psc = psc;
    row.phw = shfl_up(phc);
    row.psw = shfl_up(psc);
    row.phe = shfl_dn(phc);
    row.pse = shfl_dn(psc);
    if (lane == 0) { row.phw = phl; row.psw = psl; }
    if (lane == wlast) { row.phe = phr; row.pse = psr; }
}

template <typename R>
__device__ __forceinline__ void window(const Row3<R>& s, const Row3<R>& c, const Row3<R>& n,
                                       Win<R>& ph, Win<R>& ps)
{
    ph.sw = s.phw; ph.s = s.phc; ph.se = s.phe;
    ph.w = c.phw;  ph.c = c.phc; ph.e = c.phe;
    ph.nw = n.phw; ph.n = n.phc; ph.ne = n.phe;
    ps.sw = s.psw; ps.s = s.psc; ps.se = s.pse;
    ps.w = c.psw;  ps.c = c.psc; ps.e = c.pse;
    ps.nw = n.psw; ps.n = n.psc; ps.ne = n.pse;
}

// Push the post-collision populations of node (x, y) to their destinations in dst.
template <typename R, typename S>
__device__ __forceinline__ void push_node(S* __restrict__ dst, const Geometry& G, int x, int y,
                                          const R g[9], const R f[9])
{
    // neighbour rows/columns with periodic wrap; bounce flags where a wall is crossed
    int ym = y - 1, yp = y + 1, xm = x - 1, xp = x + 1;
    bool bys = false, byn = false, bxw = false, bxe = false;
    if (ym < 0) { if (G.wall_y) bys = true; else ym += G.ny; }
    if (yp >= G.ny) { if (G.wall_y) byn = true; else yp -= G.ny; }
    if (xm < 0) { if (G.wall_x) bxw = true; else xm += G.nx; }
    if (xp >= G.nx) { if (G.wall_x) bxe = true; else xp -= G.nx; }
    const long long P = G.plane;
    const long long rs = (long long)ym * G.pitch, rc = (long long)y * G.pitch,
                    rn = (long long)yp * G.pitch;
    const long long self = rc + x;
    // destination offsets within a plane and bounce flags, alpha = 0..8
    const long long off[9] = {self, rc + xp, rn + x, rc + xm, rs + x,
                              rn + xp, rn + xm, rs + xm, rs + xp};
    const bool bnc[9] = {false, bxe, byn, bxw, bys, bxe || byn, bxw || byn, bxw || bys,
                         bxe || bys};
    constexpr int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const long long og = bnc[a] ? OPP[a] * P + self : a * P + off[a];
        const long long of = bnc[a] ? (9 + OPP[a]) * P + self : (9 + a) * P + off[a];
        store_pop<S, R>(dst + og, g[a]);
        store_pop<S, R>(dst + of, f[a]);
    }
}

template <typename R, typename S>
__global__ void __launch_bounds__(256)
step_kernel(const S* __restrict__ src, S* __restrict__ dst, Geometry G, Consts<R> K,
            StepLaunch L)
{
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int strip = warp % L.nstrips;
    const int seg = warp / L.nstrips;
    if (seg >= L.nseg) return;                       // warp-uniform
    const int x0 = strip * 32;
    const int w = min(32, G.nx - x0);
    const int wlast = w - 1;
    const bool active = lane < w;
    const int x = active ? x0 + lane : x0 + wlast;   // idle lanes shadow the last column
    int xl = x0 - 1;
    if (xl < 0) xl = G.wall_x ? 0 : G.nx - 1;
    int xr = x0 + w;
    if (xr >= G.nx) xr = G.wall_x ? G.nx - 1 : xr - G.nx;

    const int ys = seg * L.seg_h;
    const int ye = min(ys + L.seg_h, G.ny);
    const bool up = (seg & 1) == 0;
    const int dir = up ? 1 : -1;
    int y = up ? ys : ye - 1;                        // first row updated
    const int nrows = ye - ys;

    R gA[9], fA[9], gB[9], fB[9];
    Row3<R> rb, rc, rn;   // rows behind (y - dir), current (y), ahead (y + dir)
    load_row<R, S>(src, G, map_row(y - dir, G), x, xl, xr, lane, wlast, gB, fB, rb);
    load_row<R, S>(src, G, y, x, xl, xr, lane, wlast, gA, fA, rc);
    const R xf = R(x);

    for (int it = 0; it < nrows; ++it, y += dir) {
        load_row<R, S>(src, G, map_row(y + dir, G), x, xl, xr, lane, wlast, gB, fB, rn);
        Win<R> ph, ps;
        if (up) window(rb, rc, rn, ph, ps);
        else window(rn, rc, rb, ph, ps);
        const R jgx = (gA[1] - gA[3]) + (gA[5] - gA[6]) - (gA[7] - gA[8]);
        const R jgy = (gA[2] - gA[4]) + (gA[5] + gA[6]) - (gA[7] + gA[8]);
        Macro<R> m;
        node_macro<R>(ph, ps, jgx, jgy, xf, R(y), K, m);
        collide_fluid<R>(gA, m);
        collide_ace<R>(fA, m, K.omega_phi_6);
        if (active) push_node<R, S>(dst, G, x, y, gA, fA);
        rb = rc;
        rc = rn;
#pragma unroll
        for (int a = 0; a < 9; ++a) { gA[a] = gB[a]; fA[a] = fB[a]; }
    }
}

// Equilibrium initialisation from nodal fields (double, row-major [ny][nx]).
template <typename R, typename S>
__global__ void init_kernel(const double* __restrict__ phi, const double* __restrict__ p,
                            const double* __restrict__ ux, const double* __restrict__ uy,
                            S* __restrict__ state, Geometry G, Consts<R> K)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)G.nx * G.ny) return;
    const int y = (int)(n / G.nx), x = (int)(n % G.nx);
    const R ph = R(phi[n]);
    const R rho = K.rho_b + ph * K.drho;
    R g[9], f[9];
    equilibria<R>(ph, R(p[n]), R(ux[n]), R(uy[n]), rho, g, f);
    const long long o = (long long)y * G.pitch + x;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        store_pop<S, R>(state + a * G.plane + o, g[a]);
        store_pop<S, R>(state + (9 + a) * G.plane + o, f[a]);
    }
}

// Macroscopic fields of a state: phi, corrected p, u, rho (double outputs, [ny][nx]).  One
// thread per node; the 3x3 neighbourhood sums are recomputed per node (diagnostic path).
template <typename R, typename S>
__global__ void fields_kernel(const S* __restrict__ state, Geometry G, Consts<R> K,
                              double* __restrict__ phi_o, double* __restrict__ p_o,
                              double* __restrict__ ux_o, double* __restrict__ uy_o,
                              double* __restrict__ rho_o)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)G.nx * G.ny) return;
    const int y = (int)(n / G.nx), x = (int)(n % G.nx);
    R vph[3][3], vps[3][3];
    for (int j = -1; j <= 1; ++j) {
        const int yy = map_row(y + j, G);
        for (int i = -1; i <= 1; ++i) {
            int xx = x + i;
            if (xx < 0) xx = G.wall_x ? 0 : xx + G.nx;
            if (xx >= G.nx) xx = G.wall_x ? G.nx - 1 : xx - G.nx;
            const S* b = state + (long long)yy * G.pitch + xx;
            R sg = R(0), sf = R(0);
            R gq[9], fq[9];
            for (int a = 0; a < 9; ++a) {
                gq[a] = load_pop<S, R>(b + a * G.plane);
                fq[a] = load_pop<S, R>(b + (9 + a) * G.plane);
            }
            sf = ((fq[0] + fq[1]) + (fq[2] + fq[3])) + ((fq[4] + fq[5]) + (fq[6] + fq[7])) + fq[8];
            sg = ((gq[0] + gq[1]) + (gq[2] + gq[3])) + ((gq[4] + gq[5]) + (gq[6] + gq[7])) + gq[8];
            vph[j + 1][i + 1] = sf;
            vps[j + 1][i + 1] = sg;
        }
    }
    Win<R> ph = {vph[0][0], vph[0][1], vph[0][2], vph[1][0], vph[1][1], vph[1][2],
                 vph[2][0], vph[2][1], vph[2][2]};
    Win<R> ps = {vps[0][0], vps[0][1], vps[0][2], vps[1][0], vps[1][1], vps[1][2],
                 vps[2][0], vps[2][1], vps[2][2]};
    const S* b = state + (long long)y * G.pitch + x;
    R gq[9];
    for (int a = 0; a < 9; ++a) gq[a] = load_pop<S, R>(b + a * G.plane);
    const R jgx = (gq[1] - gq[3]) + (gq[5] - gq[6]) - (gq[7] - gq[8]);
    const R jgy = (gq[2] - gq[4]) + (gq[5] + gq[6]) - (gq[7] + gq[8]);
    Macro<R> m;
    node_macro<R>(ph, ps, jgx, jgy, R(x), R(y), K, m);
    if (phi_o) phi_o[n] = double(ph.c);
    if (p_o) p_o[n] = double(m.p);
    if (ux_o) ux_o[n] = double(m.ux);
    if (uy_o) uy_o[n] = double(m.uy);
    if (rho_o) rho_o[n] = double(m.rho);
}

// Copy between the padded device state and a dense [18][ny][nx] double array.
template <typename S>
__global__ void pack_kernel(const S* __restrict__ state, double* __restrict__ out, Geometry G)
{
    const long long N = (long long)G.nx * G.ny;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 18 * N) return;
    const long long a = t / N, n = t % N;
    const int y = (int)(n / G.nx), x = (int)(n % G.nx);
    out[t] = double(state[a * G.plane + (long long)y * G.pitch + x]);
}

template <typename S>
__global__ void unpack_kernel(const double* __restrict__ in, S* __restrict__ state, Geometry G)
{
    const long long N = (long long)G.nx * G.ny;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 18 * N) return;
    const long long a = t / N, n = t % N;
    const int y = (int)(n / G.nx), x = (int)(n % G.nx);
    state[a * G.plane + (long long)y * G.pitch + x] = static_cast<S>(in[t]);
}

// ---------------------------------------------------------------------------------------------
// Host-side launchers (called from lbm_api.cu)
// ---------------------------------------------------------------------------------------------
template <typename R, typename S>
cudaError_t launch_step(const void* src, void* dst, const Geometry& G, const Consts<R>& K,
                        int seg_h, int block, cudaStream_t st)
{
    StepLaunch L;
    L.seg_h = seg_h;
    L.nstrips = (G.nx + 31) / 32;
    L.nseg = (G.ny + seg_h - 1) / seg_h;
    const long long warps = (long long)L.nstrips * L.nseg;
    const int wpb = block / 32;
    const long long grid = (warps + wpb - 1) / wpb;
    step_kernel<R, S><<<(unsigned)grid, block, 0, st>>>(static_cast<const S*>(src),
                                                        static_cast<S*>(dst), G, K, L);
    return cudaGetLastError();
}

template <typename R, typename S>
cudaError_t launch_init(const double* phi, const double* p, const double* ux, const double* uy,
                        void* state, const Geometry& G, const Consts<R>& K, cudaStream_t st)
{
    const long long N = (long long)G.nx * G.ny;
    init_kernel<R, S><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(phi, p, ux, uy,
                                                                  static_cast<S*>(state), G, K);
    return cudaGetLastError();
}

template <typename R, typename S>
cudaError_t launch_fields(const void* state, const Geometry& G, const Consts<R>& K,
                          double* phi, double* p, double* ux, double* uy, double* rho,
                          cudaStream_t st)
{
    const long long N = (long long)G.nx * G.ny;
    fields_kernel<R, S><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(
        static_cast<const S*>(state), G, K, phi, p, ux, uy, rho);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_pack(const void* state, double* out, const Geometry& G, cudaStream_t st)
{
    const long long T = 18LL * G.nx * G.ny;
    pack_kernel<S><<<(unsigned)((T + 255) / 256), 256, 0, st>>>(static_cast<const S*>(state),
                                                               out, G);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_unpack(const double* in, void* state, const Geometry& G, cudaStream_t st)
{
    const long long T = 18LL * G.nx * G.ny;
    unpack_kernel<S><<<(unsigned)((T + 255) / 256), 256, 0, st>>>(in, static_cast<S*>(state), G);
    return cudaGetLastError();
}

template cudaError_t launch_step<double, double>(const void*, void*, const Geometry&,
                                                 const Consts<double>&, int, int, cudaStream_t);
template cudaError_t launch_step<float, float>(const void*, void*, const Geometry&,
                                               const Consts<float>&, int, int, cudaStream_t);
template cudaError_t launch_init<double, double>(const double*, const double*, const double*,
                                                 const double*, void*, const Geometry&,
                                                 const Consts<double>&, cudaStream_t);
template cudaError_t launch_init<float, float>(const double*, const double*, const double*,
                                               const double*, void*, const Geometry&,
                                               const Consts<float>&, cudaStream_t);
template cudaError_t launch_fields<double, double>(const void*, const Geometry&,
                                                   const Consts<double>&, double*, double*,
                                                   double*, double*, double*, cudaStream_t);
template cudaError_t launch_fields<float, float>(const void*, const Geometry&,
                                                 const Consts<float>&, double*, double*,
                                                 double*, double*, double*, cudaStream_t);
template cudaError_t launch_pack<double>(const void*, double*, const Geometry&, cudaStream_t);
template cudaError_t launch_pack<float>(const void*, double*, const Geometry&, cudaStream_t);
template cudaError_t launch_unpack<double>(const double*, void*, const Geometry&, cudaStream_t);
template cudaError_t launch_unpack<float>(const double*, void*, const Geometry&, cudaStream_t);

}  // namespace cmlbm
