// Fused time-step kernel, equilibrium initialisation and field extraction for the coupled
// cascaded central-moment LB schemes of arXiv:1909.04166 on sm_103a.
//
// State layout ("tiled SoA"): for every row y and every strip of 32 columns, the 18 planes
// (9 fluid g-bar, then 9 interface f) of those 32 nodes are contiguous: element (a, x, y) sits
// at ((y * nstrips + x / 32) * 18 + a) * 32 + x % 32.  One warp-row tile is 18 * 32 elements
// (2304 bytes in FP32), a single contiguous block.  The 16-bit forms prefix each tile with two
// FP32 planes of zeroth moments (see lbm_device.cuh).
//
// Step kernel (one launch = one time step of both lattices over the whole grid):
//   * Each warp owns a strip of columns and a segment of rows and marches along the rows.  With
//     FP32 arithmetic (march2) the strip is two adjacent tiles and lane l owns the two adjacent
//     columns x0 + 32 (l / 16) + 2 (l % 16) and the next one, updated together on the packed
//     FP32x2 instructions (one 64- or 32-bit shared load brings a plane's pair; in full strips
//     without walls FP32 pairs are stored as aligned 64-bit words); in FP64 (march) the strip is
//     one tile and lane l owns column x0 + l.  Segments alternate direction so that
//     neighbours read a shared boundary row at about the same time and the re-read hits L2;
//     every segment also reverses its direction from one step to the next, so that a step
//     starts on the rows the previous one wrote last, many of which are still in L2.
//   * The tiles of a row are staged in shared memory by bulk asynchronous copies
//     (cp.async.bulk, completion on an mbarrier), S stages deep: while row i is collided,
//     rows i+2 .. i+S-1 are in flight.
//   * phi = sum f and p* = sum g-bar form a rolling 3x3 window in registers: east/west
//     neighbours by warp shuffles; the two halo columns of the strip by one load per lane
//     (lanes 0..8 read the g-bar planes, 16..24 the f planes) and a half-warp reduction,
//     prefetched one row ahead.
//   * Row y is updated once its upper and lower rows' (phi, p*) are known: stencils, forces,
//     corrected p and u, both cascaded collisions in registers, then the 18 post-collision
//     populations are pushed to x + e_a in the other buffer (half-way bounce-back or specular
//     reflection at walls).  The state therefore always holds streamed (pre-collision)
//     populations.
//   * Every mbarrier wait is bounded; on timeout the warp records an error code, waits (again
//     bounded) for its copies in flight and returns.
//   * Kernels: step_kernel (FP32 / FP64 storage), step_kernel_narrow (16-bit storage, held to
//     168 registers), step_kernel_checked (every global access range-checked, for debugging),
//     batch_step_kernel / batch_step_kernel_narrow (many grids per launch).
#include "lbm_device.cuh"

#include <type_traits>

namespace cmlbm {

static constexpr unsigned FULL = 0xffffffffu;
static constexpr int TILE = 18 * 32;               // elements per warp-row tile
static constexpr unsigned WAIT_LIMIT = 1u << 22;   // bounded mbarrier polling (iterations)
// and in time: a row copy arrives within microseconds, so two seconds of the global timer
// without it means it never will
static constexpr unsigned long long WAIT_NS = 2000000000ull;

struct StepLaunch {
    int seg_h;     // rows per segment
    int nseg;      // ceil(ny / seg_h)
    int* err;      // device error word (0 = ok)
    int flow_sign; // imposed flow: +1, or -1 once reversed
    int flip;      // 0 / 1 on alternate steps: reverses the march direction of every segment
    long long chk_shrink;   // checked kernel only: elements left out of the declared buffer ends
    int cut_first_wait;     // 1: the first mbarrier wait of every warp gives up at once (tests
                            // of the timeout path); the drain of copies in flight keeps its limit
};

// March direction parity of a step: the two state buffers alternate as source, so consecutive
// steps march in opposite directions.
__host__ __device__ inline int flip_of(const void* src, const void* dst)
{
    return reinterpret_cast<uintptr_t>(src) > reinterpret_cast<uintptr_t>(dst) ? 1 : 0;
}

// Step variants: bit 0 single relaxation time (Sec. 7) instead of the cascaded rates; bit 1 the
// interface lattice alone in the imposed shear flow (Sec. 6.1); bit 2 the Langmuir isotherm
// (Sec. 6.7) instead of the linear sigma(T).
enum : int { kVarSRT = 1, kVarShear = 2, kVarLangmuir = 4 };

template <typename S> struct Stages { static constexpr int value = 4; };
template <> struct Stages<double> { static constexpr int value = 3; };

// Per-warp shared memory: the stage tiles (NT adjacent tiles per stage), then one mbarrier per
// stage; 128-byte multiple so that every warp's tiles stay 16-byte aligned for the bulk copies.
template <typename S, int NT = 1>
__host__ __device__ constexpr int warp_smem_bytes()
{
    return (Stages<S>::value * (NT * Tile<S>::BYTES + 8) + 127) / 128 * 128;
}

// ---------------------------------------------------------------------------------------------
// mbarrier / bulk-copy primitives (inline PTX)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// Invalidate an mbarrier whose phases have all completed, so that its memory may be initialised
// again (the multi-step kernel re-initialises the ring's barriers at every step).
__device__ __forceinline__ void mbar_inval(uint32_t bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Warp-collective bounded wait for phase `parity` of barrier `bar`; false on timeout (after
// WAIT_NS of the global timer, or WAIT_LIMIT polls should the timer not advance).  The timer is
// read only once the first poll has failed, every 64 polls, by lane 0 for the warp.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity)
{
    if (__all_sync(FULL, mbar_try_wait(bar, parity))) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1; it < WAIT_LIMIT; ++it) {
        if (__all_sync(FULL, mbar_try_wait(bar, parity))) return true;
        if ((it & 63) == 0) {
            int late = 0;
            if ((threadIdx.x & 31) == 0) late = global_ns() - t0 > WAIT_NS ? 1 : 0;
            if (__shfl_sync(FULL, late, 0)) return false;
        }
    }
    return false;
}

// A halo load: through the read-only cache, or (COH) through L2 only, for data that other SMs
// wrote earlier in the same launch.
template <bool COH, typename T>
__device__ __forceinline__ T ld_halo(const T* p)
{
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}

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

__device__ __forceinline__ int map_col(int x, const Geometry& G)
{
    if (x < 0) return G.wall_x ? 0 : x + G.nx;
    if (x >= G.nx) return G.wall_x ? G.nx - 1 : x - G.nx;
    return x;
}

// Element offset of column x (population plane 0) within a row of tiles.
template <typename S = float>
__device__ __forceinline__ int col_off(int x)
{
    return (x >> 5) * Tile<S>::ELEMS + Tile<S>::P0 + (x & 31);
}
// 16-bit forms: element offset of column x's value in the Z_g plane (Z_f follows 64 elements on).
template <typename S>
__device__ __forceinline__ int z_off(int x) { return (x >> 5) * Tile<S>::ELEMS + 2 * (x & 31); }

// One (phi, p*) row of the window for this lane: own column, west and east neighbours.
template <typename R>
struct Row3 {
    R phw, phc, phe, psw, psc, pse;
};

// Sum the lane's column of a staged tile and assemble its window row; hl/hr are this lane's
// halo loads (one plane of the left / right halo column, or 0).  PHI_ONLY: p* is not formed.
template <typename R, typename S, bool PHI_ONLY = false>
__device__ __forceinline__ void window_row(const S* tile, int lane, int wlast, R hl, R hr,
                                           const Consts<R>& K, Row3<R>& row)
{
    R ps = R(0), ph = R(0);
    const S* q = tile + Tile<S>::P0 + lane;
    if constexpr (Narrow<S>::value) {       // Z + (sum of the deviations) / s
        const float* z = reinterpret_cast<const float*>(tile);
        float dg = 0.0f, df = 0.0f;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            dg += narrow_to_f(q[a * 32]);
            df += narrow_to_f(q[(9 + a) * 32]);
        }
        ps = fmad(R(dg), K.st_inv[0], R(z[lane]));
        ph = fmad(R(df), K.st_inv[1], R(z[32 + lane]));
    } else {
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            if (!PHI_ONLY) ps += R(q[a * 32]);
            ph += R(q[(9 + a) * 32]);
        }
    }
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
        hl += __shfl_xor_sync(FULL, hl, off);
        hr += __shfl_xor_sync(FULL, hr, off);
    }
    const R psl = __shfl_sync(FULL, hl, 0), phl = __shfl_sync(FULL, hl, 16);
    const R psr = __shfl_sync(FULL, hr, 0), phr = __shfl_sync(FULL, hr, 16);
    row.phc = ph;
    row.psc = ps;
    row.phw = shfl_up(ph);
    row.psw = shfl_up(ps);
    row.phe = shfl_dn(ph);
    row.pse = shfl_dn(ps);
    if (lane == 0) { row.phw = phl; row.psw = psl; }
    if (lane == wlast) { row.phe = phr; row.pse = psr; }
}

template <typename R>
__device__ __forceinline__ void make_window(const Row3<R>& s, const Row3<R>& c,
                                            const Row3<R>& n, Win<R>& ph, Win<R>& ps)
{
    ph.sw = s.phw; ph.s = s.phc; ph.se = s.phe;
    ph.w = c.phw;  ph.c = c.phc; ph.e = c.phe;
    ph.nw = n.phw; ph.n = n.phc; ph.ne = n.phe;
    ps.sw = s.psw; ps.s = s.psc; ps.se = s.pse;
    ps.w = c.psw;  ps.c = c.psc; ps.e = c.pse;
    ps.nw = n.psw; ps.n = n.psc; ps.ne = n.pse;
}

template <typename S, typename R, bool F_ONLY = false>
__device__ __forceinline__ void ld_pops_t(const S* tile, int lane, const Consts<R>& K, R g[9],
                                          R f[9])
{
    R zg = R(0), zf = R(0);
    if constexpr (Narrow<S>::value) {
        const float* z = reinterpret_cast<const float*>(tile);
        zg = R(z[lane]);
        zf = R(z[32 + lane]);
    }
    const S* q = tile + Tile<S>::P0 + lane;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        if (!F_ONLY) g[a] = decode<S, R>(q[a * 32], zg, 0, a, K);
        f[a] = decode<S, R>(q[(9 + a) * 32], zf, 1, a, K);
    }
}

// Range checks of a step's global accesses, for the bounds-checked step kernel: halo loads and
// bulk copies must lie inside the source state buffer, stores inside the destination buffer.
// An access outside is skipped and bit 1 of the error word is set.  The plain kernels use
// Bounds<false>, whose checks are constant true and compile to nothing.
template <bool ON>
struct Bounds {
    __device__ __forceinline__ bool rd(const void*, unsigned) const { return true; }
    __device__ __forceinline__ bool wr(const void*, unsigned) const { return true; }
};
template <>
struct Bounds<true> {
    uintptr_t src_lo, src_hi, dst_lo, dst_hi;
    int* err;
    __device__ __forceinline__ bool in(const void* p, unsigned n, uintptr_t lo,
                                       uintptr_t hi) const
    {
        const uintptr_t q = reinterpret_cast<uintptr_t>(p);
        if (q >= lo && q <= hi && n <= hi - q) return true;
        atomicOr(err, 2);
        return false;
    }
    __device__ __forceinline__ bool rd(const void* p, unsigned n) const
    {
        return in(p, n, src_lo, src_hi);
    }
    __device__ __forceinline__ bool wr(const void* p, unsigned n) const
    {
        return in(p, n, dst_lo, dst_hi);
    }
};
template <bool CK, typename S>
__device__ __forceinline__ Bounds<CK> make_bounds(const S* src, const S* dst, long long elems,
                                                  int* err)
{
    if constexpr (CK) {
        return Bounds<true>{reinterpret_cast<uintptr_t>(src),
                            reinterpret_cast<uintptr_t>(src + elems),
                            reinterpret_cast<uintptr_t>(dst),
                            reinterpret_cast<uintptr_t>(dst + elems), err};
    } else {
        return Bounds<false>{};
    }
}
// Store through a bounds check.
template <class BND, typename T>
__device__ __forceinline__ void st_chk(const BND& B, T* p, T v)
{
    if (B.wr(p, sizeof(T))) *p = v;
}

// Value of a window at offset (dx, dy) in {-1, 0, 1}^2.
template <typename R>
__device__ __forceinline__ R win_at(const Win<R>& w, int dx, int dy)
{
    const R s = dx < 0 ? w.sw : (dx > 0 ? w.se : w.s);
    const R c = dx < 0 ? w.w : (dx > 0 ? w.e : w.c);
    const R n = dx < 0 ? w.nw : (dx > 0 ? w.ne : w.n);
    return dy < 0 ? s : (dy > 0 ? n : c);
}

// Push the 18 post-collision populations of one node to x + e_a in the row buffers rS, rC, rN
// (rows y - 1, y, y + 1) at the column offsets cw, cc, ce (columns x - 1, x, x + 1).  fast:
// warp-uniform, no wall is crossed by any node of this warp row.  Otherwise a population crossing
// a no-slip wall returns to this node reversed (half-way bounce-back); one crossing only free-slip
// walls has its normal components reversed and stays on this side of them (specular reflection).
// bxw / bxe / bys / byn: the node lies next to the west / east / south / north wall.
template <typename S, typename R, bool F_ONLY, class BND = Bounds<false>>
__device__ __forceinline__ void push_node(const R g[9], const R f[9], S* rS, S* rC, S* rN, int cw,
                                          int cc, int ce, bool bxw, bool bxe, bool bys,
                                          bool byn, int slip, bool fast, const Consts<R>& K,
                                          const BND& B = BND())
{
    S* pc = rC + cc;
    S* p[9] = {pc, rC + ce, rN + cc, rC + cw, rS + cc, rN + ce, rN + cw, rS + cw, rS + ce};
    if (fast) {
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            if (!F_ONLY) st_chk(B, &p[a][a * 32], static_cast<S>(g[a]));
            st_chk(B, &p[a][(9 + a) * 32], static_cast<S>(f[a]));
        }
        return;
    }
    constexpr int EXc[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int EYc[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    constexpr int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    constexpr int MX[9] = {0, 3, 2, 1, 4, 6, 5, 8, 7};    // e_x reversed
    constexpr int MY[9] = {0, 1, 4, 3, 2, 8, 7, 6, 5};    // e_y reversed
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const int ex = EXc[a], ey = EYc[a];
        const bool cx = (ex < 0 && bxw) || (ex > 0 && bxe);
        const bool cy = (ey < 0 && bys) || (ey > 0 && byn);
        const bool sx = ((slip >> (ex < 0 ? 0 : 1)) & 1) != 0;
        const bool sy = ((slip >> (ey < 0 ? 2 : 3)) & 1) != 0;
        int plane = a;
        S* q = p[a];
        if ((cx && !sx) || (cy && !sy)) {
            plane = OPP[a];
            q = pc;
        } else if (cx || cy) {
            plane = cx ? (cy ? OPP[a] : MX[a]) : MY[a];
            S* row = cy ? rC : (ey > 0 ? rN : (ey < 0 ? rS : rC));
            q = row + (cx ? cc : (ex > 0 ? ce : (ex < 0 ? cw : cc)));
        }
        if (!F_ONLY) st_chk(B, &q[plane * 32], static_cast<S>(g[a]));
        st_chk(B, &q[(9 + plane) * 32], static_cast<S>(f[a]));
    }
}

// Rounding compensation of the 16-bit forms.  Each node stores its eight moving populations
// first and keeps the sum of their rounding errors (stored minus exact scaled deviation; the
// difference of a value and its 16-bit rounding is exact in FP32); its rest population, which
// lands on the node itself, is stored with that sum subtracted.  The stored populations a node
// sends out then sum to what it computed up to one 16-bit rounding of the rest population's
// deviation, which is small (the rest state carries no flux), so the lattice sums (the phase
// mass of the interface lattice) no longer drift with the rounding of every population.
//
// Stored value of a population that lands on a node with zeroth moment z: its scaled deviation
// (v - w z) s, less adj when ADJ; err receives the stored value's rounding error, scaled.
template <typename S, bool ADJ, typename R>
__device__ __forceinline__ S encode_err(R v, R z, R w, R scale, R adj, R& err)
{
    R d = fmad(-w, z, v) * scale;
    if constexpr (ADJ) d = d - adj;
    const S h = f_to_narrow<S>(float(d));
    err = R(narrow_to_f(h)) - d;
    return h;
}

// As push_node for the 16-bit forms: every population is stored as its deviation from the rest
// state of the node it lands on, whose zeroth moments are the window values ps (p*) and ph (phi)
// at the landing offset; the node's own zeroth moments go to its Z planes (element offset zc).
// The rest population goes last and takes up the rounding of the others (see encode_err).
template <typename S, typename R, class BND = Bounds<false>>
__device__ __forceinline__ void push_node_z(const R g[9], const R f[9], const Win<R>& ps,
                                            const Win<R>& ph, S* rS, S* rC, S* rN, int cw,
                                            int cc, int ce, int zc, bool bxw, bool bxe,
                                            bool bys, bool byn, int slip, bool fast,
                                            const Consts<R>& K, const BND& B = BND())
{
    float* zp = reinterpret_cast<float*>(rC + zc);
    st_chk(B, &zp[0], float(ps.c));
    st_chk(B, &zp[32], float(ph.c));
    S* pc = rC + cc;
    S* p[9] = {pc, rC + ce, rN + cc, rC + cw, rS + cc, rN + ce, rN + cw, rS + cw, rS + ce};
    constexpr int EXc[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int EYc[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const R sg = K.st_scale[0], sf = K.st_scale[1];
    R eg = R(0), ef = R(0), e;
    if (fast) {
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            const R w = R(d2q9_w(a));
            st_chk(B, &p[a][a * 32],
                   encode_err<S, false>(g[a], win_at(ps, EXc[a], EYc[a]), w, sg, R(0), e));
            eg += e;
            st_chk(B, &p[a][(9 + a) * 32],
                   encode_err<S, false>(f[a], win_at(ph, EXc[a], EYc[a]), w, sf, R(0), e));
            ef += e;
        }
        st_chk(B, &pc[0], encode_err<S, true>(g[0], ps.c, R(d2q9_w(0)), sg, eg, e));
        st_chk(B, &pc[9 * 32], encode_err<S, true>(f[0], ph.c, R(d2q9_w(0)), sf, ef, e));
        return;
    }
    constexpr int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    constexpr int MX[9] = {0, 3, 2, 1, 4, 6, 5, 8, 7};
    constexpr int MY[9] = {0, 1, 4, 3, 2, 8, 7, 6, 5};
#pragma unroll
    for (int a = 1; a < 9; ++a) {
        const int ex = EXc[a], ey = EYc[a];
        const bool cx = (ex < 0 && bxw) || (ex > 0 && bxe);
        const bool cy = (ey < 0 && bys) || (ey > 0 && byn);
        const bool sx = ((slip >> (ex < 0 ? 0 : 1)) & 1) != 0;
        const bool sy = ((slip >> (ey < 0 ? 2 : 3)) & 1) != 0;
        // landing node: x + e_a, or this node (bounce-back, or both components reflected), or
        // the tangential neighbour (one component reflected); its zeroth moments are window
        // values at constant offsets, chosen by selects
        const bool bounce = (cx && !sx) || (cy && !sy) || (cx && cy);
        int plane = a;
        S* q = p[a];
        R zg = win_at(ps, ex, ey), zf = win_at(ph, ex, ey);
        if (bounce) {
            plane = OPP[a];
            q = pc;
            zg = ps.c;
            zf = ph.c;
        } else if (cx) {
            plane = MX[a];
            q = (ey > 0 ? rN : (ey < 0 ? rS : rC)) + cc;
            zg = win_at(ps, 0, ey);
            zf = win_at(ph, 0, ey);
        } else if (cy) {
            plane = MY[a];
            q = rC + (ex > 0 ? ce : (ex < 0 ? cw : cc));
            zg = win_at(ps, ex, 0);
            zf = win_at(ph, ex, 0);
        }
        const R w = R(d2q9_w(a));
        st_chk(B, &q[plane * 32], encode_err<S, false>(g[a], zg, w, sg, R(0), e));
        eg += e;
        st_chk(B, &q[(9 + plane) * 32], encode_err<S, false>(f[a], zf, w, sf, R(0), e));
        ef += e;
    }
    st_chk(B, &pc[0], encode_err<S, true>(g[0], ps.c, R(d2q9_w(0)), sg, eg, e));
    st_chk(B, &pc[9 * 32], encode_err<S, true>(f[0], ph.c, R(d2q9_w(0)), sf, ef, e));
}

// Stored values of population a for a lane's two nodes at once (the packed form of
// encode_err): d = (v - w_a z) s (less adj when ADJ) for both halves with FFMA2 / FMUL2, rounded
// to 16 bits by one paired conversion; returns the pair's scaled rounding errors.  Same
// roundings as encode_err, element by element.
template <typename S, bool ADJ>
__device__ __forceinline__ F2 encode_pair(F2 v, F2 z, float w, float scale, F2 adj, S& lo,
                                          S& hi)
{
    F2 d = fmad(F2(-w), z, v) * F2(scale);
    if constexpr (ADJ) d = d - adj;
    float2 back;
    if constexpr (std::is_same<S, __half>::value) {
        const __half2 h = __float22half2_rn(d.v);
        lo = __low2half(h);
        hi = __high2half(h);
        back = __half22float2(h);
    } else {
        const __nv_bfloat162 h = __float22bfloat162_rn(d.v);
        lo = __low2bfloat16(h);
        hi = __high2bfloat16(h);
        back = __bfloat1622float2(h);
    }
    return F2(back) - d;
}

// push_node_z for both nodes of a lane when no node of the warp row touches a wall (the fast
// path): encodes each population pair once, then stores node A's value if A is active and
// node B's if B is.  c*A / c*B: column offsets of x - 1, x, x + 1 for the two nodes.
template <typename S, class BND = Bounds<false>>
__device__ __forceinline__ void push_pair_z(const F2 g[9], const F2 f[9], const Win<F2>& ps,
                                            const Win<F2>& ph, S* rS, S* rC, S* rN, int cwA,
                                            int ccA, int ceA, int cwB, int ccB, int ceB,
                                            int zcA, int zcB, bool actA, bool actB,
                                            const Consts<float>& K, const BND& B = BND())
{
    if (actA) {
        float* z = reinterpret_cast<float*>(rC + zcA);
        st_chk(B, &z[0], ps.c.v.x);
        st_chk(B, &z[32], ph.c.v.x);
    }
    if (actB) {
        float* z = reinterpret_cast<float*>(rC + zcB);
        st_chk(B, &z[0], ps.c.v.y);
        st_chk(B, &z[32], ph.c.v.y);
    }
    S* pA[9] = {rC + ccA, rC + ceA, rN + ccA, rC + cwA, rS + ccA, rN + ceA, rN + cwA, rS + cwA,
                rS + ceA};
    S* pB[9] = {rC + ccB, rC + ceB, rN + ccB, rC + cwB, rS + ccB, rN + ceB, rN + cwB, rS + cwB,
                rS + ceB};
    constexpr int EXc[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int EYc[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    F2 eg(0.0f), ef(0.0f);   // rounding errors of the moving populations (see encode_err)
    auto put = [&](int a, S gA, S gB, S fA, S fB) {
        if (actA) {
            st_chk(B, &pA[a][a * 32], gA);
            st_chk(B, &pA[a][(9 + a) * 32], fA);
        }
        if (actB) {
            st_chk(B, &pB[a][a * 32], gB);
            st_chk(B, &pB[a][(9 + a) * 32], fB);
        }
    };
#pragma unroll
    for (int a = 1; a < 9; ++a) {
        const float w = float(d2q9_w(a));
        S gA, gB, fA, fB;
        eg += encode_pair<S, false>(g[a], win_at(ps, EXc[a], EYc[a]), w, K.st_scale[0],
                                    F2(0.0f), gA, gB);
        ef += encode_pair<S, false>(f[a], win_at(ph, EXc[a], EYc[a]), w, K.st_scale[1],
                                    F2(0.0f), fA, fB);
        put(a, gA, gB, fA, fB);
    }
    S gA, gB, fA, fB;
    const float w0 = float(d2q9_w(0));
    encode_pair<S, true>(g[0], ps.c, w0, K.st_scale[0], eg, gA, gB);
    encode_pair<S, true>(f[0], ph.c, w0, K.st_scale[1], ef, fA, fB);
    put(0, gA, gB, fA, fB);
}

// Global store executed only where p holds, as one predicated instruction (no branch): the FP32
// pair and edge stores of the packed fast path are taken by all but one or two lanes of a warp.
// The bounds-checked kernel keeps its checked, branching form.
__device__ __forceinline__ void st_global_if(bool p, float2* a, float2 v)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t"
                 "@q st.global.v2.f32 [%1], {%2, %3};\n\t}" ::"r"((int)p), "l"(a), "f"(v.x),
                 "f"(v.y));
}
__device__ __forceinline__ void st_global_if(bool p, float* a, float v)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t"
                 "@q st.global.f32 [%1], %2;\n\t}" ::"r"((int)p), "l"(a), "f"(v));
}
template <class BND, typename T>
__device__ __forceinline__ void st_chk_if(const BND& B, bool p, T* a, T v)
{
    if constexpr (std::is_same<BND, Bounds<false>>::value) st_global_if(p, a, v);
    else if (p) st_chk(B, a, v);
}

// The packed form of encode_pair: the two stored 16-bit values as one 32-bit word (node A in the
// low half, node B in the high half); same roundings, same returned errors.
template <typename S, bool ADJ>
__device__ __forceinline__ F2 encode_word(F2 v, F2 z, float w, float scale, F2 adj,
                                          uint32_t& word)
{
    F2 d = fmad(F2(-w), z, v) * F2(scale);
    if constexpr (ADJ) d = d - adj;
    float2 back;
    if constexpr (std::is_same<S, __half>::value) {
        const __half2 h = __float22half2_rn(d.v);
        word = *reinterpret_cast<const uint32_t*>(&h);
        back = __half22float2(h);
    } else {
        const __nv_bfloat162 h = __float22bfloat162_rn(d.v);
        word = *reinterpret_cast<const uint32_t*>(&h);
        back = __bfloat1622float2(h);
    }
    return F2(back) - d;
}

// Stores of the fast path for a full strip (64 active columns, no wall in the warp row).  FP32:
// for every population plane one store writes a whole aligned pair of adjacent columns for most
// lanes.  With e_x = 0 a lane writes its own pair; with e_x = +1 the pair (c_A, c_B) receives the
// previous lane's B and this lane's A (one shuffle), lane 0 writing only its B half and lane 31
// sending its B into the next strip (column offset ceB); with e_x = -1 it receives this lane's B
// and the next lane's A, lane 31 writing only its A half and lane 0 sending its A into the
// previous strip (cwA).  16-bit forms: one 32-bit store of the lane's pair for the planes with
// e_x = 0 and one 16-bit store per node for the others (measured faster there than shuffled
// pairs); every population is encoded against the rest state of the node it lands on (the window
// values at its offset), and the rest population goes last with the rounding errors of the
// moving ones subtracted (see encode_err).  woff / zoff: element offsets of column c_A's plane 0
// and zeroth moments; ccB: column c_B's.  The stored values are those of push_node / push_pair_z,
// bit for bit.
template <typename S, bool F_ONLY, class BND>
__device__ __forceinline__ void push_packed(const F2 g[9], const F2 f[9], const Win<F2>& ps,
                                            const Win<F2>& ph, S* rS, S* rC, S* rN, int woff,
                                            int ccB, int cwA, int ceB, int zoff, int lane,
                                            const Consts<float>& K, const BND& B)
{
    constexpr bool NARROW = Narrow<S>::value;
    constexpr int EXc[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int EYc[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    auto row_at = [&](int ey) { return ey < 0 ? rS : (ey > 0 ? rN : rC); };
    if constexpr (NARROW) {
        // plane `plane` of the pair word `mine` (node A low half, B high half), moving by ex
        auto put = [&](S* row, int plane, int ex, uint32_t mine) {
            S* base = row + plane * 32;
            if (ex == 0) {
                st_chk(B, reinterpret_cast<uint32_t*>(base + woff), mine);
                return;
            }
            auto* pa = reinterpret_cast<unsigned short*>(base + (ex > 0 ? ccB : cwA));
            auto* pb = reinterpret_cast<unsigned short*>(base + (ex > 0 ? ceB : woff));
            st_chk(B, pa, static_cast<unsigned short>(mine & 0xffffu));
            st_chk(B, pb, static_cast<unsigned short>(mine >> 16));
        };
        float* z = reinterpret_cast<float*>(rC + zoff);
        st_chk(B, reinterpret_cast<float2*>(z), ps.c.v);
        st_chk(B, reinterpret_cast<float2*>(z + 32), ph.c.v);
        F2 eg(0.0f), ef(0.0f);   // rounding errors of the moving populations (see encode_err)
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            const float w = float(d2q9_w(a));
            uint32_t wg, wf;
            eg += encode_word<S, false>(g[a], win_at(ps, EXc[a], EYc[a]), w, K.st_scale[0],
                                        F2(0.0f), wg);
            ef += encode_word<S, false>(f[a], win_at(ph, EXc[a], EYc[a]), w, K.st_scale[1],
                                        F2(0.0f), wf);
            put(row_at(EYc[a]), a, EXc[a], wg);
            put(row_at(EYc[a]), 9 + a, EXc[a], wf);
        }
        const float w0 = float(d2q9_w(0));
        uint32_t wg, wf;
        encode_word<S, true>(g[0], ps.c, w0, K.st_scale[0], eg, wg);
        encode_word<S, true>(f[0], ph.c, w0, K.st_scale[1], ef, wf);
        put(rC, 0, 0, wg);
        put(rC, 9, 0, wf);
    } else {
        // the edge stores: lane 0 writes its A, lane 31 its B, at these element offsets for
        // e_x = +1 / -1
        const int eoff_p = lane == 0 ? woff + 1 : ceB;
        const int eoff_m = lane == 31 ? woff : cwA;
        const bool edge = lane == 0 || lane == 31;
        auto put = [&](S* row, int plane, int ex, float2 mine) {
            S* base = row + plane * 32;
            float2* wp = reinterpret_cast<float2*>(base + woff);
            if (ex == 0) {
                st_chk(B, wp, mine);
                return;
            }
            if (ex > 0)   // (previous lane's B, this A)
                st_chk_if(B, lane >= 1, wp,
                          make_float2(__shfl_up_sync(FULL, mine.y, 1), mine.x));
            else          // (this B, next lane's A)
                st_chk_if(B, lane <= 30, wp,
                          make_float2(mine.y, __shfl_down_sync(FULL, mine.x, 1)));
            st_chk_if(B, edge, base + (ex > 0 ? eoff_p : eoff_m), lane == 0 ? mine.x : mine.y);
        };
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            if (!F_ONLY) put(row_at(EYc[a]), a, EXc[a], g[a].v);
            put(row_at(EYc[a]), 9 + a, EXc[a], f[a].v);
        }
    }
}

// The march of one warp over one strip x segment of one grid: everything the step does for
// those nodes.  Used by the single-grid kernels and by the batched kernel.  False if a wait
// timed out (the error word is set and no copy is left in flight).  COH: the halo columns are
// read through L2 only (ld.global.cg) instead of the read-only cache, as the multi-step kernel
// needs, whose source buffer was written by other SMs during the same launch.
template <typename R, typename S, int V, bool CK = false, bool COH = false>
__device__ __forceinline__ bool march(const S* __restrict__ src, S* __restrict__ dst,
                                      const Geometry& G, const Consts<R>& K, int strip, int seg,
                                      int seg_h, int* err, int flow_sign, int flip,
                                      long long chk_shrink = 0, bool cut_first = false)
{
    constexpr int NS = Stages<S>::value;
    constexpr bool SRT = (V & kVarSRT) != 0;
    constexpr bool SHEAR = (V & kVarShear) != 0;
    constexpr bool LANGMUIR = (V & kVarLangmuir) != 0;
    constexpr bool NARROW = Narrow<S>::value;
    constexpr int TE = Tile<S>::ELEMS;               // elements per tile
    const auto B =
        make_bounds<CK>(src, dst, (long long)G.ny * G.nstrips * TE - chk_shrink, err);
    // the interface lattice alone copies only the f half of every tile (planes 9..17)
    constexpr int COPY_OFF = SHEAR ? Tile<S>::P0 + 9 * 32 : 0;
    constexpr uint32_t COPY_BYTES = SHEAR ? 9 * 32 * sizeof(S) : Tile<S>::BYTES;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;

    S* tiles = reinterpret_cast<S*>(smem_raw + wib * warp_smem_bytes<S>());
    const uint32_t bar0 = smem_u32(tiles + NS * TE);
    if (lane == 0)
        for (int s = 0; s < NS; ++s) mbar_init(bar0 + 8 * s, 1);
    mbar_init_fence();
    __syncwarp();

    const int x0 = strip * 32;
    const int w = min(32, G.nx - x0);
    const int wlast = w - 1;
    const bool active = lane < w;
    const int x = active ? x0 + lane : x0 + wlast;   // idle lanes shadow the last column
    const int xl = map_col(x0 - 1, G), xr = map_col(x0 + w, G);
    const int row_elems = G.nstrips * TE;            // < 2^31 for nx <= 65536
    auto row_ptr = [&](const S* base, int row) { return base + (long long)row * row_elems; };

    const int ys = seg * seg_h;
    const int ye = min(ys + seg_h, G.ny);
    const int nrows = ye - ys;
    const bool up = ((seg + flip) & 1) == 0;
    // row visited at step k (k = -1 .. nrows): behind/current/ahead rows of the march
    auto row_of = [&](int k) { return map_row(up ? ys + k : ye - 1 - k, G); };

    // halo: lanes 0..8 load g-bar plane q, lanes 16..24 f plane q, at columns xl and xr; in
    // the 16-bit forms lanes 9 and 25 add the columns' Z_g and Z_f to the scaled deviations
    const int hq = lane & 15, hlat = lane >> 4;
    const bool hlane = hq < 9 && (!SHEAR || lane >= 16);
    const bool zlane = NARROW && hq == 9;
    const int hplane = hlat * 9 + hq;
    const int hoffl = zlane ? z_off<S>(xl) + 64 * hlat : col_off<S>(xl) + hplane * 32;
    const int hoffr = zlane ? z_off<S>(xr) + 64 * hlat : col_off<S>(xr) + hplane * 32;
    const R hinv = NARROW ? (hlat ? K.st_inv[1] : K.st_inv[0]) : R(1);
    auto halo_load = [&](int k, R& hl, R& hr) {
        hl = R(0);
        hr = R(0);
        const S* rb = row_ptr(src, row_of(k));
        if (hlane) {
            if constexpr (NARROW) {
                if (B.rd(rb + hoffl, sizeof(S))) hl = R(narrow_to_f(ld_halo<COH>(rb + hoffl))) * hinv;
                if (B.rd(rb + hoffr, sizeof(S))) hr = R(narrow_to_f(ld_halo<COH>(rb + hoffr))) * hinv;
            } else {
                if (B.rd(rb + hoffl, sizeof(S))) hl = R(ld_halo<COH>(rb + hoffl));
                if (B.rd(rb + hoffr, sizeof(S))) hr = R(ld_halo<COH>(rb + hoffr));
            }
        } else if (zlane) {
            const float* zl = reinterpret_cast<const float*>(rb + hoffl);
            const float* zr = reinterpret_cast<const float*>(rb + hoffr);
            if (B.rd(zl, sizeof(float))) hl = R(ld_halo<COH>(zl));
            if (B.rd(zr, sizeof(float))) hr = R(ld_halo<COH>(zr));
        }
    };

    // stage of row k is (k + 1) % NS; its barrier completes one phase per use, so the wait for
    // row k expects parity ((k + 1) / NS) & 1
    int issued = -2;           // highest k whose tile copy was issued
    auto issue = [&](int k, int st) {
        if (k > nrows) return;
        __syncwarp();
        if (lane == 0) {
            fence_proxy_async();
            const uint32_t bar = bar0 + 8 * st;
            const S* from = row_ptr(src, row_of(k)) + strip * TE + COPY_OFF;
            const bool okc = B.rd(from, COPY_BYTES);   // a refused copy only arrives
            mbar_expect_tx(bar, okc ? COPY_BYTES : 0u);
            if (okc) bulk_g2s(smem_u32(tiles + st * TE + COPY_OFF), from, COPY_BYTES, bar);
        }
        issued = k;
    };
    auto wait_k = [&](int k, int st) -> bool {
        return warp_wait(bar0 + 8 * st, (uint32_t)(((k + 1) / NS) & 1));
    };
    // timeout: record the error, wait (bounded) for every copy still in flight, then return
    auto fail = [&](int k_failed) {
        if (lane == 0) atomicCAS(err, 0, 1);
        for (int k = k_failed; k <= issued; ++k) wait_k(k, (k + 1) % NS);
    };

    for (int k = -1; k <= NS - 2; ++k) issue(k, (k + 1) % NS);

    Row3<R> rb, rc, rn;   // rows behind, current, ahead (in marching order)
    R hl, hr, hl2, hr2;
    halo_load(-1, hl, hr);
    if (cut_first || !wait_k(-1, 0)) { fail(-1); return false; }
    window_row<R, S, SHEAR>(tiles, lane, wlast, hl, hr, K, rb);
    issue(NS - 1, 0);
    halo_load(0, hl, hr);
    if (!wait_k(0, 1)) { fail(0); return false; }
    window_row<R, S, SHEAR>(tiles + TE, lane, wlast, hl, hr, K, rc);
    halo_load(1, hl2, hr2);

    // neighbour columns of this lane (periodic wrap; walls handled by bounce flags)
    int xm = x - 1, xp = x + 1;
    const bool bxw = xm < 0 && G.wall_x, bxe = xp >= G.nx && G.wall_x;
    if (xm < 0) xm += G.nx;
    if (xp >= G.nx) xp -= G.nx;
    const int cw = col_off<S>(xm), cc = col_off<S>(x), ce = col_off<S>(xp);
    const int zc = NARROW ? z_off<S>(x) : 0;
    const bool xwall_warp = __any_sync(FULL, bxw || bxe);
    const R xf = R(x);
    bool ok = true;
    // imposed flow: sin / cos of pi (x / L0 - 1/2) for this lane's column
    R sxl = R(0), cxl = R(0);
    if (SHEAR) sincospi_(xf * K.inv_nx - R(0.5), &sxl, &cxl);
    const R fsign = R(flow_sign);

    // one row of the march; st = stage of row i
    auto body = [&](int i, int st) {
        const int st1 = st + 1 == NS ? 0 : st + 1;       // stage of row i + 1
        if (!wait_k(i + 1, st1)) { fail(i + 1); ok = false; return; }
        window_row<R, S, SHEAR>(tiles + st1 * TE, lane, wlast, hl2, hr2, K, rn);
        if (i + 2 <= nrows) halo_load(i + 2, hl2, hr2);

        const int y = up ? ys + i : ye - 1 - i;
        Win<R> ph, ps;
        if (up) make_window(rb, rc, rn, ph, ps);
        else make_window(rn, rc, rb, ph, ps);
        R g[9], f[9];
        ld_pops_t<S, R, SHEAR>(tiles + st * TE, lane, K, g, f);
        Macro<R> m;
        if constexpr (SHEAR) {
            R syr, cyr;
            sincospi_(R(y) * K.inv_ny - R(0.5), &syr, &cyr);
            imposed_velocity<R>(sxl, cxl, syr, cyr, fsign, K, m.ux, m.uy);
            interface_flux<R>(ph, K, m.jx, m.jy);
        } else {
            const R jgx = (g[1] - g[3]) + (g[5] - g[6]) - (g[7] - g[8]);
            const R jgy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
            node_macro<R, LANGMUIR>(ph, ps, jgx, jgy, xf, R(y), K, m);
            if constexpr (SRT) collide_fluid_srt<R>(g, ps.c, m);
            else collide_fluid<R>(g, ps.c, m);
        }
        if constexpr (SRT) collide_ace_srt<R>(f, ph.c, m, K.omega_phi);
        else collide_ace<R>(f, ph.c, m, K.omega_phi);

        // push to x + e_a: rows y-1, y, y+1 and columns x-1, x, x+1 of the other buffer
        int ym = y - 1, yp = y + 1;
        const bool bys = ym < 0 && G.wall_y, byn = yp >= G.ny && G.wall_y;
        if (ym < 0) ym += G.ny;
        if (yp >= G.ny) yp -= G.ny;
        S* rS = const_cast<S*>(row_ptr(dst, ym));
        S* rC = const_cast<S*>(row_ptr(dst, y));
        S* rN = const_cast<S*>(row_ptr(dst, yp));
        if (active) {
            const bool fast = !(bys || byn) && !xwall_warp;
            if constexpr (NARROW)
                push_node_z<S, R>(g, f, ps, ph, rS, rC, rN, cw, cc, ce, zc, bxw, bxe, bys, byn,
                                  G.slip, fast, K, B);
            else
                push_node<S, R, SHEAR>(g, f, rS, rC, rN, cw, cc, ce, bxw, bxe, bys, byn,
                                       G.slip, fast, K, B);
        }
        issue(i + NS, st);      // the tile of row i is consumed: refill its stage
        rb = rc;
        rc = rn;
    };

    // a rolled loop: unrolling by the stage count makes the stages literals but the larger body
    // misses in the instruction cache (measured slower)
    for (int i = 0, st = 1; i < nrows; ++i, st = (st + 1 == NS ? 0 : st + 1)) {
        body(i, st);
        if (!ok) return false;
    }
    // every copy issued has completed (the last wait was for row nrows): release the barriers
    __syncwarp();
    if (lane == 0)
        for (int s = 0; s < NS; ++s) mbar_inval(bar0 + 8 * s);
    __syncwarp();
    return true;
}

// ---------------------------------------------------------------------------------------------
// Paired FP32 march: a warp owns two adjacent tiles (64 columns) and lane l the two adjacent
// columns c_A = 32 t + 2 j and c_B = c_A + 1 of tile t = l / 16 (j = l % 16): node A and node B.
// Both nodes go through the update at once in the packed FP32x2 arithmetic (F2), which halves the
// issued floating-point instructions per node, and the per-row work of the pipeline (waits,
// copies, halo, row addressing) is shared by 64 nodes.  A lane's two values of a population plane
// are adjacent in memory, so one 64-bit (FP32) or 32-bit (16-bit) shared load brings both, and
// where no node of the warp row touches a wall, one store per plane writes a whole aligned pair
// for most lanes (the x-shifted planes take one shuffle for that; the two pairs at the strip's
// ends are split into single stores).  One bulk copy per row brings both tiles (they are adjacent
// in memory).  An odd last strip has one tile; lanes of the missing tile read tile A again and
// store nothing.
// ---------------------------------------------------------------------------------------------
struct Row3P {
    F2 phw, phc, phe, psw, psc, pse;
};

// The two values of population plane p at a lane's pair of columns (tp: the lane's tile plus
// 2 j), converted to float.
template <typename S>
__device__ __forceinline__ F2 load_pair(const S* tp, int p)
{
    const S* q = tp + Tile<S>::P0 + p * 32;
    if constexpr (std::is_same<S, float>::value) {
        return F2(*reinterpret_cast<const float2*>(q));
    } else if constexpr (std::is_same<S, __half>::value) {
        return F2(__half22float2(*reinterpret_cast<const __half2*>(q)));
    } else {
        return F2(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(q)));
    }
}

// The zeroth moments Z (lattice lat) of a lane's two columns in a 16-bit tile (tz: the lane's
// tile; j: its pair index).
template <typename S>
__device__ __forceinline__ F2 load_z_pair(const S* tz, int j, int lat)
{
    return F2(*reinterpret_cast<const float2*>(reinterpret_cast<const float*>(tz) + 32 * lat +
                                               2 * j));
}

// Sums of a lane's two columns and their east / west neighbours; hl / hr: this lane's halo
// loads (summed over the half warp into the halo columns' zeroth moments); lastA / lastB: this
// lane's node A / B is the last active column of the warp (its east neighbour is the right halo
// column).  tt: the lane's tile in shared memory, j: its pair index.
template <typename S, bool PHI_ONLY = false>
__device__ __forceinline__ void window_row2(const S* tt, int j, int lane, bool lastA, bool lastB,
                                            float hl, float hr, const Consts<float>& K,
                                            Row3P& row)
{
    const S* tp = tt + 2 * j;
    F2 ps(0.0f), ph = load_pair(tp, 9);
    if (!PHI_ONLY) ps = load_pair(tp, 0);
#pragma unroll
    for (int a = 1; a < 9; ++a) {
        if (!PHI_ONLY) ps += load_pair(tp, a);
        ph += load_pair(tp, 9 + a);
    }
    if constexpr (Narrow<S>::value) {   // Z + (sum of the deviations) / s
        ps = fmad(ps, F2(K.st_inv[0]), load_z_pair(tt, j, 0));
        ph = fmad(ph, F2(K.st_inv[1]), load_z_pair(tt, j, 1));
    }
    F2 h(hl, hr);
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1)
        h += F2(__shfl_xor_sync(FULL, h.v.x, off), __shfl_xor_sync(FULL, h.v.y, off));
    const float psl = __shfl_sync(FULL, h.v.x, 0), phl = __shfl_sync(FULL, h.v.x, 16);
    const float psr = __shfl_sync(FULL, h.v.y, 0), phr = __shfl_sync(FULL, h.v.y, 16);
    // west of A: the previous lane's B (the left halo column for lane 0); east of A: B; west of
    // B: A; east of B: the next lane's A (the right halo column after the last active column)
    auto neighbours = [&](F2 c, float left, float right, F2& w, F2& e) {
        const float upB = __shfl_up_sync(FULL, c.v.y, 1);
        const float dnA = __shfl_down_sync(FULL, c.v.x, 1);
        w = F2(lane == 0 ? left : upB, c.v.x);
        e = F2(lastA ? right : c.v.y, lastB ? right : dnA);
    };
    row.psc = ps;
    row.phc = ph;
    neighbours(ps, psl, psr, row.psw, row.pse);
    neighbours(ph, phl, phr, row.phw, row.phe);
}

__device__ __forceinline__ void make_window2(const Row3P& s, const Row3P& c, const Row3P& n,
                                             Win<F2>& ph, Win<F2>& ps)
{
    ph.sw = s.phw; ph.s = s.phc; ph.se = s.phe;
    ph.w = c.phw;  ph.c = c.phc; ph.e = c.phe;
    ph.nw = n.phw; ph.n = n.phc; ph.ne = n.phe;
    ps.sw = s.psw; ps.s = s.psc; ps.se = s.pse;
    ps.w = c.psw;  ps.c = c.psc; ps.e = c.pse;
    ps.nw = n.psw; ps.n = n.psc; ps.ne = n.pse;
}

// One half (node A: x, node B: y) of a pair window.
__device__ __forceinline__ Win<float> half_win(const Win<F2>& w, bool b)
{
    auto h = [b](F2 v) { return b ? v.v.y : v.v.x; };
    return Win<float>{h(w.sw), h(w.s), h(w.se), h(w.w), h(w.c), h(w.e), h(w.nw), h(w.n), h(w.ne)};
}

template <typename S, int V, bool CK = false, bool COH = false>
__device__ __forceinline__ bool march2(const S* __restrict__ src, S* __restrict__ dst,
                                       const Geometry& G, const Consts<float>& K, int wstrip,
                                       int seg, int seg_h, int* err, int flow_sign, int flip,
                                       long long chk_shrink = 0, bool cut_first = false)
{
    constexpr int NS = Stages<S>::value;
    constexpr bool SRT = (V & kVarSRT) != 0;
    constexpr bool SHEAR = (V & kVarShear) != 0;
    constexpr bool LANGMUIR = (V & kVarLangmuir) != 0;
    static_assert(!(SHEAR && Narrow<S>::value), "the imposed flow runs in FP32 storage");
    constexpr bool NARROW = Narrow<S>::value;
    constexpr int TE = Tile<S>::ELEMS;               // elements per tile
    const auto B =
        make_bounds<CK>(src, dst, (long long)G.ny * G.nstrips * TE - chk_shrink, err);
    constexpr int STAGE = 2 * TE;                    // elements per stage (two tiles)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;

    S* tiles = reinterpret_cast<S*>(smem_raw + wib * warp_smem_bytes<S, 2>());
    const uint32_t bar0 = smem_u32(tiles + NS * STAGE);
    if (lane == 0)
        for (int s = 0; s < NS; ++s) mbar_init(bar0 + 8 * s, 1);
    mbar_init_fence();
    __syncwarp();

    const int t0 = 2 * wstrip;                       // first tile of the warp
    const int nt = min(2, G.nstrips - t0);           // tiles present
    const int x0 = t0 * 32;
    const int w = min(64, G.nx - x0);                // active columns
    const int wl = w - 1;                            // last active column (0..63)
    const int jp = lane & 15;                        // the lane's pair within its tile
    const int cA = 32 * (lane >> 4) + 2 * jp;        // its columns c_A and c_B = c_A + 1
    const bool actA = cA < w, actB = cA + 1 < w;
    const bool lastA = cA == wl, lastB = cA + 1 == wl;
    const int TB = (nt == 2 && lane >= 16) ? TE : 0; // offset of the lane's tile in a stage
    const int xA = actA ? x0 + cA : x0 + wl;         // idle lanes shadow the last column
    const int xB = actB ? x0 + cA + 1 : x0 + wl;
    const bool full = w == 64;                       // warp-uniform: pair stores
    const int xl = map_col(x0 - 1, G), xr = map_col(x0 + w, G);
    const int row_elems = G.nstrips * TE;
    auto row_ptr = [&](const S* base, int row) { return base + (long long)row * row_elems; };

    const int ys = seg * seg_h;
    const int ye = min(ys + seg_h, G.ny);
    const int nrows = ye - ys;
    const bool up = ((seg + flip) & 1) == 0;
    auto row_of = [&](int k) { return map_row(up ? ys + k : ye - 1 - k, G); };

    // halo: lanes 0..8 load g-bar plane q, lanes 16..24 f plane q, at columns xl and xr; in
    // the 16-bit forms lanes 9 and 25 add the columns' Z_g and Z_f to the scaled deviations
    const int hq = lane & 15, hlat = lane >> 4;
    const bool hlane = hq < 9 && (!SHEAR || hlat == 1);
    const bool zlane = NARROW && hq == 9;
    const int hplane = hlat * 9 + hq;
    const int hoffl = zlane ? z_off<S>(xl) + 64 * hlat : col_off<S>(xl) + hplane * 32;
    const int hoffr = zlane ? z_off<S>(xr) + 64 * hlat : col_off<S>(xr) + hplane * 32;
    const float hinv = NARROW ? (hlat ? K.st_inv[1] : K.st_inv[0]) : 1.0f;
    auto halo_load = [&](int k, float& hl, float& hr) {
        hl = 0.0f;
        hr = 0.0f;
        const S* rb = row_ptr(src, row_of(k));
        if (hlane) {
            if (B.rd(rb + hoffl, sizeof(S))) hl = narrow_to_f_or_self(ld_halo<COH>(rb + hoffl)) * hinv;
            if (B.rd(rb + hoffr, sizeof(S))) hr = narrow_to_f_or_self(ld_halo<COH>(rb + hoffr)) * hinv;
        } else if (zlane) {
            const float* zl = reinterpret_cast<const float*>(rb + hoffl);
            const float* zr = reinterpret_cast<const float*>(rb + hoffr);
            if (B.rd(zl, sizeof(float))) hl = ld_halo<COH>(zl);
            if (B.rd(zr, sizeof(float))) hr = ld_halo<COH>(zr);
        }
    };

    int issued = -2;
    // the interface lattice alone copies only the f half (planes 9..17) of each of the tiles
    const uint32_t copy_bytes = SHEAR ? (uint32_t)(nt * 9 * 32 * sizeof(S))
                                      : (uint32_t)(nt * Tile<S>::BYTES);
    auto issue = [&](int k, int st) {
        if (k > nrows) return;
        __syncwarp();
        if (lane == 0) {
            fence_proxy_async();
            const uint32_t bar = bar0 + 8 * st;
            const S* rowk = row_ptr(src, row_of(k)) + t0 * TE;
            if constexpr (SHEAR) {
                constexpr int FOFF = 9 * 32;
                constexpr uint32_t FB = 9 * 32 * sizeof(S);
                const bool ok0 = B.rd(rowk + FOFF, FB);   // a refused copy only arrives
                const bool ok1 = nt == 2 && B.rd(rowk + TE + FOFF, FB);
                mbar_expect_tx(bar, (ok0 ? FB : 0u) + (ok1 ? FB : 0u));
                if (ok0) bulk_g2s(smem_u32(tiles + st * STAGE + FOFF), rowk + FOFF, FB, bar);
                if (ok1)
                    bulk_g2s(smem_u32(tiles + st * STAGE + TE + FOFF), rowk + TE + FOFF, FB, bar);
            } else {
                const bool okc = B.rd(rowk, copy_bytes);
                mbar_expect_tx(bar, okc ? copy_bytes : 0u);
                if (okc) bulk_g2s(smem_u32(tiles + st * STAGE), rowk, copy_bytes, bar);
            }
        }
        issued = k;
    };
    auto wait_k = [&](int k, int st) -> bool {
        return warp_wait(bar0 + 8 * st, (uint32_t)(((k + 1) / NS) & 1));
    };
    auto fail = [&](int k_failed) {
        if (lane == 0) atomicCAS(err, 0, 1);
        for (int k = k_failed; k <= issued; ++k) wait_k(k, (k + 1) % NS);
    };

    for (int k = -1; k <= NS - 2; ++k) issue(k, (k + 1) % NS);

    Row3P rb, rc, rn;
    float hl, hr, hl2, hr2;
    halo_load(-1, hl, hr);
    if (cut_first || !wait_k(-1, 0)) { fail(-1); return false; }
    window_row2<S, SHEAR>(tiles + TB, jp, lane, lastA, lastB, hl, hr, K, rb);
    issue(NS - 1, 0);
    halo_load(0, hl, hr);
    if (!wait_k(0, 1)) { fail(0); return false; }
    window_row2<S, SHEAR>(tiles + STAGE + TB, jp, lane, lastA, lastB, hl, hr, K, rc);
    halo_load(1, hl2, hr2);

    // neighbour columns of the two nodes (periodic wrap; walls handled by the push)
    auto cols = [&](int x, int& cw, int& cc, int& ce, bool& bxw, bool& bxe) {
        int xm = x - 1, xp = x + 1;
        bxw = xm < 0 && G.wall_x;
        bxe = xp >= G.nx && G.wall_x;
        if (xm < 0) xm += G.nx;
        if (xp >= G.nx) xp -= G.nx;
        cw = col_off<S>(xm);
        cc = col_off<S>(x);
        ce = col_off<S>(xp);
    };
    int cwA, ccA, ceA, cwB, ccB, ceB;
    bool bxwA, bxeA, bxwB, bxeB;
    cols(xA, cwA, ccA, ceA, bxwA, bxeA);
    cols(xB, cwB, ccB, ceB, bxwB, bxeB);
    const int zcA = NARROW ? z_off<S>(xA) : 0, zcB = NARROW ? z_off<S>(xB) : 0;
    const bool xwall_warp = __any_sync(FULL, bxwA || bxeA || bxwB || bxeB);
    const F2 xf{static_cast<float>(xA), static_cast<float>(xB)};
    const F2 omega_phi(K.omega_phi);
    bool ok = true;
    // imposed flow: sin / cos of pi (x / L0 - 1/2) for the two columns, and the signed U_0 pi
    F2 sxl(0.0f), cxl(0.0f);
    if constexpr (SHEAR) {
        float sa, ca, sb, cb;
        sincospif(float(xA) * K.inv_nx - 0.5f, &sa, &ca);
        sincospif(float(xB) * K.inv_nx - 0.5f, &sb, &cb);
        sxl = F2(sa, sb);
        cxl = F2(ca, cb);
    }
    const float u0s = float(flow_sign) * K.u0pi;

    auto body = [&](int i, int st) {
        const int st1 = st + 1 == NS ? 0 : st + 1;
        if (!wait_k(i + 1, st1)) { fail(i + 1); ok = false; return; }
        window_row2<S, SHEAR>(tiles + st1 * STAGE + TB, jp, lane, lastA, lastB, hl2, hr2, K,
                              rn);
        if (i + 2 <= nrows) halo_load(i + 2, hl2, hr2);

        const int y = up ? ys + i : ye - 1 - i;
        Win<F2> ph, ps;
        if (up) make_window2(rb, rc, rn, ph, ps);
        else make_window2(rn, rc, rb, ph, ps);
        const S* tt = tiles + st * STAGE + TB;
        const S* tp = tt + 2 * jp;
        F2 g[9], f[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            if (!SHEAR) g[a] = load_pair(tp, a);
            f[a] = load_pair(tp, 9 + a);
        }
        if constexpr (NARROW) {   // q_a = w_a Z + d_a / s
            const F2 zg = load_z_pair(tt, jp, 0), zf = load_z_pair(tt, jp, 1);
            const F2 ig(K.st_inv[0]), ifl(K.st_inv[1]);
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const F2 wa(float(d2q9_w(a)));
                g[a] = fmad(g[a], ig, wa * zg);
                f[a] = fmad(f[a], ifl, wa * zf);
            }
        }
        Macro<F2> m;
        if constexpr (SHEAR) {
            float syr, cyr;
            sincospif(float(y) * K.inv_ny - 0.5f, &syr, &cyr);
            m.ux = F2(-u0s * syr) * cxl;
            m.uy = F2(u0s * cyr) * sxl;
            interface_flux<F2>(ph, K, m.jx, m.jy);
        } else {
            const F2 jgx = ((g[1] - g[3]) + (g[5] - g[6])) - (g[7] - g[8]);
            const F2 jgy = ((g[2] - g[4]) + (g[5] + g[6])) - (g[7] + g[8]);
            node_macro<F2, LANGMUIR>(ph, ps, jgx, jgy, xf, F2(float(y)), K, m);
            if constexpr (SRT) collide_fluid_srt<F2>(g, ps.c, m);
            else collide_fluid<F2>(g, ps.c, m);
        }
        if constexpr (SRT) collide_ace_srt<F2>(f, ph.c, m, omega_phi);
        else collide_ace<F2>(f, ph.c, m, omega_phi);

        int ym = y - 1, yp = y + 1;
        const bool bys = ym < 0 && G.wall_y, byn = yp >= G.ny && G.wall_y;
        if (ym < 0) ym += G.ny;
        if (yp >= G.ny) yp -= G.ny;
        S* rS = const_cast<S*>(row_ptr(dst, ym));
        S* rC = const_cast<S*>(row_ptr(dst, y));
        S* rN = const_cast<S*>(row_ptr(dst, yp));
        const bool fast = !(bys || byn) && !xwall_warp;
        auto push = [&](bool b, int cw, int cc, int ce, int zc, bool bxw, bool bxe) {
            float gq[9], fq[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                gq[a] = SHEAR ? 0.0f : (b ? g[a].v.y : g[a].v.x);
                fq[a] = b ? f[a].v.y : f[a].v.x;
            }
            if constexpr (NARROW)
                push_node_z<S, float>(gq, fq, half_win(ps, b), half_win(ph, b), rS, rC, rN, cw,
                                      cc, ce, zc, bxw, bxe, bys, byn, G.slip, fast, K, B);
            else
                push_node<S, float, SHEAR>(gq, fq, rS, rC, rN, cw, cc, ce, bxw, bxe, bys, byn,
                                           G.slip, fast, K, B);
        };
        if (fast && full) {
            push_packed<S, SHEAR>(g, f, ps, ph, rS, rC, rN, ccA, ccB, cwA, ceB, zcA, lane, K,
                                  B);
        } else if (NARROW && fast) {
            push_pair_z<S>(g, f, ps, ph, rS, rC, rN, cwA, ccA, ceA, cwB, ccB, ceB, zcA, zcB,
                           actA, actB, K, B);
        } else {
            if (actA) push(false, cwA, ccA, ceA, zcA, bxwA, bxeA);
            if (actB) push(true, cwB, ccB, ceB, zcB, bxwB, bxeB);
        }
        issue(i + NS, st);
        rb = rc;
        rc = rn;
    };

    for (int i = 0, st = 1; i < nrows; ++i, st = (st + 1 == NS ? 0 : st + 1)) {
        body(i, st);
        if (!ok) return false;
    }
    // every copy issued has completed (the last wait was for row nrows): release the barriers
    __syncwarp();
    if (lane == 0)
        for (int s = 0; s < NS; ++s) mbar_inval(bar0 + 8 * s);
    __syncwarp();
    return true;
}

// Every step with FP32 arithmetic runs paired (two tiles per warp); FP64 one tile per warp.
template <typename R, typename S, int V>
struct Paired {
    static constexpr bool value = std::is_same<R, float>::value;
};
template <typename R, typename S, int V>
__host__ __device__ constexpr int tiles_per_warp() { return Paired<R, S, V>::value ? 2 : 1; }

template <typename R, typename S, int V, bool CK = false>
__device__ __forceinline__ void step_body(const S* __restrict__ src, S* __restrict__ dst,
                                          const Geometry& G, const Consts<R>& K,
                                          const StepLaunch& L)
{
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    constexpr int NT = tiles_per_warp<R, S, V>();
    const int wstrips = (G.nstrips + NT - 1) / NT;   // strips of NT tiles
    const int strip = warp % wstrips;
    const int seg = warp / wstrips;
    if (seg >= L.nseg) return;                       // warp-uniform
    const bool cut = L.cut_first_wait != 0;
    if constexpr (NT == 2)
        march2<S, V, CK>(src, dst, G, K, strip, seg, L.seg_h, L.err, L.flow_sign, L.flip,
                         L.chk_shrink, cut);
    else
        march<R, S, V, CK>(src, dst, G, K, strip, seg, L.seg_h, L.err, L.flow_sign, L.flip,
                           L.chk_shrink, cut);
}

template <typename R, typename S, int V>
__global__ void __launch_bounds__(256)
step_kernel(const S* __restrict__ src, S* __restrict__ dst, Geometry G, Consts<R> K,
            StepLaunch L)
{
    step_body<R, S, V>(src, dst, G, K, L);
}

// The 16-bit forms: at most 256 threads per block, like step_kernel, and at most 168 registers
// per thread, so that three 128-thread blocks (12 warps, the residency the shared memory allows
// the FP32 form) fit in the register file.  (Without the cap they take 172 and only 8 warps fit;
// a cap through __launch_bounds__(128, 3) instead gives slower code, 56.6 against 54.9 us per
// step on the 2048 x 1024 impact.)
template <typename S>
struct NarrowRegs {
    static constexpr int value = 168;
};

template <typename R, typename S, int V>
__global__ void __launch_bounds__(256) __maxnreg__(NarrowRegs<S>::value)
step_kernel_narrow(const S* __restrict__ src, S* __restrict__ dst, Geometry G, Consts<R> K,
                   StepLaunch L)
{
    step_body<R, S, V>(src, dst, G, K, L);
}

// The bounds-checked step (a debugging aid: see Bounds); same arithmetic, same results.
template <typename R, typename S, int V>
__global__ void __launch_bounds__(256)
step_kernel_checked(const S* __restrict__ src, S* __restrict__ dst, Geometry G, Consts<R> K,
                    StepLaunch L)
{
    step_body<R, S, V, true>(src, dst, G, K, L);
}

// The step kernel of a form.
template <typename R, typename S, int V>
constexpr auto step_kernel_of()
{
    if constexpr (Narrow<S>::value) return step_kernel_narrow<R, S, V>;
    else return step_kernel<R, S, V>;
}

// ---------------------------------------------------------------------------------------------
// Several time steps in one launch.  Every warp keeps its strip and segment from step to step,
// and before a step it waits only for the warps whose nodes that step reads or overwrites.  A
// warp reads its nodes and one halo row and column around them; each of those was written in
// the previous step by pushes from at most one row and column further out, and the nodes a warp
// writes (its own and one row and column around them) were read in the previous step by the
// warps whose halos reach them.  Both reach two nodes beyond the warp's own: the neighbouring
// strip and segment in each direction when every strip and segment is at least two nodes wide
// (reach 1), two strips or segments when one of them is a single column or row (reach 2, the
// host decides).  A warp publishes s + 1 in its progress word once all its stores of step s are
// visible at device scope; step s + 1 of a warp starts when the progress words of itself and of
// the warps within the reach are all >= s + 1.
// Within one step warps never wait for each other, so the step-to-step barrier of separate
// launches (every warp waits for the slowest) becomes a local one; the launch must be
// co-resident (cooperative), which the host guarantees.  Every wait is bounded: on a timeout,
// or once another warp has set the error word, a warp returns between two steps, when none of
// its copies is in flight.
// ---------------------------------------------------------------------------------------------
// Bound of a wait for the neighbouring warps: two seconds of the global timer (a neighbour's
// step takes microseconds to tens of milliseconds), and an iteration cap in case the timer
// does not advance.
constexpr unsigned long long NEIGHBOUR_WAIT_NS = 2000000000ull;
constexpr unsigned NEIGHBOUR_WAIT_ITERS = 1u << 27;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Warp-collective: wait until the progress words of the warp at (seg, strip) and of the warps
// within rx strips and ry segments of it (at most 25; periodic wrap in both directions, so a
// warp beyond a wall is waited for without need, which is harmless) reach `target`.  False on
// timeout (error word set) or when another warp has already failed.  far: test hook, the target
// is never reached.
__device__ __forceinline__ bool wait_neighbours(const unsigned* prog, int seg, int strip, int nseg,
                                                int nstrip, int rx, int ry, unsigned target,
                                                int* err, int lane, bool far)
{
    const unsigned* p = prog;
    const int wx = 2 * rx + 1;
    const bool mine = lane < wx * (2 * ry + 1);
    if (mine) {
        int s2 = seg + lane / wx - ry, t2 = strip + lane % wx - rx;
        s2 = ((s2 % nseg) + nseg) % nseg;
        t2 = ((t2 % nstrip) + nstrip) % nstrip;
        p = prog + (long long)s2 * nstrip + t2;
    }
    if (far) target += 0x40000000u;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0; it < NEIGHBOUR_WAIT_ITERS; ++it) {
        const unsigned v = mine ? ld_acquire(p) : target;
        if (__all_sync(FULL, (int)(v - target) >= 0)) {
            // the warp barrier orders every lane's later accesses after the acquires of lanes
            // 0 .. 24; the next copies go through the async proxy, so a proxy fence orders them
            // after the acquired stores as well
            __syncwarp();
            asm volatile("fence.proxy.async.global;" ::: "memory");
            return true;
        }
        // lane 0 decides for the warp: another warp failed, or this wait ran out of time
        int stop = 0;
        if (lane == 0)
            stop = *reinterpret_cast<volatile int*>(err) != 0
                       ? 1
                       : (global_ns() - t0 > NEIGHBOUR_WAIT_NS ? 2 : 0);
        stop = __shfl_sync(FULL, stop, 0);
        if (stop == 1) return false;
        if (stop == 2) break;
        __nanosleep(64);
    }
    if (lane == 0) atomicCAS(err, 0, 4);   // 4: a neighbour wait (1: a shared-memory wait)
    return false;
}

// Publish the end of step s of this warp: after the warp barrier, lane 0's release store of the
// progress word orders every lane's stores of the step before it (release is cumulative over
// what the barrier made lane 0 observe), as a grid barrier's single releasing thread does.
__device__ __forceinline__ void publish_step(unsigned* word, unsigned v, int lane)
{
    __syncwarp();
    if (lane == 0) st_release(word, v);
}

// Launch fields of the multi-step kernel beyond those of one step.
struct MultiLaunch {
    int nsteps;        // steps of this launch (the buffers alternate: a -> b -> a ...)
    unsigned* prog;    // one progress word per warp, zero at launch
    int rx, ry;        // reach of the waits in strips and segments (1 or 2)
    int far_wait;      // test hook: the waits for neighbours never succeed
};

template <typename R, typename S, int V>
__device__ __forceinline__ void multi_body(S* a, S* b, const Geometry& G, const Consts<R>& K,
                                           const StepLaunch& L, const MultiLaunch& M)
{
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    constexpr int NT = tiles_per_warp<R, S, V>();
    const int wstrips = (G.nstrips + NT - 1) / NT;
    const int strip = warp % wstrips;
    const int seg = warp / wstrips;
    if (seg >= L.nseg) return;                       // warp-uniform; not anyone's neighbour
    for (int s = 0; s < M.nsteps; ++s) {
        if (s > 0 && !wait_neighbours(M.prog, seg, strip, L.nseg, wstrips, M.rx, M.ry,
                                      (unsigned)s, L.err, lane, M.far_wait != 0))
            return;
        const S* src = (s & 1) ? b : a;
        S* dst = (s & 1) ? a : b;
        const int flip = flip_of(src, dst);
        bool ok;
        if constexpr (NT == 2)
            ok = march2<S, V, false, true>(src, dst, G, K, strip, seg, L.seg_h, L.err,
                                           L.flow_sign, flip);
        else
            ok = march<R, S, V, false, true>(src, dst, G, K, strip, seg, L.seg_h, L.err,
                                             L.flow_sign, flip);
        if (!ok) return;
        publish_step(M.prog + warp, (unsigned)(s + 1), lane);
    }
}

// Launched with one block of 12 warps per SM (kMultiBlock threads, lbm_device.cuh): the warps
// of an SM then share one block, and the scheduler favours none of them over the others, as it
// favours the older of several blocks; with several blocks per SM the warps of the youngest
// block fall behind, and through the waits between neighbours they pace every warp.
template <typename R, typename S, int V>
__global__ void __launch_bounds__(kMultiBlock)
step_kernel_multi(S* a, S* b, Geometry G, Consts<R> K, StepLaunch L, MultiLaunch M)
{
    multi_body<R, S, V>(a, b, G, K, L, M);
}

// The 16-bit forms, held to the register budget of step_kernel_narrow.
template <typename R, typename S, int V>
__global__ void __launch_bounds__(kMultiBlock) __maxnreg__(NarrowRegs<S>::value)
step_kernel_multi_narrow(S* a, S* b, Geometry G, Consts<R> K, StepLaunch L, MultiLaunch M)
{
    multi_body<R, S, V>(a, b, G, K, L, M);
}

template <typename R, typename S, int V>
constexpr auto multi_kernel_of()
{
    if constexpr (Narrow<S>::value) return step_kernel_multi_narrow<R, S, V>;
    else return step_kernel_multi<R, S, V>;
}

// One time step of many independent grids in one launch: warp w takes task w = (case, local
// warp index) from a flattened task list; every case has its own geometry, constants and pair
// of buffers inside one allocation.  All cases share the buffer parity (they step together) and
// the step variant V (no imposed flow).
template <typename R, typename S, int V>
__device__ __forceinline__ void batch_body(S* __restrict__ base,
                                           const BatchCase<R>* __restrict__ cases,
                                           const int2* __restrict__ tasks, int ntasks,
                                           int parity, int* err)
{
    static_assert((V & kVarShear) == 0, "batches take the coupled lattices");
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (warp >= ntasks) return;                      // warp-uniform
    const int2 t = tasks[warp];
    const BatchCase<R>& c = cases[t.x];
    const Geometry G = c.G;
    constexpr int NT = tiles_per_warp<R, S, V>();
    const int wstrips = (G.nstrips + NT - 1) / NT;
    const int strip = t.y % wstrips;
    const int seg = t.y / wstrips;
    const S* src = base + (parity ? c.off1 : c.off0);
    S* dst = base + (parity ? c.off0 : c.off1);
    if constexpr (NT == 2) march2<S, V>(src, dst, G, c.K, strip, seg, c.seg_h, err, 1, parity);
    else march<R, S, V>(src, dst, G, c.K, strip, seg, c.seg_h, err, 1, parity);
}

template <typename R, typename S, int V>
__global__ void __launch_bounds__(256)
batch_step_kernel(S* __restrict__ base, const BatchCase<R>* __restrict__ cases,
                  const int2* __restrict__ tasks, int ntasks, int parity, int* err)
{
    batch_body<R, S, V>(base, cases, tasks, ntasks, parity, err);
}

// The batched step of the 16-bit forms, held to 168 registers per thread like
// step_kernel_narrow (200 without the cap, which leaves 8 warps per SM).
template <typename R, typename S, int V>
__global__ void __launch_bounds__(256) __maxnreg__(NarrowRegs<S>::value)
batch_step_kernel_narrow(S* __restrict__ base, const BatchCase<R>* __restrict__ cases,
                         const int2* __restrict__ tasks, int ntasks, int parity, int* err)
{
    batch_body<R, S, V>(base, cases, tasks, ntasks, parity, err);
}

// The batched step kernel of a storage form and step variant.
template <typename R, typename S, int V>
constexpr auto batch_kernel_of()
{
    if constexpr (Narrow<S>::value) return batch_step_kernel_narrow<R, S, V>;
    else return batch_step_kernel<R, S, V>;
}

// ---------------------------------------------------------------------------------------------
// Several time steps of a batch in one launch.  The warps (one 12-warp block per SM, all
// resident: a cooperative launch) share the batch's tasks out once, balanced by nodes; every
// step, a warp takes its tasks in a fixed order, and before a task's step it waits only for the
// tasks of the same case within reach of that task's reads and writes (cases never wait for one
// another), through one progress word per task, as the single-grid multi-step kernel does per
// warp.  A step's waits are for work of the previous step only, so with every warp resident the
// waits always end; each is bounded all the same.
// ---------------------------------------------------------------------------------------------
struct BatchMulti {
    const int* order;   // task indices in the order the warps take them
    const int* wbeg;    // warp w takes order[wbeg[w] .. wbeg[w + 1])
    unsigned* prog;     // one progress word per task (tasks of a case are consecutive), zero at
                        // launch
    int nwarps, nsteps, parity0;
    int far_wait;       // test hook: the waits for neighbouring tasks never succeed
};

template <typename R, typename S, int V>
__device__ __forceinline__ void batch_multi_body(S* base, const BatchCase<R>* __restrict__ cases,
                                                 const int2* __restrict__ tasks,
                                                 const BatchMulti& M, int* err)
{
    static_assert((V & kVarShear) == 0, "batches take the coupled lattices");
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= M.nwarps) return;                    // warp-uniform
    constexpr int NT = tiles_per_warp<R, S, V>();
    const int j0 = M.wbeg[warp], j1 = M.wbeg[warp + 1];
    for (int s = 0; s < M.nsteps; ++s) {
        const int parity = M.parity0 ^ (s & 1);
        for (int j = j0; j < j1; ++j) {
            const int id = M.order[j];
            const int2 t = tasks[id];                // (case, local index seg * wstrips + strip)
            const BatchCase<R>& c = cases[t.x];
            const Geometry G = c.G;
            const int wstrips = (G.nstrips + NT - 1) / NT;
            const int strip = t.y % wstrips;
            const int seg = t.y / wstrips;
            if (s > 0) {
                // reach 2 where the case's last strip or segment is one node wide
                const int last_w = G.nx - (wstrips - 1) * 32 * NT;
                const int last_h = G.ny - (c.nseg - 1) * c.seg_h;
                const int rx = last_w >= 2 || wstrips == 1 ? 1 : 2;
                const int ry = (c.seg_h >= 2 && last_h >= 2) || c.nseg == 1 ? 1 : 2;
                if (!wait_neighbours(M.prog + (id - t.y), seg, strip, c.nseg, wstrips, rx, ry,
                                     (unsigned)s, err, lane, M.far_wait != 0))
                    return;
            }
            const S* src = base + (parity ? c.off1 : c.off0);
            S* dst = base + (parity ? c.off0 : c.off1);
            bool ok;
            if constexpr (NT == 2)
                ok = march2<S, V, false, true>(src, dst, G, c.K, strip, seg, c.seg_h, err, 1,
                                               parity);
            else
                ok = march<R, S, V, false, true>(src, dst, G, c.K, strip, seg, c.seg_h, err, 1,
                                                 parity);
            if (!ok) return;
            publish_step(M.prog + id, (unsigned)(s + 1), lane);
        }
    }
}

template <typename R, typename S, int V>
__global__ void __launch_bounds__(kMultiBlock)
batch_multi_kernel(S* base, const BatchCase<R>* __restrict__ cases,
                   const int2* __restrict__ tasks, BatchMulti M, int* err)
{
    batch_multi_body<R, S, V>(base, cases, tasks, M, err);
}

template <typename R, typename S, int V>
__global__ void __launch_bounds__(kMultiBlock) __maxnreg__(NarrowRegs<S>::value)
batch_multi_kernel_narrow(S* base, const BatchCase<R>* __restrict__ cases,
                          const int2* __restrict__ tasks, BatchMulti M, int* err)
{
    batch_multi_body<R, S, V>(base, cases, tasks, M, err);
}

template <typename R, typename S, int V>
constexpr auto batch_multi_kernel_of()
{
    if constexpr (Narrow<S>::value) return batch_multi_kernel_narrow<R, S, V>;
    else return batch_multi_kernel<R, S, V>;
}

// ---------------------------------------------------------------------------------------------
// Initialisation, field extraction, packing (one thread per node; not on the hot path)
// ---------------------------------------------------------------------------------------------
// Element index of population plane p (0..17) of node (x, y) in a state of storage type S, and
// (16-bit forms) of the node's Z plane lat (an FP32 value spanning two elements).
template <typename S>
__device__ __forceinline__ long long elem_index(const Geometry& G, int p, int x, int y)
{
    return ((long long)y * G.nstrips + (x >> 5)) * Tile<S>::ELEMS + Tile<S>::P0 + p * 32 +
           (x & 31);
}
template <typename S>
__device__ __forceinline__ long long z_index(const Geometry& G, int lat, int x, int y)
{
    return ((long long)y * G.nstrips + (x >> 5)) * Tile<S>::ELEMS + 64 * lat + 2 * (x & 31);
}

// The 18 populations of node (x, y) (decoded).
template <typename R, typename S>
__device__ __forceinline__ void load_node(const S* state, const Geometry& G, const Consts<R>& K,
                                          int x, int y, R g[9], R f[9])
{
    R zg = R(0), zf = R(0);
    if constexpr (Narrow<S>::value) {
        zg = R(*reinterpret_cast<const float*>(state + z_index<S>(G, 0, x, y)));
        zf = R(*reinterpret_cast<const float*>(state + z_index<S>(G, 1, x, y)));
    }
    for (int a = 0; a < 9; ++a) {
        g[a] = decode<S, R>(state[elem_index<S>(G, a, x, y)], zg, 0, a, K);
        f[a] = decode<S, R>(state[elem_index<S>(G, 9 + a, x, y)], zf, 1, a, K);
    }
}

// Store the 18 populations of node (x, y); the 16-bit forms take the node's own zeroth moments
// as their references.
template <typename R, typename S>
__device__ __forceinline__ void store_node(S* state, const Geometry& G, const Consts<R>& K,
                                           int x, int y, const R g[9], const R f[9])
{
    R zg = R(0), zf = R(0);
    if constexpr (Narrow<S>::value) {
        for (int a = 0; a < 9; ++a) {
            zg += g[a];
            zf += f[a];
        }
        *reinterpret_cast<float*>(state + z_index<S>(G, 0, x, y)) = float(zg);
        *reinterpret_cast<float*>(state + z_index<S>(G, 1, x, y)) = float(zf);
        zg = R(float(zg));   // the reader decodes against the stored FP32 value
        zf = R(float(zf));
    }
    for (int a = 0; a < 9; ++a) {
        state[elem_index<S>(G, a, x, y)] = encode<S, R>(g[a], zg, 0, a, K);
        state[elem_index<S>(G, 9 + a, x, y)] = encode<S, R>(f[a], zf, 1, a, K);
    }
}

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
    store_node<R, S>(state, G, K, x, y, g, f);
}

// Macroscopic fields of a state: phi, corrected p, u, rho (double outputs, [ny][nx]).  One
// thread per node; the 3x3 neighbourhood sums are recomputed per node (diagnostic path).
template <typename R, typename S>
__global__ void fields_kernel(const S* __restrict__ state, Geometry G, Consts<R> K,
                              int flow_sign, double* __restrict__ phi_o, double* __restrict__ p_o,
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
            const int xx = map_col(x + i, G);
            R gq[9], fq[9];
            load_node<R, S>(state, G, K, xx, yy, gq, fq);
            vph[j + 1][i + 1] =
                ((fq[0] + fq[1]) + (fq[2] + fq[3])) + ((fq[4] + fq[5]) + (fq[6] + fq[7])) + fq[8];
            vps[j + 1][i + 1] =
                ((gq[0] + gq[1]) + (gq[2] + gq[3])) + ((gq[4] + gq[5]) + (gq[6] + gq[7])) + gq[8];
        }
    }
    Win<R> ph = {vph[0][0], vph[0][1], vph[0][2], vph[1][0], vph[1][1], vph[1][2],
                 vph[2][0], vph[2][1], vph[2][2]};
    Win<R> ps = {vps[0][0], vps[0][1], vps[0][2], vps[1][0], vps[1][1], vps[1][2],
                 vps[2][0], vps[2][1], vps[2][2]};
    R gq[9], fq[9];
    load_node<R, S>(state, G, K, x, y, gq, fq);
    const R jgx = (gq[1] - gq[3]) + (gq[5] - gq[6]) - (gq[7] - gq[8]);
    const R jgy = (gq[2] - gq[4]) + (gq[5] + gq[6]) - (gq[7] + gq[8]);
    Macro<R> m;
    if (K.langmuir) node_macro<R, true>(ph, ps, jgx, jgy, R(x), R(y), K, m);
    else node_macro<R, false>(ph, ps, jgx, jgy, R(x), R(y), K, m);
    if (flow_sign) {   // imposed flow: u from the field, no pressure
        R sx, cx, sy, cy;
        sincospi_(R(x) * K.inv_nx - R(0.5), &sx, &cx);
        sincospi_(R(y) * K.inv_ny - R(0.5), &sy, &cy);
        imposed_velocity<R>(sx, cx, sy, cy, R(flow_sign), K, m.ux, m.uy);
        m.p = R(0);
    }
    if (phi_o) phi_o[n] = double(ph.c);
    if (p_o) p_o[n] = double(m.p);
    if (ux_o) ux_o[n] = double(m.ux);
    if (uy_o) uy_o[n] = double(m.uy);
    if (rho_o) rho_o[n] = double(m.rho);
}

// Copy between the tiled device state and a dense [18][ny][nx] double array (decoded values);
// one thread per node.
template <typename R, typename S>
__global__ void pack_kernel(const S* __restrict__ state, double* __restrict__ out, Geometry G,
                            Consts<R> K)
{
    const long long N = (long long)G.nx * G.ny;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    R g[9], f[9];
    load_node<R, S>(state, G, K, (int)(n % G.nx), (int)(n / G.nx), g, f);
    for (int a = 0; a < 9; ++a) {
        out[a * N + n] = double(g[a]);
        out[(9 + a) * N + n] = double(f[a]);
    }
}

template <typename R, typename S>
__global__ void unpack_kernel(const double* __restrict__ in, S* __restrict__ state, Geometry G,
                              Consts<R> K)
{
    const long long N = (long long)G.nx * G.ny;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    R g[9], f[9];
    for (int a = 0; a < 9; ++a) {
        g[a] = R(in[a * N + n]);
        f[a] = R(in[(9 + a) * N + n]);
    }
    store_node<R, S>(state, G, K, (int)(n % G.nx), (int)(n / G.nx), g, f);
}

// ---------------------------------------------------------------------------------------------
// Host-side launchers (called from lbm_api.cu)
// ---------------------------------------------------------------------------------------------
template <typename S, int NT>
size_t tile_smem_bytes(int block) { return (size_t)(block / 32) * warp_smem_bytes<S, NT>(); }
template <typename R, typename S, int V>
size_t step_smem_bytes(int block) { return tile_smem_bytes<S, tiles_per_warp<R, S, V>()>(block); }

// Warp strips of a row: tiles per warp for this variant.
template <typename R, typename S, int V>
int step_warp_strips(int nstrips)
{
    constexpr int NT = tiles_per_warp<R, S, V>();
    return (nstrips + NT - 1) / NT;
}

// Allow the dynamic shared memory of a block of `block` threads (call once per device).
template <typename R, typename S, int V>
cudaError_t configure_step(int block)
{
    cudaError_t e = cudaFuncSetAttribute(step_kernel_of<R, S, V>(),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_smem_bytes<R, S, V>(block));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_kernel_of<R, S, V>(),
                                cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

// Resident blocks of `block` threads per SM for the step kernel.
template <typename R, typename S, int V>
int step_blocks_per_sm(int block)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, step_kernel_of<R, S, V>(), block,
                                                      step_smem_bytes<R, S, V>(block)) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}


template <typename R, typename S, int V>
cudaError_t launch_step(const void* src, void* dst, const Geometry& G, const Consts<R>& K,
                        int seg_h, int block, int* err, int flow_sign, int cut_first_wait,
                        cudaStream_t st)
{
    StepLaunch L = {};
    L.seg_h = seg_h;
    L.nseg = (G.ny + seg_h - 1) / seg_h;
    L.err = err;
    L.flow_sign = flow_sign;
    L.flip = flip_of(src, dst);
    L.cut_first_wait = cut_first_wait;
    const long long warps = (long long)step_warp_strips<R, S, V>(G.nstrips) * L.nseg;
    const int wpb = block / 32;
    const long long grid = (warps + wpb - 1) / wpb;
    step_kernel_of<R, S, V>()<<<(unsigned)grid, block, step_smem_bytes<R, S, V>(block), st>>>(
        static_cast<const S*>(src), static_cast<S*>(dst), G, K, L);
    return cudaGetLastError();
}

// The multi-step kernel: configuration, residency and launch.  launch_multi clears the progress
// words, then launches cooperatively (every block resident at once, or the launch fails and
// nothing runs); the host calls it only when the grid fits (multi_blocks_per_sm).
template <typename R, typename S, int V>
cudaError_t configure_multi(int block)
{
    cudaError_t e = cudaFuncSetAttribute(multi_kernel_of<R, S, V>(),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_smem_bytes<R, S, V>(block));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(multi_kernel_of<R, S, V>(),
                                cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

template <typename R, typename S, int V>
int multi_blocks_per_sm(int block)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, multi_kernel_of<R, S, V>(), block,
                                                      step_smem_bytes<R, S, V>(block)) !=
        cudaSuccess)
        return 0;
    return nb;
}

template <typename R, typename S, int V>
cudaError_t launch_multi(void* a, void* b, const Geometry& G, const Consts<R>& K, int seg_h,
                         int block, int* err, int flow_sign, int nsteps, unsigned* prog,
                         int far_wait, cudaStream_t st)
{
    StepLaunch L = {};
    L.seg_h = seg_h;
    L.nseg = (G.ny + seg_h - 1) / seg_h;
    L.err = err;
    L.flow_sign = flow_sign;
    // reach of the waits: 2 where the last strip (columns) or segment (rows) is one node wide
    constexpr int COLS = 32 * tiles_per_warp<R, S, V>();
    const int wstrips = step_warp_strips<R, S, V>(G.nstrips);
    const int last_w = G.nx - (wstrips - 1) * COLS;
    const int last_h = G.ny - (L.nseg - 1) * seg_h;
    MultiLaunch M = {nsteps, prog, last_w >= 2 || wstrips == 1 ? 1 : 2,
                     (seg_h >= 2 && last_h >= 2) || L.nseg == 1 ? 1 : 2, far_wait};
    const long long warps = (long long)wstrips * L.nseg;
    const int wpb = block / 32;
    const unsigned grid = (unsigned)((warps + wpb - 1) / wpb);
    cudaError_t e = cudaMemsetAsync(prog, 0, (size_t)warps * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    S* pa = static_cast<S*>(a);
    S* pb = static_cast<S*>(b);
    Geometry g = G;
    Consts<R> k = K;
    void* args[] = {(void*)&pa, (void*)&pb, (void*)&g, (void*)&k, (void*)&L, (void*)&M};
    return cudaLaunchCooperativeKernel((const void*)multi_kernel_of<R, S, V>(), dim3(grid),
                                       dim3(block), args, step_smem_bytes<R, S, V>(block), st);
}

// The bounds-checked step of the coupled cascaded form (variant 0): configuration and launch,
// as configure_step / launch_step.
template <typename R, typename S>
cudaError_t configure_step_checked(int block)
{
    return cudaFuncSetAttribute(step_kernel_checked<R, S, 0>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)step_smem_bytes<R, S, 0>(block));
}

template <typename R, typename S>
cudaError_t launch_step_checked(const void* src, void* dst, const Geometry& G,
                                const Consts<R>& K, int seg_h, int block, int* err,
                                int shrink_rows, cudaStream_t st)
{
    StepLaunch L = {};
    L.chk_shrink = (long long)shrink_rows * G.nstrips * Tile<S>::ELEMS;
    L.seg_h = seg_h;
    L.nseg = (G.ny + seg_h - 1) / seg_h;
    L.err = err;
    L.flow_sign = 1;
    L.flip = flip_of(src, dst);
    const long long warps = (long long)step_warp_strips<R, S, 0>(G.nstrips) * L.nseg;
    const int wpb = block / 32;
    const long long grid = (warps + wpb - 1) / wpb;
    step_kernel_checked<R, S, 0><<<(unsigned)grid, block, step_smem_bytes<R, S, 0>(block), st>>>(
        static_cast<const S*>(src), static_cast<S*>(dst), G, K, L);
    return cudaGetLastError();
}

// A graph of `chunk` consecutive steps starting from buffer `a` (a -> b -> a -> ...), replayed
// by lbm_step to cut the per-launch gaps between steps.
template <typename R, typename S, int V>
cudaError_t build_step_graph(const void* a, const void* b, const Geometry& G, const Consts<R>& K,
                             int seg_h, int block, int* err, int flow_sign, int chunk,
                             cudaGraphExec_t* out)
{
    StepLaunch L = {};
    L.seg_h = seg_h;
    L.nseg = (G.ny + seg_h - 1) / seg_h;
    L.err = err;
    L.flow_sign = flow_sign;
    const long long warps = (long long)step_warp_strips<R, S, V>(G.nstrips) * L.nseg;
    const int wpb = block / 32;
    const unsigned grid = (unsigned)((warps + wpb - 1) / wpb);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    cudaGraphNode_t prev = nullptr;
    Geometry g = G;
    Consts<R> k = K;
    for (int s = 0; s < chunk && e == cudaSuccess; ++s) {
        const S* src = static_cast<const S*>((s & 1) ? b : a);
        S* dst = const_cast<S*>(static_cast<const S*>((s & 1) ? a : b));
        L.flip = flip_of(src, dst);
        void* args[] = {(void*)&src, (void*)&dst, (void*)&g, (void*)&k, (void*)&L};
        cudaKernelNodeParams p = {};
        p.func = (void*)step_kernel_of<R, S, V>();
        p.gridDim = dim3(grid);
        p.blockDim = dim3(block);
        p.sharedMemBytes = (unsigned)step_smem_bytes<R, S, V>(block);
        p.kernelParams = args;
        cudaGraphNode_t node;
        e = cudaGraphAddKernelNode(&node, graph, prev ? &prev : nullptr, prev ? 1 : 0, &p);
        prev = node;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

template <typename R, typename S, int V>
cudaError_t configure_batch(int block)
{
    cudaError_t e = cudaFuncSetAttribute(batch_kernel_of<R, S, V>(),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_smem_bytes<R, S, V>(block));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(batch_kernel_of<R, S, V>(),
                                cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

template <typename R, typename S, int V>
cudaError_t launch_batch_step(void* base, const BatchCase<R>* cases, const int2* tasks,
                              int ntasks, int parity, int block, int* err, cudaStream_t st)
{
    const int wpb = block / 32;
    const unsigned grid = (unsigned)((ntasks + wpb - 1) / wpb);
    batch_kernel_of<R, S, V>()<<<grid, block, step_smem_bytes<R, S, V>(block), st>>>(
        static_cast<S*>(base), cases, tasks, ntasks, parity, err);
    return cudaGetLastError();
}

// The batched multi-step kernel: configuration, residency and launch (cooperative; the host
// calls it only when its warps fit on the device at once).
template <typename R, typename S, int V>
cudaError_t configure_batch_multi()
{
    cudaError_t e = cudaFuncSetAttribute(batch_multi_kernel_of<R, S, V>(),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_smem_bytes<R, S, V>(kMultiBlock));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(batch_multi_kernel_of<R, S, V>(),
                                cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

template <typename R, typename S, int V>
int batch_multi_blocks_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_multi_kernel_of<R, S, V>(),
                                                      kMultiBlock,
                                                      step_smem_bytes<R, S, V>(kMultiBlock)) !=
        cudaSuccess)
        return 0;
    return nb;
}

template <typename R, typename S, int V>
cudaError_t launch_batch_multi(void* base, const BatchCase<R>* cases, const int2* tasks,
                               const int* order, const int* wbeg, unsigned* prog, int ntasks,
                               int nwarps, int nsteps, int parity0, int far_wait, int* err,
                               cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(prog, 0, (size_t)ntasks * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    BatchMulti M = {order, wbeg, prog, nwarps, nsteps, parity0, far_wait};
    S* b = static_cast<S*>(base);
    const int wpb = kMultiBlock / 32;
    const unsigned grid = (unsigned)((nwarps + wpb - 1) / wpb);
    void* args[] = {(void*)&b, (void*)&cases, (void*)&tasks, (void*)&M, (void*)&err};
    return cudaLaunchCooperativeKernel((const void*)batch_multi_kernel_of<R, S, V>(), dim3(grid),
                                       dim3(kMultiBlock), args,
                                       step_smem_bytes<R, S, V>(kMultiBlock), st);
}

// A graph of `chunk` consecutive batched steps starting from buffer parity `parity0`.
template <typename R, typename S, int V>
cudaError_t build_batch_graph(void* base, const BatchCase<R>* cases, const int2* tasks,
                              int ntasks, int parity0, int block, int* err, int chunk,
                              cudaGraphExec_t* out)
{
    const int wpb = block / 32;
    const unsigned grid = (unsigned)((ntasks + wpb - 1) / wpb);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    cudaGraphNode_t prev = nullptr;
    S* b = static_cast<S*>(base);
    for (int s = 0; s < chunk && e == cudaSuccess; ++s) {
        int parity = (parity0 + s) & 1;
        int n = ntasks;
        void* args[] = {(void*)&b, (void*)&cases, (void*)&tasks, (void*)&n, (void*)&parity,
                        (void*)&err};
        cudaKernelNodeParams p = {};
        p.func = (void*)batch_kernel_of<R, S, V>();
        p.gridDim = dim3(grid);
        p.blockDim = dim3(block);
        p.sharedMemBytes = (unsigned)step_smem_bytes<R, S, V>(block);
        p.kernelParams = args;
        cudaGraphNode_t node;
        e = cudaGraphAddKernelNode(&node, graph, prev ? &prev : nullptr, prev ? 1 : 0, &p);
        prev = node;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    return e;
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
                          int flow_sign, double* phi, double* p, double* ux, double* uy,
                          double* rho, cudaStream_t st)
{
    const long long N = (long long)G.nx * G.ny;
    fields_kernel<R, S><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(
        static_cast<const S*>(state), G, K, flow_sign, phi, p, ux, uy, rho);
    return cudaGetLastError();
}

template <typename R, typename S>
cudaError_t launch_pack(const void* state, double* out, const Geometry& G, const Consts<R>& K,
                        cudaStream_t st)
{
    const long long T = (long long)G.nx * G.ny;
    pack_kernel<R, S><<<(unsigned)((T + 255) / 256), 256, 0, st>>>(
        static_cast<const S*>(state), out, G, K);
    return cudaGetLastError();
}

template <typename R, typename S>
cudaError_t launch_unpack(const double* in, void* state, const Geometry& G, const Consts<R>& K,
                          cudaStream_t st)
{
    const long long T = (long long)G.nx * G.ny;
    unpack_kernel<R, S><<<(unsigned)((T + 255) / 256), 256, 0, st>>>(in, static_cast<S*>(state),
                                                                     G, K);
    return cudaGetLastError();
}

#define CMLBM_INSTANTIATE_STEP(R, S, V)                                                           \
    template int step_warp_strips<R, S, V>(int);                                                \
    template cudaError_t configure_step<R, S, V>(int);                                          \
    template int step_blocks_per_sm<R, S, V>(int);                                              \
    template cudaError_t build_step_graph<R, S, V>(const void*, const void*, const Geometry&,   \
                                                   const Consts<R>&, int, int, int*, int, int,  \
                                                   cudaGraphExec_t*);                           \
    template cudaError_t launch_step<R, S, V>(const void*, void*, const Geometry&,              \
                                              const Consts<R>&, int, int, int*, int, int,       \
                                              cudaStream_t);                                    \
    template cudaError_t configure_multi<R, S, V>(int);                                         \
    template int multi_blocks_per_sm<R, S, V>(int);                                             \
    template cudaError_t launch_multi<R, S, V>(void*, void*, const Geometry&, const Consts<R>&, \
                                               int, int, int*, int, int, unsigned*, int,        \
                                               cudaStream_t);

#define CMLBM_INSTANTIATE(R, S)                                                                   \
    template cudaError_t configure_step_checked<R, S>(int);                                     \
    template cudaError_t launch_step_checked<R, S>(const void*, void*, const Geometry&,         \
                                                   const Consts<R>&, int, int, int*, int,       \
                                                   cudaStream_t);                               \
    template cudaError_t launch_init<R, S>(const double*, const double*, const double*,         \
                                           const double*, void*, const Geometry&,               \
                                           const Consts<R>&, cudaStream_t);                     \
    template cudaError_t launch_fields<R, S>(const void*, const Geometry&, const Consts<R>&,    \
                                             int, double*, double*, double*, double*, double*,  \
                                             cudaStream_t);

#define CMLBM_INSTANTIATE_BATCH(R, S, V)                                                          \
    template cudaError_t configure_batch_multi<R, S, V>();                                      \
    template int batch_multi_blocks_per_sm<R, S, V>();                                          \
    template cudaError_t launch_batch_multi<R, S, V>(void*, const BatchCase<R>*, const int2*,   \
                                                     const int*, const int*, unsigned*, int,    \
                                                     int, int, int, int, int*, cudaStream_t);   \
    template cudaError_t configure_batch<R, S, V>(int);                                         \
    template cudaError_t build_batch_graph<R, S, V>(void*, const BatchCase<R>*, const int2*,    \
                                                    int, int, int, int*, int,                   \
                                                    cudaGraphExec_t*);                          \
    template cudaError_t launch_batch_step<R, S, V>(void*, const BatchCase<R>*, const int2*,    \
                                                    int, int, int, int*, cudaStream_t);

// Populations are copied in and out in double; the codec of the 16-bit formats is applied in
// double there so that a value read out and written back is stored exactly as before.
#define CMLBM_INSTANTIATE_PACK(S)                                                                 \
    template cudaError_t launch_pack<double, S>(const void*, double*, const Geometry&,          \
                                                const Consts<double>&, cudaStream_t);           \
    template cudaError_t launch_unpack<double, S>(const double*, void*, const Geometry&,        \
                                                  const Consts<double>&, cudaStream_t);

CMLBM_INSTANTIATE(double, double)
CMLBM_INSTANTIATE(float, float)
CMLBM_INSTANTIATE(float, __half)
CMLBM_INSTANTIATE(float, __nv_bfloat16)
// every variant in FP64 and FP32; the 16-bit storage modes take the cascaded coupled step only
CMLBM_INSTANTIATE_STEP(double, double, 0)
CMLBM_INSTANTIATE_STEP(double, double, 1)
CMLBM_INSTANTIATE_STEP(double, double, 2)
CMLBM_INSTANTIATE_STEP(double, double, 3)
CMLBM_INSTANTIATE_STEP(double, double, 4)
CMLBM_INSTANTIATE_STEP(double, double, 5)
CMLBM_INSTANTIATE_STEP(float, float, 0)
CMLBM_INSTANTIATE_STEP(float, float, 1)
CMLBM_INSTANTIATE_STEP(float, float, 2)
CMLBM_INSTANTIATE_STEP(float, float, 3)
CMLBM_INSTANTIATE_STEP(float, float, 4)
CMLBM_INSTANTIATE_STEP(float, float, 5)
CMLBM_INSTANTIATE_STEP(float, __half, 0)
CMLBM_INSTANTIATE_STEP(float, __nv_bfloat16, 0)
// batches: the coupled-lattice variants (cascaded / SRT, linear sigma / Langmuir) in FP64 and
// FP32, the cascaded linear-sigma step in the 16-bit storage modes
CMLBM_INSTANTIATE_BATCH(double, double, 0)
CMLBM_INSTANTIATE_BATCH(double, double, 1)
CMLBM_INSTANTIATE_BATCH(double, double, 4)
CMLBM_INSTANTIATE_BATCH(double, double, 5)
CMLBM_INSTANTIATE_BATCH(float, float, 0)
CMLBM_INSTANTIATE_BATCH(float, float, 1)
CMLBM_INSTANTIATE_BATCH(float, float, 4)
CMLBM_INSTANTIATE_BATCH(float, float, 5)
CMLBM_INSTANTIATE_BATCH(float, __half, 0)
CMLBM_INSTANTIATE_BATCH(float, __nv_bfloat16, 0)
CMLBM_INSTANTIATE_PACK(double)
CMLBM_INSTANTIATE_PACK(float)
CMLBM_INSTANTIATE_PACK(__half)
CMLBM_INSTANTIATE_PACK(__nv_bfloat16)
#undef CMLBM_INSTANTIATE
#undef CMLBM_INSTANTIATE_STEP
#undef CMLBM_INSTANTIATE_PACK
#undef CMLBM_INSTANTIATE_BATCH

}  // namespace cmlbm
