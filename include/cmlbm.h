/*
 * cmlbm.h - C ABI of the GB300 (sm_103a) library for the coupled cascaded central-moment
 * lattice Boltzmann schemes of Hajabdollahi, Premnath & Welch, "Central Moment Lattice
 * Boltzmann Method using a Pressure-based Formulation for Multiphase Flows at High Density
 * Ratios and including Effects of Surface Tension and Marangoni Stresses" (arXiv:1909.04166).
 *
 * What one time step computes (lbm_step), for every node of an nx x ny D2Q9 lattice:
 *   - phi = sum_a f_a (Sec. 5) and p* = sum_a g-bar_a (Sec. 4) on the node and its neighbours;
 *   - rho = rho_B + phi (rho_A - rho_B), mu = mu_B + phi (mu_A - mu_B) (Sec. 2, linear
 *     interpolation with phi_A = 1, phi_B = 0);
 *   - second-order isotropic gradients / Laplacian / Hessian of phi and the gradient of p*
 *     (Sec. 4, closing remark);
 *   - the geometric surface-tension force with its Marangoni part (Sec. 2 Eq.
 *     surfacetensiongeometric; Sec. 6.7 Eqs. surfacetensiongeometricsurfactantsxcomp/ycomp),
 *     kappa-tilde = (3/2) sigma(T) W, sigma(T) = sigma0 + dsigma_dT (T - T0),
 *     T = T0 + gradT_x x + gradT_y y;
 *   - F_ext = (rho - rho_ref) (gx, gy); F_t = F_s + F_ext; F_p = -grad p* + c_s^2 (rho_A -
 *     rho_B) grad phi (Sec. 3 Eq. netgradientpressureforce);
 *   - corrected u and p (Sec. 4 Eq. hydrodynamicfields);
 *   - the fluid cascaded collision with its cumulative source (Sec. 4 Eqs.
 *     cascadedcollisionoperator, cumulativesourcetermcomponents, postcollisioncascadedLBscheme),
 *     shear rates from mu (Eq. fluidviscosity), all other rates 1;
 *   - the interface (conservative Allen-Cahn) cascaded collision with M_phi theta n in its
 *     first-order equilibria (Sec. 5), omega^phi_{1,2} from M_phi, all other rates 1;
 *   - streaming of both lattices, with half-way bounce-back at no-slip walls and specular
 *     reflection at free-slip walls.
 * lbm_params also selects the paper's other forms: the single-relaxation-time operators of its
 * stability comparison (Sec. 7), the Langmuir isotherm of its surfactant Marangoni case (Sec.
 * 6.7) and the interface lattice alone in its imposed reversing shear flow (Sec. 6.1).
 *
 * Conventions: c_s^2 = 1/3, lattice units (dx = dt = 1).  Node (i, j) is at x = i, y = j.
 * Host nodal arrays are row-major [ny][nx] doubles.  Population arrays are [9][ny][nx] doubles
 * with the D2Q9 ordering e_x = (0,1,0,-1,0,1,-1,-1,1), e_y = (0,0,1,0,-1,1,1,-1,-1) (Sec. 4
 * Eq. particlevelocities); g is the fluid lattice (g-bar of Sec. 4), f the interface lattice.
 * The library state holds the streamed (pre-collision) populations of the current time level.
 *
 * Ownership: the caller owns every host array; the library copies in and out and never keeps a
 * host pointer.  The library owns its device buffers unless they are supplied through
 * lbm_create_with_buffer, in which case the caller owns them and must keep them alive until
 * lbm_destroy.  All device work is issued on params.stream (a cudaStream_t; NULL = the legacy
 * default stream).  Calls that return host data synchronise that stream.
 *
 * Errors: every int-returning call returns LBM_OK (0) or a negative code; no call aborts, exits
 * or traps on the device.  lbm_strerror gives a message.  A failed call leaves the context
 * usable unless the code is LBM_ERR_CUDA (then the CUDA context may be unusable; see
 * lbm_last_cuda_error).
 */
#ifndef CMLBM_H
#define CMLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_ERR_ARG (-1)        /* NULL pointer, size out of range, unknown enum value */
#define LBM_ERR_PARAM (-2)      /* physically invalid parameter (rho <= 0, mu <= 0, W <= 0,
                                   M_phi <= 0, non-finite value) */
#define LBM_ERR_CUDA (-3)       /* a CUDA runtime call failed */
#define LBM_ERR_NOMEM (-4)      /* device allocation failed */
#define LBM_ERR_STATE (-5)      /* the state was never initialised */
#define LBM_ERR_NONFINITE (-6)  /* a diagnostic found NaN or Inf in the fields */
#define LBM_ERR_UNSUPPORTED (-7)/* precision mode not built into this library, or a collision
                                   model / flow mode not offered with the precision or in a
                                   batch */
#define LBM_ERR_TIMEOUT (-8)    /* a bounded wait inside the step kernel gave up (every wait
                                   gives up after two seconds of the GPU's global timer); the
                                   state of that step is invalid (reported by the next
                                   synchronising call or lbm_check) */
#define LBM_ERR_INDEX (-9)      /* the bounds-checked step kernel (lbm_set_checked) met a load,
                                   store or copy outside the state buffers and skipped it; the
                                   state is invalid (reported as LBM_ERR_TIMEOUT is) */

/* Storage / compute precision of a context. */
typedef enum {
    LBM_FP64 = 0,       /* populations stored and collided in double (correctness mode) */
    LBM_FP32 = 1,       /* populations stored and collided in float */
    LBM_FP32_FP16 = 2,  /* collided in float; stored as IEEE half deviations (see below) */
    LBM_FP32_BF16 = 3   /* collided in float; stored as bfloat16 deviations (see below) */
} lbm_precision;
/* 16-bit storage: every tile (32 columns of one row) holds two FP32 planes with each node's
 * zeroth moments of the previous time level, Z_g = p* and Z_f = phi, and then the 18 populations
 * as 16-bit deviations d_a = (q_a - w_a Z_L) scale_L from the rest-state populations w_a Z_L of
 * the node they sit on (w the D2Q9 weights 4/9, 1/9, 1/36; L the lattice).  The kernel that
 * pushes a population knows its destination's Z from its stencil window, so the pressure level
 * and the phase fraction are carried in FP32 and only the departures from rest are rounded, the
 * floating exponent keeping the light phase's momentum significant.  scale_L =
 * params.store_scale_g / store_scale_f, or when those are 0 the defaults 2^14 / 2^12 for FP16
 * (deviations from ~1e-6 to ~4 in the normal range) and 1 / 1 for BF16.  Collisions, forces and
 * stencils stay in float.  A step stores each node's rest population last, with the 16-bit
 * rounding errors of its eight moving populations subtracted from its deviation, so the
 * populations a node sends out sum to what it computed up to one rounding of that (small)
 * deviation: the lattice sums, the phase mass among them, do not drift with the storage
 * rounding of a nearly steady state. */

/* Boundary kind of the sides of one axis. */
typedef enum {
    LBM_PERIODIC = 0,
    LBM_WALL = 1,      /* no-slip wall half a node outside the first / last node (half-way
                          bounce-back on both lattices; mirror ghosts for the stencils) */
    LBM_FREESLIP = 2   /* free-slip wall (Secs. 6.4-6.6) half a node outside the first / last
                          node: a population crossing it reverses its normal velocity and lands on
                          the tangential neighbour inside (specular reflection); at a corner with
                          a no-slip side it bounces back; mirror ghosts for the stencils */
} lbm_bc;

/* Collision model of both lattices. */
typedef enum {
    LBM_CASCADED = 0,  /* the cascaded operators of Secs. 4 and 5 (rates as above) */
    LBM_SRT = 1        /* single relaxation time, the comparison model of Sec. 7: the same
                          operators with every rate equal to the shear rate (fluid) and to
                          omega^phi_{1,2} (interface), i.e. BGK towards the same equilibria with
                          the same sources.  LBM_FP64 / LBM_FP32 only. */
} lbm_collision;

/* Surface tension law. */
typedef enum {
    LBM_SIGMA_LINEAR_T = 0,  /* sigma = sigma0 + dsigma_dT (T - T0), T = T0 + gradT . x */
    LBM_SIGMA_LANGMUIR = 1   /* Langmuir isotherm (Sec. 6.7 Eq. Langmuirisotherm):
                                sigma = sigma0 [1 + beta ln(1 - psi)] in the imposed surfactant
                                concentration psi = psi0 + gradpsi_x x + gradpsi_y y (psi < 1 on
                                the whole grid); kappa-tilde = (3/2) sigma W with its analytic
                                gradient in the Marangoni force */
} lbm_sigma_model;

/* What is advanced. */
typedef enum {
    LBM_FLOW_COUPLED = 0,  /* both lattices, coupled (the method) */
    LBM_FLOW_SHEAR = 1     /* the interface lattice alone in the imposed shear flow of Sec. 6.1,
                              u_x = -U_0 pi cos(pi (x/nx - 1/2)) sin(pi (y/ny - 1/2)),
                              u_y =  U_0 pi sin(pi (x/nx - 1/2)) cos(pi (y/ny - 1/2)),
                              reversed (both signs) for time levels t >= reverse_step when
                              reverse_step > 0.  The fluid populations are not advanced and their
                              content is unspecified; lbm_get_fields reports this u and p = 0.
                              LBM_FP64 / LBM_FP32 only. */
} lbm_flow;

/* Problem statement of one case (Secs. 2, 4-6 of the paper). */
typedef struct {
    int32_t nx, ny;                 /* nodes along x and y, 1 .. 65536 each */
    int32_t bc_x, bc_y;             /* lbm_bc for the x pair (left/right) and y pair (bottom/top) */
    double rho_a, rho_b;            /* densities of phase A (phi = 1) and phase B (phi = 0) */
    double mu_a, mu_b;              /* dynamic viscosities */
    double sigma0, dsigma_dT;       /* sigma(T) = sigma0 + dsigma_dT (T - T0) */
    double T0, gradT_x, gradT_y;    /* prescribed temperature T = T0 + gradT_x x + gradT_y y */
    double mobility, width;         /* M_phi and interface width W of the Allen-Cahn equation */
    double gx, gy, rho_ref;         /* body force F_ext = (rho - rho_ref) (gx, gy) */
    int32_t precision;              /* lbm_precision */
    int32_t device;                 /* CUDA device ordinal */
    void* stream;                   /* cudaStream_t for all work of the context */
    double store_scale_g, store_scale_f;  /* 16-bit storage scales; 0 = default */
    /* Further forms of the paper's cases; all zero gives the coupled cascaded step above. */
    int32_t bc_x_hi, bc_y_hi;       /* lbm_bc of the right (x = nx - 1) / top (y = ny - 1) side
                                       when it differs from bc_x / bc_y (which then name the
                                       left / bottom side); 0 = same as bc_x / bc_y.  A periodic
                                       axis is periodic on both sides. */
    int32_t collision;              /* lbm_collision */
    int32_t sigma_model;            /* lbm_sigma_model */
    double beta;                    /* Langmuir: Gibbs elasticity number */
    double psi0, gradpsi_x, gradpsi_y;   /* Langmuir: imposed psi = psi0 + gradpsi . x */
    int32_t flow;                   /* lbm_flow */
    int32_t reverse_step;           /* LBM_FLOW_SHEAR: time level from which the field reverses
                                       (<= 0: never) */
    double u0;                      /* LBM_FLOW_SHEAR: amplitude U_0 */
} lbm_params;

typedef struct lbm_ctx lbm_ctx;

/* Scalar diagnostics of the current state, accumulated in double on the device. */
typedef struct {
    double sum_phi;      /* sum over nodes of phi = sum_a f_a (global phase mass) */
    double sum_p;        /* sum over nodes of the corrected pressure p */
    double max_speed;    /* max over nodes of |u| */
    double dp_laplace;   /* mean p over r < r_in minus mean p over r > r_out about (xc, yc)
                            (periodic distances; compared as r^2 against r_in^2, r_out^2), 0 if
                            a region is empty */
    int64_t nonfinite;   /* nodes whose phi, p or u is NaN or Inf */
} lbm_diag;

/* Device bytes the state of a case needs (two ping-pong population buffers); for
 * lbm_create_with_buffer.  Returns LBM_OK, or LBM_ERR_ARG / LBM_ERR_PARAM. */
int lbm_state_bytes(const lbm_params* params, size_t* bytes);

/* Validate params, derive the per-case constants and allocate the state on params.device.
 * On success *out is a new context; on error *out is NULL. */
int lbm_create(const lbm_params* params, lbm_ctx** out);

/* As lbm_create, but the state lives in the caller's device buffer (16-byte aligned, at least
 * lbm_state_bytes bytes, on params.device); the caller keeps ownership. */
int lbm_create_with_buffer(const lbm_params* params, void* device_buffer, size_t bytes,
                           lbm_ctx** out);

/* Equilibrium initialisation from host nodal fields phi, p, ux, uy ([ny][nx] doubles): the
 * fluid populations take the central moments of the transformed Maxwellian (Sec. 3 Eq.
 * centralmomentsgeqcomponents), the interface populations those of Sec. 5 with the
 * M_phi theta n term zero.  Synchronises the stream.  Resets the step counter and clears a
 * device error recorded by earlier steps (LBM_ERR_TIMEOUT / LBM_ERR_INDEX), as do
 * lbm_init_fields_device, lbm_set_populations and lbm_load_state: they replace the state that
 * error made invalid. */
int lbm_init_fields(lbm_ctx* ctx, const double* phi, const double* p, const double* ux,
                    const double* uy);

/* As lbm_init_fields with device pointers (doubles on params.device); asynchronous. */
int lbm_init_fields_device(lbm_ctx* ctx, const double* phi, const double* p, const double* ux,
                           const double* uy);

/* Advance nsteps (>= 0) time steps (the update of Secs. 3 - 5 on every node) on params.stream,
 * asynchronous; launch errors are returned.  A run of two or more steps is, where the multi-step
 * kernel is enabled (lbm_set_persistent; by default with LBM_FP32 storage where the warp
 * segments have at least 3 rows) and the grid's warps fit on the device at once, one launch of
 * that kernel: every warp keeps its strip of columns
 * and segment of rows from step to step and waits, between steps, only for the warps of the
 * neighbouring strips and segments (a cooperative launch of one 12-warp block per SM; runs
 * longer than 65536 steps take several launches).  Otherwise it is issued as replays of CUDA
 * graphs of one launch per step: graphs of 32 launches while 32 or more steps are left, then
 * one graph for the even rest (2 .. 30 launches); the first call that needs a graph builds all
 * of them (every even size up to 32, from either state buffer; a few milliseconds), so later
 * calls of any length launch at once; lbm_set_launch drops them, lbm_set_graphs switches them
 * off.  A last odd step is a single launch.  lbm_get_step_path tells which form a run takes.
 * Every form computes the same values, bit for bit. */
int lbm_step(lbm_ctx* ctx, int32_t nsteps);

/* Enable (default) or disable the graph replays of lbm_step; results are identical. */
int lbm_set_graphs(lbm_ctx* ctx, int32_t enable);

/* The multi-step kernel of lbm_step: enable = 1 uses it wherever the grid's warps fit on the
 * device at once, 0 never, 2 (automatic) where they fit and the warp segments are at least 3
 * rows tall (shorter segments spend more of a step in the waits between steps).  Results are
 * identical.  Default: 2 with LBM_FP32 storage, 0 with the others (where it measured slower
 * than graph replays).  Other values: LBM_ERR_ARG. */
int lbm_set_persistent(lbm_ctx* ctx, int32_t enable);

/* How lbm_step issues a run of two or more steps under the current settings: *path receives
 * LBM_PATH_MULTI (one multi-step launch), LBM_PATH_GRAPHS (graph replays of one launch per step)
 * or LBM_PATH_SINGLE (one launch per step: graphs off, the bounds-checked kernel, or the first-
 * wait timeout injection).  LBM_ERR_ARG for NULL arguments. */
enum { LBM_PATH_SINGLE = 0, LBM_PATH_GRAPHS = 1, LBM_PATH_MULTI = 2 };
int lbm_get_step_path(lbm_ctx* ctx, int32_t* path);

/* Debugging aid standing in for a memory checker: run the following steps through a variant of
 * the step kernel that checks every global load, store and bulk copy of a step against the
 * bounds of the source and destination state buffers before doing it.  An access outside is
 * skipped and recorded; lbm_check (or the next synchronising call) then returns LBM_ERR_INDEX.
 * The arithmetic is the plain kernel's, so results are bitwise identical when nothing is out
 * of range; steps run as single launches (no graph replays), about a third slower (78 against
 * 59 us per step on the 2048 x 1024 drop impact, FP32).  Shared-memory
 * accesses are not checked.  Only the cascaded coupled step with the linear sigma(T) (no step
 * variant): LBM_ERR_UNSUPPORTED otherwise.  enable = 0 returns to the plain kernel.
 * enable = 2 is a self-test of the checker: the declared bounds of both buffers leave out
 * their last row (memory that is allocated, so nothing stray happens), every access there is
 * reported, and the step's results are invalid.  Other values: LBM_ERR_ARG. */
int lbm_set_checked(lbm_ctx* ctx, int32_t enable);

/* Fields of the current state into host arrays ([ny][nx] doubles): phi, the corrected p, u and
 * rho as defined by Sec. 4 Eq. hydrodynamicfields.  Any pointer may be NULL.  Synchronises. */
int lbm_get_fields(lbm_ctx* ctx, double* phi, double* p, double* ux, double* uy, double* rho);

/* The populations of the current state: g and f as [9][ny][nx] doubles each (decoded from /
 * encoded to the storage format).  Synchronises.  In FP32 / FP64 storage a state written back
 * steps exactly as the one read out.  The 16-bit modes re-derive each node's zeroth-moment
 * planes from the populations given, so there a write-back is exact to one 16-bit rounding of
 * the deviations; use lbm_save_state / lbm_load_state for exact checkpoints. */
int lbm_get_populations(lbm_ctx* ctx, double* g, double* f);
int lbm_set_populations(lbm_ctx* ctx, const double* g, const double* f);

/* Exact checkpoint: the current state buffer byte for byte (bytes = lbm_state_bytes / 2) and
 * the step counter, to / from caller-owned host memory.  Synchronises.  A loaded state steps
 * exactly as the saved one in every precision mode.  LBM_ERR_ARG if bytes differs. */
int lbm_save_state(lbm_ctx* ctx, void* host, size_t bytes, int64_t* steps);
int lbm_load_state(lbm_ctx* ctx, const void* host, size_t bytes, int64_t steps);

/* Device pointer of the current state, valid until the next lbm_step.  Element type double for
 * LBM_FP64, float for LBM_FP32, half / bfloat16 (encoded as above) for the 16-bit modes.
 * Layout: tiles of 32 columns, nstrips = ceil(nx / 32) per row, E elements per tile (E = 576 for
 * FP32 / FP64, 704 for the 16-bit modes).  Population a (0..8 fluid g-bar, 9..17 interface f) of
 * node (x, y) is element (y * nstrips + x / 32) * E + P0 + 32 a + x % 32 with P0 = 0 (FP32 /
 * FP64) or 128 (16-bit); in the 16-bit modes Z_g / Z_f of the node is the float at element
 * (y * nstrips + x / 32) * E + 2 (x % 32) + 64 L, L = 0 / 1.  *elements receives the element
 * count of one state buffer. */
int lbm_state_device(lbm_ctx* ctx, void** state, int32_t* nstrips, int64_t* elements);

/* Synchronise the stream and report LBM_ERR_TIMEOUT if any step since the state was last set
 * (creation, lbm_init_fields*, lbm_set_populations, lbm_load_state) gave up on a bounded device
 * wait, LBM_ERR_INDEX if a checked step (lbm_set_checked) met an access outside the state
 * buffers; LBM_OK otherwise. */
int lbm_check(lbm_ctx* ctx);

/* Fault injection for tests of the failure path (no counterpart in the paper).  While enabled
 * with enable = 1, every step launch makes the first bounded shared-memory wait of each warp
 * give up at once, as if its row copy had never arrived: the warp records LBM_ERR_TIMEOUT in the
 * device error word, waits (with the normal bound) for the bulk copies it has in flight so that
 * none outlives the block, and returns without updating its nodes.  Steps run as single launches
 * of the plain step kernel then (the bounds-checked kernel of lbm_set_checked keeps its normal
 * waits).  With enable = 2, runs of two or more steps of a context with the multi-step kernel
 * enabled (lbm_set_persistent) go to it as usual, but its waits for the neighbouring warps
 * between steps never succeed: after the first step every warp waits out its bound (two
 * seconds), records LBM_ERR_TIMEOUT and returns, with no copy in flight.  Nothing faults or
 * hangs in either mode; the state of those steps is invalid, lbm_check reports LBM_ERR_TIMEOUT,
 * and re-initialising the state (lbm_init_fields*, lbm_set_populations, lbm_load_state) clears
 * the error.  enable = 0 (default) returns to normal waits; other values: LBM_ERR_ARG. */
int lbm_inject_timeout(lbm_ctx* ctx, int32_t enable);

/* Diagnostics of the current state; see lbm_diag.  r_in < 0 skips dp_laplace.  Synchronises.
 * Returns LBM_ERR_NONFINITE (with *out filled) when any node is non-finite. */
int lbm_diagnostics(lbm_ctx* ctx, double xc, double yc, double r_in, double r_out,
                    lbm_diag* out);

/* Tuning of the step launch: rows per warp segment (>= 1) and threads per block (a multiple of
 * 32, 32..256) of the one-launch-per-step kernels; the multi-step kernel takes the segment rows
 * and always runs blocks of 12 warps, one per SM.  0 keeps the current value.  Results do not
 * depend on these. */
int lbm_set_launch(lbm_ctx* ctx, int32_t seg_rows, int32_t block_threads);
int lbm_get_launch(lbm_ctx* ctx, int32_t* seg_rows, int32_t* block_threads);

/* Time steps taken since the last initialisation. */
int64_t lbm_steps_done(const lbm_ctx* ctx);

/* Release the context and the device memory it owns; NULL is allowed. */
void lbm_destroy(lbm_ctx* ctx);

/* Static message for a status code. */
const char* lbm_strerror(int status);

/* The last CUDA error code the context saw (cudaError_t as int), 0 if none. */
int lbm_last_cuda_error(const lbm_ctx* ctx);

/* Allocation-free variant of the diagnostics reduction (the paper has no counterpart; this is a
 * service entry point).  It serves callers that must not allocate device memory at this point:
 * code running while a CUDA graph is being captured (cudaMalloc is not capturable), real-time or
 * embedded loops that pre-size every buffer, and hosts whose allocator is owned by another
 * framework.  Unlike lbm_diagnostics it needs no context and allocates nothing: the per-block
 * partial sums go to a fixed device array inside the library (4097 x 8 doubles, 262 KB, held by
 * every GPU that loads the library until the process exits).
 *
 * Inputs: device arrays phi, p, ux, uy of nx * ny doubles, row-major [ny][nx] (for instance
 * the fields lbm_get_fields returns, copied to the device), the boundary kinds of the two axes
 * (lbm_bc, used for periodic distances) and the Laplace regions as in lbm_diagnostics.
 * Output: *out, an lbm_diag in DEVICE memory, written asynchronously on `stream` (cudaStream_t,
 * NULL = legacy default stream); read it after synchronising.  The call itself does not
 * synchronise and does not report LBM_ERR_NONFINITE: inspect out->nonfinite.
 * Limit: nx * ny <= 8,388,608 nodes (4096 partial blocks of 2048 nodes); larger grids return
 * LBM_ERR_ARG.  The first call on a device looks up the array's device address with the device
 * current (make that first call before any stream capture begins); the address is cached per
 * device ordinal (0..63) together with the identity of the device's current CUDA context, and
 * looked up again when that context changes (for instance after cudaDeviceReset).  Every call
 * reuses the same array: calls that overlap on the GPU (on different streams, or on other host
 * threads) race and give wrong results; serialise them.  Each call writes every partial slot it
 * reads, so nothing needs clearing between calls.  Errors: LBM_ERR_ARG as above, LBM_ERR_CUDA if
 * the set-up or a launch fails; a CUDA error the caller left pending before the call is neither
 * reported nor cleared by it. */
int lbm_diagnostics_noalloc(const double* phi, const double* p, const double* ux,
                            const double* uy, int32_t nx, int32_t ny, int32_t bc_x, int32_t bc_y,
                            double xc, double yc, double r_in, double r_out, lbm_diag* out,
                            void* stream);

/* ---------------------------------------------------------------------------------------------
 * Batches: many independent cases (any mix of grid sizes, boundaries and physical parameters)
 * advanced together.  Every lbm_batch_step advances all cases by one time step with ONE launch
 * of the batched step kernel (each warp takes one strip x segment task of one case from a
 * flattened task list); runs of two or more steps are replays of CUDA graphs as in lbm_step.
 * The per-node arithmetic
 * is the one of lbm_step.  A warp owns strips of 64 columns (32 in FP64), so a case whose width
 * is not a multiple of that leaves lanes idle; lbm_batch_create therefore stores each case in
 * the orientation whose padded strips cover fewer nodes (LBM_BATCH_FEWEST_COLUMNS): a case
 * stored transposed is stepped as its problem reflected across the diagonal (grid, boundary
 * kinds, gradients and body force with x and y exchanged), whose solution the D2Q9 scheme of
 * Secs. 3 and 5 maps onto the reflected one.  All fields and populations are passed in the
 * case's own orientation; the transposes run on the host in those calls.  A case stored as
 * given evolves bitwise as in its own context; a transposed one agrees with it up to the
 * rounding of the reflected evaluation order.
 * ------------------------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;

/* Orientation policy of lbm_batch_create_ex. */
typedef enum {
    LBM_BATCH_AS_GIVEN = 0,        /* every case as given: bitwise as in its own context */
    LBM_BATCH_FEWEST_COLUMNS = 1   /* per case, the orientation with fewer padded columns */
} lbm_batch_layout;

/* params: array of ncases (>= 1) cases; precision, device and stream must be equal in all of
 * them.  One device allocation holds every case's two state buffers (zeroed).  Cases may mix
 * grid sizes, boundary kinds and physical parameters; they must share the collision model
 * (cascaded, Secs. 3-5, or single relaxation time, Sec. 7) and the sigma law (linear in T, or
 * the Langmuir isotherm of Sec. 6.7): LBM_ERR_ARG otherwise.  The imposed flow
 * (LBM_FLOW_SHEAR) is not batched: LBM_ERR_UNSUPPORTED.  The 16-bit storage modes take the
 * cascaded step with the linear sigma(T) only, as in lbm_create. */
int lbm_batch_create(const lbm_params* params, int32_t ncases, lbm_batch** out);

/* As lbm_batch_create with the orientation policy `layout` (lbm_batch_layout; lbm_batch_create
 * takes LBM_BATCH_FEWEST_COLUMNS); other values: LBM_ERR_ARG.  Ties keep the case as given. */
int lbm_batch_create_ex(const lbm_params* params, int32_t ncases, int32_t layout,
                        lbm_batch** out);

/* 1 if case c is stored transposed, 0 if as given; LBM_ERR_ARG for a bad batch or index. */
int lbm_batch_case_transposed(const lbm_batch* b, int32_t c);

/* Equilibrium initialisation of case c from host fields ([ny][nx] doubles of that case), as
 * lbm_init_fields.  Synchronises. */
int lbm_batch_init_fields(lbm_batch* b, int32_t c, const double* phi, const double* p,
                          const double* ux, const double* uy);

/* Advance every case by nsteps (>= 0) time steps; asynchronous on the batch's stream. */
int lbm_batch_step(lbm_batch* b, int32_t nsteps);

/* Fields / populations of case c, as lbm_get_fields / lbm_get_populations.  Synchronise. */
int lbm_batch_get_fields(lbm_batch* b, int32_t c, double* phi, double* p, double* ux,
                         double* uy, double* rho);
int lbm_batch_get_populations(lbm_batch* b, int32_t c, double* g, double* f);

/* Launch shape: rows per warp task (>= 1) and threads per block (multiple of 32, <= 256);
 * 0 keeps the current value.  Results do not depend on it. */
int lbm_batch_set_launch(lbm_batch* b, int32_t seg_rows, int32_t block_threads);
int lbm_batch_get_launch(const lbm_batch* b, int32_t* seg_rows, int32_t* block_threads);

/* The batched multi-step kernel: with enable = 1, lbm_batch_step issues a run of two or more
 * steps as one cooperative launch (runs longer than 65536 steps take several) of one 12-warp
 * block per SM, whose warps share the batch's warp tasks out once, balanced by nodes, and take
 * their tasks in a fixed order every step; a task waits, before its step, only for the tasks of
 * the same case within reach of its reads and writes.  enable = 0 (default): graph replays of
 * one launch per step.  The results are the same, bit for bit.  Other values: LBM_ERR_ARG.
 * lbm_batch_get_step_path: LBM_PATH_MULTI where the multi-step kernel takes the runs (enabled,
 * and its warps fit on the device at once), else LBM_PATH_GRAPHS. */
int lbm_batch_set_persistent(lbm_batch* b, int32_t enable);
int lbm_batch_get_step_path(const lbm_batch* b, int32_t* path);

/* Autotuner: times trial_steps (>= 1) steps of the live batch for each candidate launch shape
 * (rows per task 8..64, blocks of 64 or 128 threads), keeps the fastest and restores the state
 * it started from (a temporary device copy).  Synchronises. */
int lbm_batch_tune(lbm_batch* b, int32_t trial_steps, int32_t* seg_rows, int32_t* block_threads);

/* Total nodes of all cases; LBM_ERR_TIMEOUT check as lbm_check; release (NULL allowed). */
int64_t lbm_batch_nodes(const lbm_batch* b);
int lbm_batch_check(lbm_batch* b);
void lbm_batch_destroy(lbm_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* CMLBM_H */
