/*
 * lbm.h - C ABI of the GB300 (sm_103a) chemical-potential multiphase lattice
 * Boltzmann library.
 *
 * Method: Qin, Chen, Qin, Xu, Wen, "Spurious currents suppression by accurate
 * difference schemes in multiphase lattice Boltzmann method".  One time step
 * evaluates the bulk chemical potential from the equation of state (Eq. 10-13,
 * 16), adds the density-Laplacian term (Eq. 11, 16), takes grad mu and grad
 * rho with a selectable difference scheme (Eq. 17-25), forms the nonideal
 * force F = -rho grad mu + c_s^2 grad rho (Eq. 12), applies single-relaxation
 * (BGK) collision with exact-difference forcing (Eq. 1, 6, 8) and streams
 * (Eq. 1, left side) on a periodic D2Q9 or D3Q19 lattice.
 *
 * Conventions
 *  - Lattice units: dx = dt = c = 1, c_s^2 = 1/3.  Node (x, y, z) has linear
 *    index x + nx*(y + ny*z) (x fastest).  Fields are structure-of-arrays:
 *    population i of node n at f[i*N + n], N = nx*ny*nz.
 *  - D2Q9 velocity order is that of Eq. 2 (rest; +x, +y, -x, -y; (1,1),
 *    (-1,1), (-1,-1), (1,-1)).  D3Q19 order: rest; +x, -x, +y, -y, +z, -z;
 *    (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1),
 *    (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1).
 *  - All functions return 0 on success or a negative LBM_E* code; no call
 *    falls back to the CPU.  Host arrays passed in are borrowed for the
 *    duration of the call only.  Calls on one handle are not thread-safe;
 *    distinct handles are independent.
 *  - Device work is enqueued on the stream given at creation; functions that
 *    return host data synchronise that stream.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define LBM_OK 0
#define LBM_EINVAL -1     /* invalid argument or parameter combination */
#define LBM_ENOMEM -2     /* the allocator returned NULL */
#define LBM_ECUDA -3      /* a CUDA runtime call failed */
#define LBM_EUNSTABLE -4  /* a density became non-positive or NaN; see lbm_obs.step
                           (step 0 is also recorded when a tensor-copy wait of the
                           D3Q19 FP32DEV collision pass runs out, after ~1 s) */
#define LBM_ETIMEOUT -5   /* a bounded device-side wait gave up */
#define LBM_ENOTSUP -6    /* combination not provided (e.g. E8 on D3Q19) */
#define LBM_ESCRATCH -7   /* larger than the fixed scratch of lbm_observables_noalloc */

/* ---- enumerations ---- */
#define LBM_D2Q9 0
#define LBM_D3Q19 1

#define LBM_EOS_CS 0 /* Carnahan-Starling */
#define LBM_EOS_PR 1 /* Peng-Robinson, Eq. 14 with the chemical potential of Eq. 15 */
#define LBM_EOS_VDW 2 /* van der Waals, chemical potential by Eq. 13 */
#define LBM_EOS_RKS 3 /* Redlich-Kwong-Soave, chemical potential by Eq. 13 */

/* difference schemes (Sec. 2.3) */
#define LBM_EFDS2 0  /* Eq. 18, second-order central */
#define LBM_EFDS4 1  /* Eq. 19 */
#define LBM_EFDS6 2  /* Eq. 20 */
#define LBM_CFDS4 3  /* Eq. 22, Pade; periodic tridiagonal line solves */
#define LBM_CFDS6 4  /* Eq. 23 */
#define LBM_CFDS8 5  /* Eq. 24 */
#define LBM_OCFDS4 6 /* Sec. 3.1 optimal fourth-order compact, alpha = 0.446776, c = -0.0541132 */
#define LBM_E4 7     /* Eq. 25, fourth-order isotropic */
#define LBM_E8 8     /* Eq. 25, eighth-order isotropic (D2Q9 only) */

/* collision operator */
#define LBM_BGK 0 /* single relaxation: the MRT operator with every rate 1/tau (Sec. 2.1, after Eq. 5) */
#define LBM_MRT 1 /* Eq. 1 with M of Eq. 3 and S of Eq. 5 (D2Q9 only) */

/* storage precision */
#define LBM_FP64 0    /* populations, density and all arithmetic in FP64 */
#define LBM_FP32DEV 1 /* populations stored in FP32 as f_i - w_i rho_ref, density as rho - rho_ref */

/*
 * Simulation parameters.
 *  lattice   LBM_D2Q9 (nz must be 1) or LBM_D3Q19
 *  nx,ny,nz  periodic lattice size; each >= 8 (D2Q9: nx, ny >= 8)
 *  eos       LBM_EOS_CS, LBM_EOS_PR, LBM_EOS_VDW or LBM_EOS_RKS (VDW: p0 = rho R T /
 *            (1 - b rho) - a rho^2; RKS: p0 = rho R T / (1 - b rho) - a alpha(T) rho^2 /
 *            (1 + b rho), alpha = [1 + (0.480 + 1.574 w - 0.176 w^2)(1 - sqrt(Tr))]^2)
 *  a,b,R     CS constants: p0 = rho R T (1+eta+eta^2-eta^3)/(1-eta)^3 - a rho^2, eta = b rho/4;
 *            PR constants of Eq. 14 (the paper's: a = 2/49, b = 2/21, R = 1)
 *  Tr        reduced temperature T/T_c (T_c computed from a, b, R), 0 < Tr (PR, RKS: Tr < 1)
 *  k         proportional coefficient of Eq. 16 (mu-hat = k^2 psi' - kappa lap rho)
 *  kappa     kappa-hat of Eq. 16
 *  tau       BGK relaxation time (> 0.5)
 *  scheme    LBM_EFDS2 .. LBM_E8
 *  precision LBM_FP64 or LBM_FP32DEV
 *  mu_fp64   FP32DEV only: evaluate the EOS chemical potential in FP64
 *            (slower on GB300, whose FP64 rate is a small fraction of FP32).
 *            D3Q19 with LBM_EFDS2/4/6: k^2 psi'(rho) in FP64 from rho_ref +
 *            the float deviation, the mu field then rounded to float for the
 *            stencils (3.5x the step time at 256^3); elsewhere mu and its
 *            gradient stay in FP64 in the kernels
 *  rho_ref   FP32DEV only: reference density of the stored deviations;
 *            <= 0 selects the Maxwell gas density at Tr
 *  collision LBM_BGK, or LBM_MRT (D2Q9; LBM_ENOTSUP on D3Q19)
 *  mrt_s     LBM_MRT: the rates s_1..s_9 of Eq. 5 in the row order of Eq. 3
 *            (rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx, p_xy); all zero
 *            selects the paper's (1, 1.64, 1.54, 1, 1.7, 1, 1.7, 1/tau, 1/tau).
 *            The rates of the conserved moments (s_1, s_4, s_6) have no effect.
 *  acentric  LBM_EOS_PR, LBM_EOS_RKS: the acentric factor w of alpha(T) (Eq. 15;
 *            the paper's water: 0.344)
 */
typedef struct {
  int lattice;
  int nx, ny, nz;
  int eos;
  double a, b, R, Tr;
  double k, kappa, tau;
  int scheme;
  int precision;
  int mu_fp64;
  double rho_ref;
  int collision;
  double mrt_s[9];
  double acentric;
} lbm_params;

/*
 * Observables at the current time step t (Sec. 3.3 and 3.4):
 *  max_v       max over nodes of |v|, v = u + F/(2 rho) (Sec. 2.1, after Eq. 8)
 *  max_u       max over nodes of |u|, u = sum e_i f_i / rho (Eq. 7)
 *  rho_center  rho at node (nx/2, ny/2, nz/2)
 *  rho_corner  rho at node (0, 0, 0)
 *  mass        sum of rho over all nodes (FP64)
 *  max_drho    max over nodes |rho(t) - rho(t0)| / (t - t0), t0 the time of the
 *              previous lbm_observables call (or of initialisation); 0 if t == t0
 *  step        t; for status LBM_EUNSTABLE the first step at which a
 *              non-positive or NaN density was seen
 *  status      LBM_OK or LBM_EUNSTABLE
 */
typedef struct {
  double max_v, max_u, rho_center, rho_corner, mass, max_drho;
  long long step;
  int status;
} lbm_obs;

/*
 * Device-memory allocator supplied by the caller (for example one backed by a
 * framework's caching allocator).  alloc returns a device pointer aligned to
 * at least 256 bytes or NULL; free releases it.  If the allocator argument of
 * lbm_create is NULL the library uses cudaMalloc / cudaFree.
 */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* ctx);
  void* ctx;
} lbm_allocator;

typedef struct lbm_handle lbm_handle;

/* Create a simulation.  stream: a cudaStream_t (NULL = legacy default
 * stream) on the current device, on which all work of this handle runs.
 * The handle owns every device buffer it allocates through `alloc`.
 * Errors: LBM_EINVAL (bad parameters), LBM_ENOTSUP, LBM_ENOMEM, LBM_ECUDA. */
int lbm_create(const lbm_params* params, void* stream, const lbm_allocator* alloc, lbm_handle** out);

/* Release all device memory of the handle (after synchronising its stream). */
void lbm_destroy(lbm_handle* h);

/* Initialise a droplet by Eq. 26: rho = (rho_l+rho_g)/2 - (rho_l-rho_g)/2
 * tanh(2 (r - radius)/width), r = Euclidean distance to center (no periodic
 * image); center NULL = node (nx/2, ny/2, nz/2); rho_l or rho_g <= 0 selects
 * the Maxwell coexistence densities.  Populations start at equilibrium with
 * u = 0.  Resets the step counter and status. */
int lbm_init_droplet(lbm_handle* h, const double center[3], double radius, double width, double rho_l,
                     double rho_g);

/* Flat liquid slab of the given thickness centred on the mid-plane of axis
 * (0 = x, 1 = y, 2 = z) with a tanh interface of the given width (the
 * coexistence test of Sec. 3.4). */
int lbm_init_slab(lbm_handle* h, int axis, double thickness, double width, double rho_l, double rho_g);

/* Radial profile: rho(node) is linearly interpolated in r between samples
 * (r[j], rho[j]), j < n, r strictly increasing, held at the end values
 * outside [r[0], r[n-1]]. */
int lbm_init_profile(lbm_handle* h, const double center[3], const double* r, const double* rho, int n);

/* Arbitrary initial density field: host_rho[N] (FP64, all > 0), u = 0. */
int lbm_init_density(lbm_handle* h, const double* host_rho);

/* Set all populations from host FP64 f[Q*N] (full values, not deviations).
 * Resets the step counter. */
int lbm_set_f(lbm_handle* h, const double* host_f);

/* Chemical-potential wall boundary (Appendix A).  mask[N] (node order x
 * fastest, then y, then z): nonzero marks a wall node.  Wall nodes reached by
 * a fluid stencil are layered by their link distance to the fluid (layers
 * 1..3); every step their densities are set, layer by layer, to the
 * w_i-weighted average of the neighbours in the layer before (Eq. A.1), all
 * wall nodes carry the chemical potential mu_w in the force of Eq. 12, fluid
 * populations streaming into a wall return reversed to their node (halfway
 * bounce-back), and wall nodes neither collide nor count in the observables.
 * The wall step runs as node-parallel passes (several launches per step) on
 * the explicit schemes LBM_EFDS2/4/6 only: other schemes -> LBM_ENOTSUP.
 * mask NULL removes the walls.  The populations of wall nodes are undefined;
 * after lbm_step the density field holds the Eq. A.1 wall densities of the
 * state.  The mask is copied (host memory, read only); synchronises the
 * stream.  Errors: LBM_EINVAL (no fluid node, mu_w not finite), LBM_ENOTSUP,
 * LBM_ENOMEM, LBM_ECUDA. */
int lbm_set_solid(lbm_handle* h, const unsigned char* mask, double mu_w);

/* Advance n >= 0 time steps; asynchronous on the handle's stream.  The same
 * handle parameters, initial state and n give the same bits on every run:
 * where several thread blocks contribute to one node's next density, their
 * partial sums are combined in an order-independent way (two floating-point
 * additions onto zero, or exact 64-bit fixed-point additions). */
int lbm_step(lbm_handle* h, long long n);

/* As lbm_step (n <= 100000), timing every step on the handle's stream with
 * CUDA events recorded between the launches; synchronises once at the end.
 * ms[3] receives the summed
 * milliseconds of the mu pass (0 when the step is a single fused kernel), of
 * the collision/streaming pass (the whole step when fused), and of both. */
int lbm_step_timed(lbm_handle* h, long long n, double* ms);

/* Observables of the current state (synchronises the stream).  Returns
 * LBM_EUNSTABLE (and fills out->status, out->step) once a non-positive or
 * NaN density has been seen. */
int lbm_observables(lbm_handle* h, lbm_obs* out);

/* Advance n >= 1 time steps and return the observables of the state the last
 * of them started from (step lbm_get_step() - 1 afterwards), as
 * lbm_observables would have returned them before that step, within FP32
 * rounding.  On the split D3Q19 FP32-deviation path (EFDS2/4/6) the last step
 * computes them in its collision pass (u, F and rho are at hand there), so an
 * observed step costs one step plus a small reduction instead of a step and a
 * separate observation pass; elsewhere it observes, then steps.  Synchronises
 * the stream.  Returns LBM_EUNSTABLE as lbm_observables does.  (A performance
 * entry point; the paper's method has no counterpart.) */
int lbm_step_observe(lbm_handle* h, long long n, lbm_obs* out);

/* As lbm_step_observe without synchronising the stream: the observables are
 * reduced and packed on the device and copied to *out by the handle's stream,
 * so consecutive calls queue their steps back to back.  out: host memory
 * (page-locked for the copy to be asynchronous) or device memory, at least
 * sizeof(lbm_obs) bytes; valid once the stream has been synchronised (for
 * example by the next synchronising call); out->status and out->step report
 * instability (LBM_EUNSTABLE and the first bad step).  Returns LBM_OK once the
 * work is queued (LBM_EINVAL, LBM_ECUDA otherwise).  (A performance entry
 * point; the paper's method has no counterpart.) */
int lbm_step_observe_async(lbm_handle* h, long long n, lbm_obs* out);

/* Copy the density field rho[N] (FP64) to host memory (synchronises). */
int lbm_get_density(lbm_handle* h, double* host_rho);

/* Copy the populations as full FP64 values f[Q*N] to host memory. */
int lbm_get_f(lbm_handle* h, double* host_f);

/* Nonideal force F[dim*N] (component-major) and chemical potential mu[N] of
 * the current state, FP64 on the host; either pointer may be NULL. */
int lbm_get_force(lbm_handle* h, double* host_F, double* host_mu);

/* Current step counter. */
long long lbm_get_step(const lbm_handle* h);

/* Device pointers of the current populations and density field (for callers
 * that keep data on the GPU).  Stored forms: LBM_FP64 f and rho as double;
 * LBM_FP32DEV f_i - w_i rho_ref and rho - rho_ref as float.  Valid until the
 * next lbm_step. */
int lbm_device_state(lbm_handle* h, void** f, void** rho);

/* Work decomposition.  D3Q19 FP32DEV step (explicit schemes, and the
 * compact schemes' collision pass when nx % 4 == 0): each CTA
 * marches through a chunk of zc planes; lbm_set_zchunk fixes zc (0 = the
 * built-in heuristic, which balances the last wave of CTAs against the
 * per-chunk prologue).  D2Q9 FP32DEV split step (explicit and isotropic
 * schemes, no walls): tiles of 16 x rows-per-thread rows; lbm_set_tile_rows
 * fixes rows per thread (1, 2 or 4; 0 = 2).  lbm_autotune times the
 * candidates on this handle's lattice and keeps the fastest: chunk lengths
 * over a few steps each, tile rows in three interleaved rounds of ten steps
 * (each shape's fastest round counting); the steps run on the handle's
 * state, which is left undefined (initialise after tuning).  *zc_out
 * receives the choice (the z chunk, or the tile rows per thread), 0 if the
 * handle has nothing to tune.  The choices give identical results. */
int lbm_set_zchunk(lbm_handle* h, int zc);
int lbm_set_tile_rows(lbm_handle* h, int rows_per_thread);
int lbm_autotune(lbm_handle* h, int* zc_out);

/* Carnahan-Starling critical point for constants (a, b, R), solving
 * dp0/drho = d2p0/drho2 = 0. */
int lbm_critical(double a, double b, double R, double* rho_c, double* T_c);

/* Maxwell equal-area coexistence densities for params->(a, b, R, Tr):
 * equal chemical potential and pressure in both bulk phases. */
int lbm_maxwell(const lbm_params* params, double* rho_g, double* rho_l);

/* Bulk chemical potential k^2 psi'(rho) of the EOS that p selects at
 * T = Tr T_c, with the additive constant the step's mu (Eq. 16) uses: the mu
 * of a uniform fluid of density rho.  For choosing the wall chemical
 * potential of lbm_set_solid relative to the saturation value
 * lbm_bulk_mu(p, rho_g) (Appendix A).  Host only.  Errors: LBM_EINVAL (rho
 * outside (0, the EOS's packing limit), bad parameters). */
int lbm_bulk_mu(const lbm_params* p, double rho, double* mu);

/* Critical density and temperature of the EOS that p selects (p0' = p0'' = 0;
 * for Peng-Robinson with alpha = 1, which holds at T_c).  Host only.  (A
 * companion of lbm_critical, which keeps its Carnahan-Starling signature.) */
int lbm_eos_critical(const lbm_params* p, double* rho_c, double* T_c);

/* Equilibrium flat interface (Eq. 29) along one axis for the EOS, T_r, k and
 * kappa-hat of p: rho[n] and, if drho is not NULL, drho/dy[n] at nodes
 * j = 0..n-1 (lattice units), gas for j < y0, liquid beyond, rho(y0) =
 * (rho_g + rho_l) / 2.  Uniform mu-hat (Eq. 16) gives the first integral
 * (kappa-hat / 2) rho'^2 = k^2 [rho (psi'(rho) - psi'(rho_g)) - (p0(rho) - p0(rho_g))],
 * integrated numerically (~1e-10).  The analytic reference of Sec. 3.1 (Fig. 3);
 * host only; fill a slab with it through lbm_init_density. */
int lbm_flat_profile(const lbm_params* p, int n, double y0, double* rho, double* drho);

/* Force-direction error of Sec. 3.2 (Eq. 30) on the current state: for nodes
 * with |F| >= frac max|F| (F of Eq. 12), the angle between F and the line
 * from center (NULL: the lattice centre node) through the node, atan2(|F x r|,
 * |F . r|) in radians (Eq. 30's atan gives the direction modulo pi; this is
 * its absolute value, in any dimension).  out[0] = max angle, out[1] =
 * |F|-weighted mean angle, out[2] = number of nodes.  Synchronises. */
int lbm_force_angle(lbm_handle* h, const double center[3], double frac, double out[3]);

/* Lattice size Q (9 or 19) of a lattice id, 0 if unknown. */
int lbm_lattice_q(int lattice);

/* Static text for an error code. */
const char* lbm_strerror(int code);

/* ====================================================== no device allocation
 * Observables (as lbm_observables) of a state the caller holds in its own
 * device buffers, computed without allocating any device memory.  For callers
 * that cannot let a library allocate: an application that owns all device
 * memory under a fixed budget, or code running where a new cudaMalloc would
 * stall or fail.  The paper has no counterpart; it is an interface choice.
 *
 *  p                 the parameters the state was produced with (explicit and
 *                    isotropic schemes only: compact schemes -> LBM_ENOTSUP;
 *                    a state without walls: the pass has no wall mask, so
 *                    the wall nodes of a lbm_set_solid state would enter the
 *                    mass and the velocity maxima)
 *  d_f, d_rho        device pointers to the populations and density field in
 *                    the stored form of lbm_device_state (read only)
 *  d_rho_prev        density field of an earlier step (stored form) for
 *                    max_drho, or NULL (max_drho = 0)
 *  steps_since_prev  steps between d_rho_prev and d_rho (max_drho divisor)
 *  step              step index reported back in out->step
 *  stream            cudaStream_t the work is ordered on (synchronised)
 *
 * The reduction's partial results live in a fixed file-scope device array of
 * 65536 x 4 doubles plus 16 result words (about 2 MiB), held by every GPU that
 * loads the library until the process exits.  Lattices whose observation pass
 * needs more than 65536 CTAs (D2Q9 above about 16.7 M nodes) return
 * LBM_ESCRATCH.  On D3Q19 the node limit of 2^31 / 19 (about 113 M nodes,
 * 32-bit population indexing; LBM_EINVAL) comes first, except for very thin
 * lattices (a few nodes across x and y, millions along z).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for that device; make that first call
 * before any stream capture.  After a cudaDeviceReset the library is not
 * usable on that device again in the same process.  All calls share the array and it keeps the last
 * call's contents: calls that overlap on the GPU race and must be serialised.
 * Returns LBM_OK, or LBM_EUNSTABLE (out->status too) if a density is
 * non-positive or NaN. */
int lbm_observables_noalloc(const lbm_params* p, const void* d_f, const void* d_rho, const void* d_rho_prev,
                            long long steps_since_prev, long long step, void* stream, lbm_obs* out);

/* ==================================================================== batches
 * Many independent D2Q9 droplets of different sizes and parameters advanced
 * together (the parameter sweeps of Sec. 3.3-3.4 run as one job).  All cases
 * must share lattice (LBM_D2Q9), precision and mu_fp64; schemes may differ
 * freely, the compact ones included (Eq. 21-24 and OCFDS4 of Sec. 3.1: their
 * steps add a chemical-potential phase where the precision needs one, and a
 * phase of periodic tridiagonal line solves along x and y, groups of lines
 * being work items of the same launch, each phase behind the barrier).  Each
 * case owns its own populations and density; lbm_batch_step runs n steps of
 * every case in ONE persistent kernel launch whose resident CTAs fetch
 * (case, tile) work items dynamically and meet at a device-wide barrier
 * between steps; the launch is captured in a CUDA graph (one per distinct n)
 * and replayed.  Barrier waits are bounded (about one second): if a wait runs
 * out the kernel returns and lbm_batch_observables reports LBM_ETIMEOUT.
 */
typedef struct lbm_batch lbm_batch;

/* cases[n] as for lbm_create; stream/alloc as for lbm_create. */
int lbm_batch_create(const lbm_params* cases, int n, void* stream, const lbm_allocator* alloc, lbm_batch** out);
void lbm_batch_destroy(lbm_batch* b);

/* Every case: droplet of Eq. 26 centred on node (nx/2, ny/2) with radius[c],
 * interface width `width` and its Maxwell densities; resets the step counter. */
int lbm_batch_init_droplets(lbm_batch* b, const double* radius, double width);

/* Advance every case by n steps (asynchronous on the batch stream). */
int lbm_batch_step(lbm_batch* b, long long n);

/* Observables of every case into out[n] (lbm_obs as above; synchronises).
 * Returns LBM_ETIMEOUT if a barrier wait of the last launch ran out;
 * per-case instability is reported in out[c].status without failing. */
int lbm_batch_observables(lbm_batch* b, lbm_obs* out);

/* Density field of case c (nx*ny FP64) to host memory (synchronises). */
int lbm_batch_get_density(lbm_batch* b, int c, double* host_rho);

long long lbm_batch_get_step(const lbm_batch* b);

/* Sizes: number of cases, of (case, tile) work items and of resident CTAs. */
int lbm_batch_size(const lbm_batch* b, int* ncases, int* nitems, int* grid);

/* Failure-detection aid for tests: CTA `cta` (0 <= cta < grid) will leave at
 * its first barrier without arriving, so the others' bounded waits run out;
 * -1 clears the injection and the error status. */
int lbm_batch_inject_stall(lbm_batch* b, int cta);

/* Tile shape of the FP32-deviation batch kernel: collision tiles of
 * 30 x (16 rows - 2) and mu tiles of 32 x 16 rows, rows = 16 x (rows per
 * thread), rows per thread 1, 2 (default) or 4.  lbm_batch_set_tiles fixes
 * it; lbm_batch_autotune times `steps` steps of every shape that has a
 * resident launch configuration (after one captured warm-up launch each), in
 * three interleaved rounds, and keeps the shape with the fastest launch,
 * reported in *rows_out (18 launches of `steps` steps).  The tuning steps run on the
 * batch's state, which they advance: initialise before tuning (the timing
 * is only representative of a physical state) and again after it.  The shapes
 * give identical results (same arithmetic per node).  Errors: LBM_EINVAL,
 * LBM_ENOTSUP (not an FP32-deviation batch), LBM_ECUDA. */
int lbm_batch_set_tiles(lbm_batch* b, int rows_per_thread);
int lbm_batch_autotune(lbm_batch* b, int steps, int* rows_out);

/* ================================================================ warm start
 * A small fully connected network (FP32; GELU hidden layers, linear output)
 * that maps droplet parameters to an initial radial density profile, trained
 * by Adam on profiles the solver itself produced.  The paper has no
 * counterpart: it only seeds lbm_init_profile, and the solver relaxes the
 * state from there.  Parameters are packed per layer as W (out x in,
 * row-major) followed by b.  Layers are at most 128 wide, at most 8 deep.
 * Host arrays are row-major, one sample per row.
 */
typedef struct lbm_mlp lbm_mlp;

/* sizes[0..nlayers]: widths from input to output; max_batch: the largest
 * batch (and data set) used with this handle. */
int lbm_mlp_create(const int* sizes, int nlayers, int max_batch, void* stream, const lbm_allocator* alloc,
                   lbm_mlp** out);
void lbm_mlp_destroy(lbm_mlp* m);
long long lbm_mlp_param_count(const lbm_mlp* m);

/* Copy parameters in (resets the Adam state) or out (FP32, packed). */
int lbm_mlp_set_params(lbm_mlp* m, const float* host_params);
int lbm_mlp_get_params(lbm_mlp* m, float* host_params);

/* y[batch x out] = network(x[batch x in]). */
int lbm_mlp_forward(lbm_mlp* m, const float* host_x, int batch, float* host_y);

/* Mean-squared-error loss over batch x out entries and its gradient with
 * respect to every parameter (same packing); either output may be NULL. */
int lbm_mlp_loss_grad(lbm_mlp* m, const float* host_x, const float* host_t, int batch, float* host_loss,
                      float* host_grad);

/* Keep a training set of n samples on the device. */
int lbm_mlp_set_data(lbm_mlp* m, const float* host_x, const float* host_t, int n);

/* iters full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, step size
 * lr) on the stored data; *host_loss (may be NULL) receives the loss of the
 * last evaluated parameters. */
int lbm_mlp_train(lbm_mlp* m, int iters, float lr, float* host_loss);


#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
