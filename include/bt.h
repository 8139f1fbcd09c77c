/*
 * bt.h -- C ABI of the GB300 discrete-ordinate neutrino transport step.
 *
 * Implements one time step of the Boltzmann transport scheme of Chan &
 * Mueller, "A Novel Multi-Dimensional Boltzmann Neutrino Transport Scheme
 * for Core-Collapse Supernovae" (arXiv:2003.02845): the distribution
 * f(r, theta, eps, mu, Phi) of each species is advanced by
 *   (Sec. 3.2, Eq. transformation)  a time remap of every zone from the old
 *        background's comoving frame to the new one (Lorentz boost, conformal
 *        frame change, Hamiltonian kick);
 *   (Sec. 3.3, Eq. fullstep, Eq. halfstep) unsplit interface fluxes on every
 *        radial, polar and azimuthal face: a locally implicit Lax-Wendroff
 *        half step blended with an MC-limited upwind state (Sec. 3.3.3), with
 *        the face and neighbour contents mapped between comoving frames by
 *        the conservative trilinear remap T (Sec. 3.2);
 *   (Sec. 3.5) the local implicit absorption/emission/isotropic-scattering
 *        solve per zone and energy group (Sherman-Morrison form);
 *   (Sec. 3.4, Eq. hydrosource) the number/energy/momentum source terms.
 * Every step runs in CUDA kernels built for sm_103a; there is no CPU path.
 *
 * Conventions
 *   Units: c = 1; lengths and dt in the same length unit; kappa per length.
 *   Zones: zone = b * n_r + a (a radial, b polar).
 *   Angles: ang = j * n_phi + k (mu index j over the mu nodes in ascending
 *           order, Phi index k with centres (k + 1/2) 2pi/n_phi).
 *   f layout: f[s][zone][group][ang], float64 (BT_FP64) or float32 (BT_MIXED).
 *   Opacity layout: [s][zone][group]; vectors [zone][3] as (r, theta, phi)
 *           components in the zone's local orthonormal triad.
 *   Pointers: every array argument is a HOST pointer unless the argument
 *           `mem` says BT_MEM_DEVICE (then a device pointer on the handle's
 *           device).  The caller keeps ownership; the library copies.
 *   Streams: all device work is enqueued on bt_config.stream (a
 *           cudaStream_t, 0 = legacy default stream).  Calls that return data
 *           to host memory synchronise that stream.
 *   Errors: functions return BT_OK (0) or a negative BT_ERR_* code;
 *           bt_last_error() returns a thread-local message for the last
 *           failure.  No exception crosses the ABI.
 *   Threads: one handle must not be used by two host threads at once.
 */
#ifndef BT_H_
#define BT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  BT_OK = 0,
  BT_ERR_ARG = -1,        /* null pointer, bad size or unsupported configuration */
  BT_ERR_BACKGROUND = -2, /* NaN/Inf, alpha <= 0, phi <= 0, |v| >= 1, kappa < 0, shift != 0 */
  BT_ERR_DT = -3,         /* dt <= 0 or not finite */
  BT_ERR_CUDA = -4,       /* a CUDA runtime call failed (message has the CUDA error) */
  BT_ERR_NUMERIC = -5,    /* non-finite value produced by a step */
  BT_ERR_STATE = -6,      /* call order violated (e.g. step before a background) */
  BT_ERR_TIMEOUT = -7     /* a bounded device-side wait (asynchronous copy) gave up */
};

enum { BT_GEOM_SPHERICAL = 0, BT_GEOM_SLAB = 1 };
enum { BT_FP64 = 0, BT_MIXED = 1 };
enum { BT_MEM_HOST = 0, BT_MEM_DEVICE = 1 };
enum { BT_NUE = 0, BT_NUEBAR = 1, BT_NUX = 2 };
enum { BT_GAUSS_LEGENDRE = 0, BT_GAUSS_LOBATTO = 1 };

typedef struct bt_handle bt_handle;

/*
 * Problem description (Sec. 3.1, Discretisation).
 *  geom           BT_GEOM_SPHERICAL: flat-faced cells on spherical-polar vertices
 *                 (Sec. 3.1); a single periodic azimuthal wedge of width
 *                 dphi_wedge (Sec. 3.3.4).  If theta_periodic == 1 the grid is a
 *                 1D column (n_theta must be 1) centred on the equator with
 *                 periodic polar faces of width dtheta_column; otherwise the
 *                 polar range is [0, pi] split uniformly into n_theta >= 2 rows.
 *                 BT_GEOM_SLAB: plane-parallel z grid (r_edges are z edges),
 *                 unit face areas, open boundaries at both ends.
 *  r_edges        n_r + 1 increasing radii (host pointer, copied).  r_edges[0]
 *                 == 0 gives a zero-area inner face; r_edges[0] > 0 a
 *                 reflecting wall (spherical geometry).
 *  species_kind   n_species entries of BT_NUE/BT_NUEBAR/BT_NUX (host, copied).
 *  eps_edges      n_eps + 1 log-uniform group edges (constant ratio; host).
 *  n_mu, n_phi    angular grid: n_mu mu cells x n_phi uniform Phi cells.
 *  mu_quadrature  BT_GAUSS_LEGENDRE (0): mu nodes and cell widths are the
 *                 Gauss-Legendre nodes and weights.  BT_GAUSS_LOBATTO: the
 *                 Gauss-Lobatto ones (Sec. 3.1: cell widths equal to the
 *                 Gauss-Lobatto weights; Sec. 5: mu = 1 as a collocation
 *                 point), n_mu >= 2.  The nodes mu = -1 and +1 are then one
 *                 direction each, held by n_phi cells; content the remap
 *                 moves into such a pole node is spread evenly over its cells.
 *  theta_max      2D grids (theta_periodic == 0): the polar range is
 *                 [0, theta_max], split uniformly into n_theta rows; 0 means
 *                 pi.  Below pi the face at theta_max is an open boundary
 *                 (Sec. 4.5.2, the radiating disk): bins leaving the grid
 *                 through it are lost to the outflow tallies, and bins
 *                 entering take the distribution set by bt_set_boundary
 *                 (zero, i.e. vacuum, until set).
 *  precision      BT_FP64 or BT_MIXED (float32 f, fluxes and remap; float64
 *                 collision solve, content accumulators and sums).
 *  phase_norm     the 1/h^3 factor of the hydro source terms (Eq. hydrosource).
 *  stream         cudaStream_t for all work of this handle.
 */
typedef struct bt_config {
  int32_t geom;
  int32_t n_r, n_theta;
  const double* r_edges;
  int32_t theta_periodic;
  double dtheta_column;
  double dphi_wedge;
  int32_t n_species;
  const int32_t* species_kind;
  int32_t n_eps;
  const double* eps_edges;
  int32_t n_mu, n_phi;
  int32_t precision;
  double phase_norm;
  void* stream;
  int32_t mu_quadrature;
  double theta_max;
} bt_config;

/* Message of the last failed call on this host thread (never NULL). */
const char* bt_last_error(void);

/* Device bytes bt_create will use for this configuration (0 on error). */
size_t bt_workspace_bytes(const bt_config* cfg);

/* Validate cfg, build the geometry and momentum tables (Sec. 3.1) in float64
 * on the host, and upload them.  workspace: NULL (the library allocates with
 * cudaMalloc) or a device pointer to at least bt_workspace_bytes(cfg) bytes,
 * 256-byte aligned, that the caller keeps alive until bt_destroy.  f starts
 * at zero.  *out receives the handle. */
int bt_create(const bt_config* cfg, void* workspace, bt_handle** out);
int bt_destroy(bt_handle* h);

/* Fluid and metric background and opacities (Sec. 3.1 CFC metric, Sec. 3.2.2,
 * Sec. 3.2.3, Sec. 3.4): per zone v[3], lapse alpha, conformal factor phi,
 * shift[3] (must be zero); per (s, zone, group) kappa_a, kappa_s, f_eq.
 * rho, T, Ye are accepted for the caller's bookkeeping and not used (the
 * opacities are given).  Any may be NULL except v, alpha, phi, kappa_a,
 * kappa_s, f_eq.  A background set after an earlier one makes the next
 * bt_step first remap f from the earlier background's comoving frames to the
 * new ones (Sec. 3.2, time remap). */
int bt_set_background(bt_handle* h, int mem,
                      const double* rho, const double* T, const double* Ye,
                      const double* v, const double* alpha, const double* phi,
                      const double* shift,
                      const double* kappa_a, const double* kappa_s, const double* f_eq);

/* Distribution imposed on the bins that enter the grid through the open
 * face at theta_max (Sec. 4.5.2: an isotropic distribution imposed along the
 * boundary theta = pi/2), isotropic in the face's comoving frame, per
 * [s][radial zone a][group] (n_species x n_r x n_eps doubles; host or
 * device pointer as `mem` says).  BT_ERR_ARG if the grid has no open face
 * (theta_max == pi, a column or a slab).  It stays until set again; the
 * flux through the face counts in the outflow tallies (negative inflow). */
int bt_set_boundary(bt_handle* h, int mem, const double* f_boundary);

/* Copy f in/out (layout above; float64 for BT_FP64, float32 for BT_MIXED).
 * bt_set_f takes f as given in the current background's comoving frames and
 * cancels a pending time remap. */
int bt_set_f(bt_handle* h, int mem, const void* f);
int bt_get_f(bt_handle* h, int mem, void* f);

/* Courant limit (Sec. 3.3, global timestep limited by the smallest cell): the
 * largest dt for which no bin of any zone loses more than `cfl` of its
 * content through its faces in one step. */
int bt_max_dt(bt_handle* h, double cfl, double* dt_out);

/* One transport step of length dt (Sec. 3.3 Eq. fullstep, Sec. 3.5).  The
 * step is only enqueued: BT_OK means the launches were accepted.  A
 * non-finite result (BT_ERR_NUMERIC) or a bounded device wait that gave up
 * (BT_ERR_TIMEOUT) is recorded in device flags and reported by the next call
 * that synchronises the stream and returns data (bt_get_f, bt_moments,
 * bt_totals, bt_sur_stats, bt_autotune). */
int bt_step(bt_handle* h, double dt);

/* Local time stepping (Sec. 5: the global step is limited by the small
 * zones at the centre, while larger outer zones could take larger steps).
 * Zone z advances with its own step dt0 2^levels[z], levels in [0, n_levels);
 * bt_step_lts(h, dt0) advances every zone by the macro step dt0 2^(n_levels-1):
 *   - the time remap (if a background was set) runs once, first;
 *   - at substep k (of dt0) every face whose finer side has level l is
 *     evaluated if k is a multiple of 2^l, over dt0 2^l, from the current f
 *     (a coarser neighbour's f is still that of the start of its step); its
 *     flux goes to both sides and waits there until the side's step ends, so
 *     number is conserved face by face (Eq. fullstep);
 *   - a zone whose step ends at substep k ((k + 1) a multiple of 2^level)
 *     then takes its collision solve over its own step (Sec. 3.5);
 *   - bt_moments then returns the source terms averaged over the macro step,
 *     and the outflow tallies cover the macro step.
 * It uses the split flux form (split/256 if the handle's shape is fused; the
 * deposit rows are allocated as for bt_set_launch_shape) and updates f in
 * place.  It does not run with a learned remap (BT_ERR_ARG).
 * bt_set_levels installs levels (host array [zone], 1 <= n_levels <= 16).
 * bt_lts_levels computes them from the current background: dt0 = cfl / (the
 * largest per-zone Courant rate, as bt_max_dt), each zone the largest level
 * l < max_levels with dt0 2^l within its own limit cfl / rate, then lowered
 * until radial (and, on 2D grids, polar) neighbours differ by at most one
 * level; it installs them, returns dt0 and, if `levels` is not NULL, the
 * levels (host [zone]).  bt_n_levels returns the installed number. */
int bt_set_levels(bt_handle* h, const int32_t* levels, int n_levels);
int bt_lts_levels(bt_handle* h, double cfl, int max_levels, double* dt0, int32_t* levels);
int bt_n_levels(const bt_handle* h);
int bt_step_lts(bt_handle* h, double dt0);

/* Collision source terms of the last step (Eq. hydrosource), per unit
 * coordinate volume and time: dN[s][zone], dE[s][zone] (comoving energy),
 * dP[s][zone][3] (comoving momentum, local triad), Q_Ye[zone] =
 * -(dN_nue - dN_nuebar) * phase_norm.  Any output may be NULL.
 * Sign: dN, dE and dP are what the neutrinos gain from collisions (+ when
 * emission exceeds absorption); the hydro source terms Q_E and Q_M of Eq.
 * hydrosource are their negatives summed over species, which the caller
 * forms.  Q_Ye is returned with the equation's sign already applied. */
int bt_moments(bt_handle* h, int mem, double* dN, double* dE, double* dP, double* Q_Ye);

/* Per-species totals (host arrays of n_species): number N = sum dV phi^6 u^0
 * dGamma dOmega f; energy at infinity E (lab energy eps u^0 times alpha);
 * cumulative number and energy that left through open boundaries. */
int bt_totals(bt_handle* h, double* N, double* E, double* N_out, double* E_out);

/* Comoving angular moments J, H, K per [s][zone][group] (Sec. 4.1). */
int bt_jhk(bt_handle* h, int mem, double* J, double* H, double* K);

/* Number of device kernel launches this handle has issued (for accounting). */
int64_t bt_launch_count(const bt_handle* h);

/* Per-kernel timing with CUDA events recorded on the handle's stream around
 * every launch of bt_step while enabled (enable = 1), for measurement.
 * bt_profile(h, 1) also clears the records.  bt_profile_read synchronises
 * the stream and returns, for kernel id BT_K_TIME_REMAP / BT_K_FLUX /
 * BT_K_OUTFLOW / BT_K_SUR_TABLE (the learned remap's table) / BT_K_ZONE (the
 * split form's zone pass; BT_K_FLUX is then its face pass), the summed
 * duration in ms and the number of launches. */
enum { BT_K_TIME_REMAP = 0, BT_K_FLUX = 1, BT_K_OUTFLOW = 2, BT_K_SUR_TABLE = 3, BT_K_ZONE = 4 };
int bt_profile(bt_handle* h, int enable);
int bt_profile_read(bt_handle* h, int kernel, double* total_ms, int64_t* launches);

/* Measured fused multiply-add rate of the current device in the arithmetic
 * of `precision` (BT_FP64: float64, BT_MIXED: float32), in flop/s (an FMA is
 * two flops): independent FMA chains on every SM, timed with CUDA events on
 * `stream` (cudaStream_t).  A measurement aid with no counterpart in the
 * paper: it gives the ALU peak that the transport kernels' arithmetic is
 * compared with.  Synchronises; BT_OK, BT_ERR_ARG or BT_ERR_CUDA. */
int bt_peak_fma(int precision, double* flops_per_s, void* stream);

/* Launch shape of the flux step.  128, 256 or 512: the fused form, one
 * kernel in which each zone's CTA computes all of its faces (every interior
 * face is computed by both neighbours) and then its collision solve, with
 * that many threads per CTA (default 256, or the choice cached by the
 * autotuner).  BT_SHAPE_SPLIT | 256, | 384 or | 512: the split form, a face pass in
 * which every face is computed once (by the zone that owns it) and writes both
 * neighbours' deposits, then a zone pass that gathers a zone's deposits in
 * the fused order and solves its collision; it needs 6 x the f array in
 * deposit rows, allocated when the shape is set.  A shape needs at least one
 * thread per angle bin (threads >= n_mu * n_phi); one that does not fit the
 * problem (threads, shared memory, registers) is refused with BT_ERR_ARG and
 * is not tried by the autotuner (BT_SHAPE_SPLIT | 384 exists in the mixed
 * precision only: three 128-angle chunks of a 20-group row, for example, at
 * two CTAs per SM without spilling registers).  FP64 results are bitwise the same for
 * every shape; mixed-precision results agree to float32 rounding (their
 * exact-total sums are formed in a shape-dependent order). */
#define BT_SHAPE_SPLIT 0x10000
int bt_launch_shape(const bt_handle* h, int* threads_per_cta);
int bt_set_launch_shape(bt_handle* h, int threads_per_cta);

/* Autotuner: times the flux kernel of the current state (background and f
 * set) for every launch shape that fits, keeps the fastest, and -- if the
 * environment variable BT_TUNE_CACHE names a file -- records it there under a
 * key of the problem shape; bt_create reads that file.  The timing launches
 * leave f, the cumulative outflow and the last step's moments (bt_moments)
 * as they were: the moments are copied aside before the trials and restored
 * after them.  The split shapes are tried only if their deposit rows can be
 * allocated.  *chosen_nt may be NULL.
 * Without a cached choice, bt_create starts with the first of fused/256,
 * split/256, split/512, fused/512, fused/128 that fits the problem; it
 * refuses the problem (BT_ERR_ARG, "shared memory") only if none does. */
int bt_autotune(bt_handle* h, double dt, int* chosen_nt);

/* Batched step: n independent problems (each its own configuration, e.g. of
 * uneven size and group/angle counts) advanced together.  bt_batch_create
 * creates one member handle per configuration, all on `stream`; the members
 * are set and read through the single-problem calls above (bt_batch_member
 * returns member i's handle, owned by the batch).  bt_batch_step(b, dt[n])
 * advances every member by one step (Sec. 3.3, 3.5) with ONE launch of a CUDA
 * graph whose branches run the members' kernels concurrently; graphs are
 * captured on first use and cached by the members' buffer parity, pending
 * time remap, dt and launch shape (at most 16 graphs are kept).  `stream`
 * must be a created stream: the legacy default stream (0) cannot be
 * captured and gives BT_ERR_ARG.  A member without a background gives
 * BT_ERR_STATE, a dt[i] <= 0 or non-finite BT_ERR_DT; neither launches
 * anything.  Errors inside the kernels surface, as for bt_step, at the next
 * call that returns data for that member. */
typedef struct bt_batch bt_batch;
int bt_batch_create(const bt_config* cfgs, int n, void* stream, bt_batch** out);
int bt_batch_member(bt_batch* b, int i, bt_handle** out);
int bt_batch_step(bt_batch* b, const double* dt);
int64_t bt_batch_launch_count(const bt_batch* b);   /* kernel launches of all members */
int64_t bt_batch_graph_launches(const bt_batch* b);
int bt_batch_destroy(bt_batch* b);

/* Weighted totals of a distribution without any device allocation.
 * The paper has no counterpart: this is a library service for callers that
 * cannot allocate device memory -- e.g. a host code whose own allocator owns
 * all device memory, or a loop that must never allocate.
 *   out[s] = sum over zone z, group i, angle b of
 *            w_za[z][b] * w_e[i] * f[s][z][i][b]
 * (with w_za = dV phi^6 u^0 dOmega and w_e = dGamma this is the number of
 * species s that bt_totals reports).  All pointers are DEVICE pointers owned
 * by the caller; f is float64 (precision BT_FP64) or float32 (BT_MIXED) in the
 * layout above; out receives n_s doubles.  Work is enqueued on `stream`
 * (cudaStream_t); the call does not synchronise.
 * Scratch: per-block partial sums live in one file-scope device array of
 * 2 * BT_NOALLOC_MAX_PARTIALS doubles (1 MiB) that every GPU loading the
 * library holds until the process exits; n_s * ceil(n_zone / 64) must not
 * exceed BT_NOALLOC_MAX_PARTIALS (else BT_ERR_ARG).  The first call on a
 * device looks up that array's device address (with that device current),
 * so make it before any stream capture.  Every call overwrites the partials it
 * reads, so nothing needs clearing, but calls that overlap on the GPU race on
 * the shared array.  Returns BT_OK, BT_ERR_ARG or BT_ERR_CUDA; bt_last_error()
 * is not updated by this call.  It calls no cudaMalloc/cudaFree. */
#define BT_NOALLOC_MAX_PARTIALS (1 << 16)
int bt_weighted_totals_noalloc(const void* f, int precision, int n_s, int n_zone, int n_e, int n_ang,
                               const double* w_za, const double* w_e, double* out, void* stream);

/* ------------------------------------------------------------------------
 * Learned remap: a small network that predicts the remap's redistribution
 * weights (the paper has no counterpart; its remap weights are the exact
 * trilinear ones of Sec. 3.2, which stay the check and the fallback).
 *
 * Network: x (BT_SUR_NIN = 16 features) -> normalise (x - mean) * scale ->
 * 64 -> 64 -> 64 (GELU, exact erf form) -> 27 logits -> softmax P over the
 * offsets {-1,0,1}^3 of (energy group, mu index, Phi index), offset (de, dm,
 * dp) at index 9 (de+1) + 3 (dm+1) + (dp+1).  Evaluated and trained on the
 * tensor cores with bf16 operands and fp32 accumulation.
 *
 * Parameter block (BT_SUR_NPARAM floats, fp32): W1 [64][16], b1 [64],
 * W2 [64][64], b2 [64], W3 [64][64], b3 [64], W4 [27][64], b4 [27],
 * mean [16], scale [16]; W_l row-major [out][in].
 *
 * A bt_surrogate owns its parameters, gradient and Adam state on the device
 * and enqueues on `stream`.  X, Y, P, grad and loss below are DEVICE pointers
 * owned by the caller: X [n][16], Y and P [n][27] row-major fp32.  The calls
 * synchronise and return BT_ERR_TIMEOUT if a bounded tensor-core wait gave
 * up (the results are then invalid).
 * ------------------------------------------------------------------------ */
/* Training rows of the learned remap from the handle's exact remap (the
 * emit mode of Sec. 3.2's weights).  Row i is idx[i] = (zone, kind, source
 * angle): kind 0 is the zone's time remap from the previous to the current
 * background (G = I); kind 1 + 6 f + r (f = 0..4: inner and outer radial,
 * lower and upper polar -- or the periodic polar face of a column --, and the
 * azimuthal face of the zone) is remap r of face f: r = 0..3 carries stencil
 * cell r (zones P-1, P, Q, Q+1) into the face frame, r = 4, 5 carries the
 * face frame into cell P, Q.  Outputs, per row:
 *   X[i][16]  features: source direction n (0-2), source velocity (3-5),
 *             destination velocity in the source triad (6-8), rotation
 *             vector of the source -> destination triad rotation (9-11),
 *             ln(alpha_src/alpha_dst) on the kick axis (12-14, zero for the
 *             time remap), ln((phi_src/phi_dst)^2) (15);
 *   Y[i][27]  the exact trilinear weights on the offsets {-1,0,1}^3 of
 *             (group, mu index, Phi index), Phi offsets wrapped;
 *   valid[i]  1 = usable, 2 = a weight lands outside the offsets (Y = 0),
 *             0 = no such remap (absent face or cell, or idx out of range).
 * idx, X, Y and valid are DEVICE pointers; computed in float64, stored as
 * float32.  Needs two backgrounds set (BT_ERR_STATE otherwise).  Synchronises. */
int bt_sur_samples(bt_handle* h, const int32_t* idx, int64_t n, float* X, float* Y, int32_t* valid);

#define BT_SUR_NIN 16
#define BT_SUR_NOUT 27
#define BT_SUR_NPARAM 11195
typedef struct bt_surrogate bt_surrogate;
typedef struct {
  int32_t epochs;  /* passes over the samples */
  int32_t batch;   /* rows per Adam step (the last batch of a pass may be short) */
  float lr, lr_final;   /* cosine decay from lr to lr_final over all steps */
  float beta1, beta2, eps;
} bt_train_cfg;
int bt_sur_create(void* stream, bt_surrogate** out);
int bt_sur_destroy(bt_surrogate* s);
/* copy the BT_SUR_NPARAM parameters in (resets the Adam state) or out */
int bt_sur_set_params(bt_surrogate* s, int mem, const float* p);
int bt_sur_get_params(bt_surrogate* s, int mem, float* p);
/* mean and scale = 1/standard deviation of each feature over X [n][16] */
int bt_sur_fit_normalizer(bt_surrogate* s, const float* X, int64_t n);
/* P = network(X) */
int bt_sur_forward(bt_surrogate* s, const float* X, int64_t n, float* P);
/* grad [BT_SUR_NPARAM] = gradient of the mean cross entropy
 * -1/n sum_rows sum_o Y log P over the n rows, loss [1] = that mean
 * (normaliser entries of grad are 0) */
int bt_sur_grad(bt_surrogate* s, const float* X, const float* Y, int64_t n, float* grad, float* loss);
/* Adam on the mean cross entropy, minibatches taken in order (pass
 * shuffled samples); loss_log (HOST, [epochs] or NULL) gets each pass's mean
 * batch loss */
int bt_sur_train(bt_surrogate* s, const float* X, const float* Y, int64_t n, const bt_train_cfg* cfg,
                 float* loss_log);

/* Use the network for the remap weights of every bt_step of h (mixed
 * precision only; s = NULL returns to the exact weights).  Each step first
 * evaluates the network on all of the step's remap rows -- the time remap
 * when the background changed, and the six remaps of every face of every
 * zone --, takes each predicted distribution's mean offset per axis as the
 * trilinear bracket and weight of that axis, and compares it with the exact
 * weights of Sec. 3.2: a row whose mean offset differs by tol (in bins) or
 * more on any axis "trips" and uses the exact weights.  tol = 0 trips every
 * row and reproduces the exact mixed-precision step bit for bit.  Weights
 * sum to one per axis either way, so number is conserved.  s must stay
 * alive while set and share h's stream.  Allocates the weight table
 * (n_zone x 31 x n_ang rows of 20 bytes) on first use. */
int bt_set_surrogate(bt_handle* h, bt_surrogate* s, double tol);
/* cumulative rows evaluated by the network and rows that tripped */
int bt_sur_stats(bt_handle* h, int64_t* n_eval, int64_t* n_trip);

#ifdef __cplusplus
}
#endif
#endif /* BT_H_ */
