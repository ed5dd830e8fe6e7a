/*
 * bd3mg.h -- C ABI of the GB300 block 3MG (BD3MG) deblurring library.
 *
 * The library minimises, on one GPU, the penalised least-squares objective of
 * Section 3.1 (Eq. "crit") for a 3D volume degraded by a depth-variant blur
 * (Eq. "model"):
 *
 *   f(x) = 1/2 ||H x - y||^2                                   (data term)
 *        + eta * sum_n dist(x_n, [xmin, xmax])^2              (box term)
 *        + lambda * sum_n sum_{a in X,Y,Z} sqrt(delta^2 + ([V^a x]_n)^2)
 *
 * (the default, per-axis penalty; the form printed in Section 3.1, a joint
 * X-Y hyperbolic term plus kappa ||V^Z x||^2, is BD3MG_PENALTY_JOINT_XY, and an
 * isotropic term over the three axes is BD3MG_PENALTY_ISOTROPIC)
 *
 * with the Majorize-Minimize Memory Gradient iteration run block by block
 * (Sections 2.2-2.3): at each step a block S (a slab of depth slices) builds
 * the half-quadratic majorant Q_(S) (Eq. "maj"), the memory-gradient subspace
 * D_(S) = [-grad_(S) f | d_(S)] and the 2x2 minimiser (Eq. "minimizer"), and
 * moves x_(S) by D_(S) u (Master box step (2)).  Blocks that cannot interact
 * are processed together; the result equals visiting the blocks one after the
 * other in colour-major order (synchronous case of Section 2.4).
 *
 * Conventions (all entry points):
 *   - Volumes are float32, C order [nz][ny][nx] (x fastest).  The PSF is
 *     float32 [nz][pz][py][px]: entry (z, c+rz, b+ry, a+rx) is the tap
 *     h_z(a, b, c) of the PSF attached to OUTPUT depth z, applied as
 *     (Hx)(i,j,z) = sum_{a,b,c} h_z(a,b,c) x(i-a, j-b, z-c), zero outside.
 *   - V^a is the forward difference along axis a with a zero last row.
 *   - Every call returns a bd3mg_status and never throws.  After an error the
 *     context is poisoned: later calls return BD3MG_ESTATE until destroyed;
 *     bd3mg_error_string gives the first error's text.
 *   - All device work is ordered on the stream given at creation (a
 *     cudaStream_t passed as void*; NULL = the legacy default stream).  Calls
 *     that return host values synchronise that stream.  One host thread per
 *     context at a time.
 *   - Inputs are copied; the caller keeps ownership of its buffers.  The
 *     context owns its device state, obtained through the optional allocator
 *     (else cudaMallocAsync on the context stream).
 */
#ifndef BD3MG_H
#define BD3MG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bd3mg_ctx bd3mg_ctx;

typedef enum {
    BD3MG_OK = 0,
    BD3MG_EINVAL = 1,        /* invalid argument (message says which) */
    BD3MG_ENOMEM = 2,        /* device allocation failed */
    BD3MG_ECUDA = 3,         /* a CUDA runtime call failed */
    BD3MG_ETIMEOUT = 4,      /* a bounded device wait gave up */
    BD3MG_ENONFINITE = 5,    /* NaN/Inf met in a subspace matrix or objective */
    BD3MG_ESTATE = 6,        /* context poisoned by an earlier error */
    BD3MG_EUNSUPPORTED = 7   /* valid request the build does not implement */
} bd3mg_status;

/* Device memory hook: alloc returns device memory of `bytes` usable on `stream`
 * (NULL on failure); free releases it.  Both are called from the thread that
 * calls the library. */
typedef struct {
    void *(*alloc)(void *user, size_t bytes, void *stream);
    void (*free)(void *user, void *ptr, size_t bytes, void *stream);
    void *user;
} bd3mg_allocator;

/* Storage precision of the gradient direction (Section 2.3 subspace D = [-g, d]).
 * BD3MG_FP32: g stored in FP32.
 * BD3MG_BF16_GRADIENT: g stored in BF16 (round to nearest even), halving its
 *   traffic and the curvature pass's shared-memory ring; x, y, d, the residual
 *   and the images H d_S stay FP32 (they are carried from one iteration to the
 *   next, g is recomputed every time), all arithmetic is FP32 and every
 *   reduction and the 2x2 solve FP64.  The subspace is then spanned by
 *   [-g_bf16, d]: B = D^T A D and D^T grad f are formed from it (the gradient
 *   term as -||g_bf16||^2), and x moves by the FP32 step -u0 g_bf16 + u1 d.
 *   bd3mg_gradient and bd3mg_get_volume return g widened to FP32.
 * BD3MG_BF16_DIRECTIONS: g, the memory direction d and the images H g and H d
 *   stored in BF16 (round to nearest even); x, y and the residual r stay
 *   FP32, arithmetic FP32, reductions and the 2x2 solve FP64.  The update
 *   n = -u0 g + u1 d and H n = -u0 H g + u1 H d are formed in FP32 from the
 *   stored values: x += n and r += H n in FP32, d and H d take n and H n
 *   rounded.  r therefore drifts from H x - y by the rounding of H g and H d;
 *   the exact refresh every refresh_every iterations bounds the drift.  Runs
 *   in the fused form only (volumes without slabs, a separable PSF, the
 *   per-axis penalty, separate_update AUTO or FUSED, not persistent), else
 *   BD3MG_EUNSUPPORTED.  bd3mg_get_volume returns d widened to FP32;
 *   checkpoints hold the BF16 bits (bit-exact resume in the same mode).
 *   bd3mg_set_escalation switches it to FP32 g, d, H g and H d (the stored
 *   values widened).
 * Every volume of a batch must use the same mode. */
enum { BD3MG_FP32 = 0, BD3MG_BF16_GRADIENT = 1, BD3MG_BF16_DIRECTIONS = 2 };

/* Penalty term f3 of the objective (Section 3.1, Eq. "crit"), with forward
 * differences [V^a x]_n = x_{n+e_a} - x_n, zero on the last plane of axis a.
 * BD3MG_PENALTY_PER_AXIS (default): f3 = lambda sum_n sum_{a in X,Y,Z}
 *   sqrt(delta^2 + [V^a x]_n^2); the majorant weights each axis by
 *   w_a = 1/sqrt(delta^2 + [V^a x]_n^2).
 * BD3MG_PENALTY_JOINT_XY (the form printed in Section 3.1): f3 = lambda sum_n
 *   sqrt(delta^2 + [V^X x]_n^2 + [V^Y x]_n^2) + kappa ||V^Z x||^2; the X and Y
 *   differences share one weight w = 1/sqrt(delta^2 + [V^X x]_n^2 + [V^Y x]_n^2)
 *   in the majorant and the Z term contributes its exact Hessian
 *   2 kappa V^ZT V^Z.
 * BD3MG_PENALTY_ISOTROPIC: f3 = lambda sum_n sqrt(delta^2 + [V^X x]_n^2
 *   + [V^Y x]_n^2 + [V^Z x]_n^2); the three differences of a voxel share one
 *   weight w = 1/sqrt(delta^2 + sum_a [V^a x]_n^2) in the majorant (kappa is
 *   not used).
 * Every volume of a batch must use the same penalty mode. */
enum { BD3MG_PENALTY_PER_AXIS = 0, BD3MG_PENALTY_JOINT_XY = 1, BD3MG_PENALTY_ISOTROPIC = 2 };

/* Ablation variants of the ablation study (Section 3.2, Table 1), as switches
 * on the same kernels.  The paper's methods map to:
 *   BD3MG / 3MG:  METRIC_MAJORANT, DIR_MEMORY_GRADIENT, SCHEDULE_COLOURED (defaults)
 *   BP3MG:        METRIC_MAJORANT, DIR_MEMORY_GRADIENT, SCHEDULE_JACOBI
 *   Async-GD:     METRIC_LIPSCHITZ, DIR_GRADIENT
 *   Async-CG:     METRIC_LIPSCHITZ, DIR_CONJUGATE
 * (Async-MM, whose worker inverts A(x) with an inner BiCG solve, is not built.)
 * metric: the block majorant's curvature matrix.  METRIC_MAJORANT: the
 *   half-quadratic A(x) of bd3mg_create; METRIC_LIPSCHITZ: A = L I with L the
 *   caller's lipschitz, or (lipschitz = 0) the library's bound on the
 *   Lipschitz constant of grad f, ||H||_1 ||H||_inf + 2 eta + the penalty's
 *   Hessian bound (12 lambda / delta; mode 1: 8 lambda / delta + 8 kappa).
 * direction: DIR_MEMORY_GRADIENT, D = [-g, d] and the 2x2 minimiser;
 *   DIR_GRADIENT, D = -g (one-dimensional minimiser, u = ||g||^2 / g^T A g);
 *   DIR_CONJUGATE, p = -g + beta p_prev with the Fletcher-Reeves beta =
 *   ||g||^2 / ||g_prev||^2 of the slab and the step minimising the majorant
 *   along p, restarted along -g when p is not a descent direction.  (Read
 *   literally, D = [-g, d] with A = L I minimises an isotropic quadratic over a
 *   subspace that contains g, which gives the gradient step whatever d is; the
 *   conjugate direction is the reading that keeps the memory term.)
 * schedule: SCHEDULE_COLOURED, the colour-major sweep (equal to visiting the
 *   slabs one after the other); SCHEDULE_JACOBI, every slab's step computed
 *   from the same iterate and all applied together (the parallel block update
 *   without delay of BP3MG); r and H d_S are then recomputed exactly after
 *   every sweep.
 * inflation: the subspace matrix is multiplied by this factor >= 1 (Assumption
 *   C: the block curvature must dominate what the delayed or simultaneous
 *   updates need; m slabs updated from one iterate descend when it is >= m).
 *   0 -> 1 for SCHEDULE_COLOURED, the number of slabs for SCHEDULE_JACOBI. */
enum { BD3MG_METRIC_MAJORANT = 0, BD3MG_METRIC_LIPSCHITZ = 1 };
enum { BD3MG_DIR_MEMORY_GRADIENT = 0, BD3MG_DIR_GRADIENT = 1, BD3MG_DIR_CONJUGATE = 2 };
enum { BD3MG_SCHEDULE_COLOURED = 0, BD3MG_SCHEDULE_JACOBI = 1 };

/* Blur path.  The separable path factors each depth's PSF as fx(a) fy(b)
 * fz(c) and convolves axis by axis inside the tile kernels.  The dense path
 * (a PSF that does not factor, such as the rotated Gaussians of Section 3.1,
 * or radii beyond the separable kernels) applies the taps as given with a
 * direct convolution per output depth: PSF extents up to 11 x 11 in x, y and
 * 21 in z (the paper's 11 x 11 x 21 and 5 x 5 x 11), FP32 gradient only; the
 * iteration, slab form, batches, variants and stopping are the same.  With a
 * dense PSF, bd3mg_objective and bd3mg_gradient first recompute r and H d_S
 * exactly (the refresh an iteration does every refresh_every sweeps).  The
 * allocation-free objective takes separable PSFs only. */
enum { BD3MG_PSF_AUTO = 0, BD3MG_PSF_DENSE = 1 };

/* How an iteration without slabs applies its update (bd3mg_params.separate_update). */
enum { BD3MG_UPDATE_AUTO = 0, BD3MG_UPDATE_SEPARATE = 1, BD3MG_UPDATE_FUSED = 2 };

typedef struct {
    int nx, ny, nz;           /* volume extents, each >= 1 */
    int px, py, pz;           /* PSF extents, odd, >= 1 */
    const float *psf;         /* HOST pointer, nz*pz*py*px floats, copied at creation */
    double lambda;            /* > 0 penalty weight */
    double delta;             /* > 0 hyperbolic smoothing */
    double eta;               /* >= 0 box weight */
    double xmin, xmax;        /* box bounds, xmin <= xmax */
    int precision;            /* BD3MG_FP32, BD3MG_BF16_GRADIENT or BD3MG_BF16_DIRECTIONS */
    int nslabs;               /* number of depth blocks; 0 or 1 = plain 3MG on the whole volume */
    const int *slab_bounds;   /* HOST, nslabs+1 increasing slice indices from 0 to nz (ignored if nslabs <= 1) */
    double pinv_rtol;         /* eigenvalues <= rtol*max are dropped in the 2x2 pseudo-inverse; 0 -> 1e-12 */
    int zchunk;               /* output slices per work item; 0 -> chosen by the library's cost model,
                                 and chosen again for the volumes still running when some volumes
                                 of a batch stop (their sums regroup: iterates equal to rounding);
                                 > 0 -> kept for every launch (stopping then leaves every running
                                 volume bit-identical to an uncompacted run) */
    int penalty;              /* BD3MG_PENALTY_PER_AXIS, BD3MG_PENALTY_JOINT_XY or BD3MG_PENALTY_ISOTROPIC */
    double kappa;             /* >= 0, finite: weight of kappa ||V^Z x||^2 (BD3MG_PENALTY_JOINT_XY only) */
    int refresh_every;        /* >= 0: iterations between exact recomputations of r and H d_S; 0 -> 256 */
    int barrier_timeout_ms;   /* 0..600000: limit of every bounded device wait (TMA slice copies);
                                 0 -> 2000.  A wait that runs out makes the call return BD3MG_ETIMEOUT */
    int separate_update;      /* BD3MG_UPDATE_AUTO (0, default), BD3MG_UPDATE_SEPARATE (1) or
                                 BD3MG_UPDATE_FUSED (2); taken from p[0] of a batch.  FUSED: a
                                 context whose volumes are not split into slabs (separable PSF)
                                 applies each iteration's update inside the next gradient pass (two
                                 passes per iteration, see bd3mg_create); SEPARATE: objective,
                                 gradient, curvature and update passes, as the slab form always
                                 runs; AUTO: FUSED from 2^24 voxels in the context, else SEPARATE */
    int metric;               /* BD3MG_METRIC_MAJORANT (default) or BD3MG_METRIC_LIPSCHITZ */
    double lipschitz;         /* L of BD3MG_METRIC_LIPSCHITZ (> 0), or 0: the library's bound */
    int direction;            /* BD3MG_DIR_MEMORY_GRADIENT (default), BD3MG_DIR_GRADIENT, BD3MG_DIR_CONJUGATE */
    int schedule;             /* BD3MG_SCHEDULE_COLOURED (default) or BD3MG_SCHEDULE_JACOBI (from p[0]) */
    double inflation;         /* >= 1, or 0: 1 (coloured) / the number of slabs (Jacobi) */
    int curv_rows;            /* output rows of a curvature tile: 0 (default: 16 with an FP32 gradient, 32
                                 with BF16), 16 or 32 (32 only with BF16); taken from p[0].  The
                                 autotuner times both shapes with every z-chunk */
    int psf_mode;             /* BD3MG_PSF_AUTO (default): the separable fast path when every depth's PSF
                                 factors and its radii are compiled (xy <= 5, z <= 5), else the dense path;
                                 BD3MG_PSF_DENSE: the dense path always (taken from p[0]) */
    int persistent;           /* 0 (default): every iteration is a replay of the captured iteration
                                 graph; 1: the fused form runs its iterations inside one persistent
                                 cooperative launch per refresh period (see bd3mg_iterate).  Needs
                                 the fused form (no slabs, separable PSF, coloured schedule;
                                 separate_update AUTO or FUSED), an FP32 gradient and 16-row
                                 curvature tiles, else BD3MG_EUNSUPPORTED.  Taken from p[0]. */
} bd3mg_params;

/* Fill *p with defaults (plain FP32, per-axis penalty, lambda = delta = 1e-2,
 * eta = 1, box [0, 1], no slabs, kappa = 0, refresh every 256 iterations,
 * 2 s device wait limit, extents zero: the caller must set nx..pz and psf).
 * refresh_every and barrier_timeout_ms of a batch are taken from p[0]. */
void bd3mg_params_default(bd3mg_params *p);

/* Create a context: validates *p, factors each depth's PSF (the fast path
 * needs h_z(a,b,c) = fx_z(a) fy_z(b) fz_z(c) to FP64 relative residual <=
 * 1e-6; otherwise BD3MG_EUNSUPPORTED), plans the slab colouring, copies y and
 * x0 (NULL -> x0 = y) into library memory, sets d = 0 and captures the
 * per-iteration CUDA graph.  An iteration blurs twice (H^T r and H g_S per
 * slab): the residual r = H x - y and the images H d_S of the slabs' memory
 * directions follow the iterate through the update (H d_S(new) = -u0 H g_S +
 * u1 H d_S, r += H d_S(new)), and are recomputed exactly before the first
 * iteration after creation or bd3mg_set_x, and every refresh_every (256)
 * iterations; bd3mg_load restores them with the refresh schedule.  Each
 * sweep's objective takes its data term from the carried r.
 * Without slabs, in the fused form (separate_update, below) an iteration is two kernel passes:
 * the gradient pass first applies the previous iteration's update (x, d, r
 * and H d) as it reads them, forms g and the objective of the new iterate,
 * and writes the new state into a second buffer set; the curvature pass then
 * builds and solves the 2x2 system.  The last update of bd3mg_iterate_async
 * stays pending until a call that reads the state (bd3mg_iterate's end,
 * bd3mg_objective, bd3mg_gradient, bd3mg_get_*, bd3mg_set_x, bd3mg_save,
 * bd3mg_set_stopping) applies it.  The iterates are the same bits as with
 * the separate update pass; the objective's summation order differs.
 * data_on_device: y and x0 are device pointers (else host).  stream:
 * cudaStream_t as void*.  alloc may be NULL. */
bd3mg_status bd3mg_create(const bd3mg_params *p, const float *y, const float *x0, int data_on_device,
                          void *stream, const bd3mg_allocator *alloc, bd3mg_ctx **out);

/* Create a context over nvol >= 1 independent volumes that iterate in lockstep
 * (one sweep of every volume per iteration, all volumes in the same kernel
 * launches).  p[v], y[v] and x0[v] (x0 may be NULL, or hold NULL entries, for
 * x0 = y) describe volume v exactly as for bd3mg_create; sizes, PSFs,
 * lambda, delta, eta and the box may differ between volumes.  The kernels are
 * chosen for the largest PSF radii (smaller PSFs are zero padded); pinv_rtol,
 * zchunk, refresh_every and barrier_timeout_ms are taken from p[0], and every
 * volume must share p[0]'s precision and penalty mode.  Per-volume results: bd3mg_objectives,
 * bd3mg_get_volume, and the nvol traces of bd3mg_iterate.  Functions without a
 * volume index act on volume 0. */
bd3mg_status bd3mg_batch_create(int nvol, const bd3mg_params *p, const float *const *y, const float *const *x0,
                                int data_on_device, void *stream, const bd3mg_allocator *alloc, bd3mg_ctx **out);

/* Number of volumes of the context (0 for NULL). */
int bd3mg_volume_count(bd3mg_ctx *ctx);

/* Run n >= 0 iterations (one iteration = one sweep over all slabs of every
 * volume).  If f_trace is not NULL it receives nvol*(n+1) host doubles,
 * volume-major: f(x^k) of each volume before each sweep and after the last.
 * Every entry takes its data term 1/2 ||r||^2 from the carried residual r
 * (bd3mg_objective applies H to x afresh; the two agree to ~1e-8 relative, the
 * FP32 evaluation accuracy), so a run split across calls reports the same
 * trace.  Synchronises the stream.
 * With bd3mg_params.persistent = 1, the iterations between two exact
 * refreshes run in one cooperative launch (k_persist): all its CTAs are
 * resident, take the work items of each pass from a queue and wait at a
 * grid-wide barrier (bounded by barrier_timeout_ms) between passes.  Volumes
 * of a batch stop inside the launch (no host round trip between iterations,
 * no re-planning of the work lists).  The iterates and the trace are the bits
 * of the graph form with the same work items. */
bd3mg_status bd3mg_iterate(bd3mg_ctx *ctx, int n, double *f_trace);

/* Enqueue n iterations without synchronising and without reading anything back
 * (for timing and overlap).  Errors raised on the device surface at the next
 * synchronising call. */
bd3mg_status bd3mg_iterate_async(bd3mg_ctx *ctx, int n);

/* Per-volume stopping.  Before each sweep k >= 1 the device tests every
 * running volume with the rule of the paper's scaling experiment (Section 3.3),
 *     ||x^k - x^{k-1}|| <= tol * ||x^{k-1}||,
 * where the step length is summed over the slab steps of sweep k-1 from the
 * FP64 subspace sums (||-u0 g + u1 d||^2 = u0^2 g.g - 2 u0 u1 g.d + u1^2 d.d)
 * and ||x^{k-1}||^2 is summed over the same slab steps (each slab is read
 * before its own update); it also stops a volume
 * once f(x^k) <= f_target[v].  A stopped volume keeps x^k: the work items of
 * its later sweeps exit at once and its trace repeats f(x^k).
 * tol: >= 0 (0 disables the step rule).  f_target: HOST array of nvol doubles,
 * or NULL for no targets (-INFINITY disables one volume's target).
 * Clears every volume's stopped state.  Default: tol 0, no targets.
 * Synchronises the stream.  EINVAL for a negative or non-finite tol or a NaN target. */
bd3mg_status bd3mg_set_stopping(bd3mg_ctx *ctx, double tol, const double *f_target);

/* sweeps: HOST array of nvol ints; receives, per volume, the number of sweeps
 * k after which it stopped (x^k is its result), or -1 while it runs.
 * Synchronises the stream. */
bd3mg_status bd3mg_stopped(bd3mg_ctx *ctx, int *sweeps);

/* Objective at the current iterate, with H applied to x afresh (valid at any
 * point, e.g. right after bd3mg_set_x); parts (optional, 3 doubles) = data
 * term, box term, penalty term.  Synchronises. */
bd3mg_status bd3mg_objective(bd3mg_ctx *ctx, double *f, double *parts);

/* Objective of every volume at the current iterates: f receives nvol host
 * doubles.  Synchronises. */
bd3mg_status bd3mg_objectives(bd3mg_ctx *ctx, double *f);

/* Copy volume vol's iterate (which = 0), memory direction d (1) or last
 * gradient g (2) to dst (nx*ny*nz floats of that volume; device pointer if
 * on_device else host).  Synchronises. */
bd3mg_status bd3mg_get_volume(bd3mg_ctx *ctx, int vol, int which, float *dst, int on_device);

/* Gradient of f at the current iterate (full volume) written to g (nx*ny*nz
 * floats; device pointer if on_device else host); f (optional) receives f.
 * Synchronises. */
bd3mg_status bd3mg_gradient(bd3mg_ctx *ctx, float *g, int on_device, double *f);

/* Copy the current iterate x (or the memory direction d) out / in.  set_x
 * also resets d to zero.  Pointers are device if on_device else host. */
bd3mg_status bd3mg_get_x(bd3mg_ctx *ctx, float *x, int on_device);
bd3mg_status bd3mg_get_d(bd3mg_ctx *ctx, float *d, int on_device);
bd3mg_status bd3mg_set_x(bd3mg_ctx *ctx, const float *x, int on_device);

/* Diagnostics of the most recent block steps: for each slab s of each volume
 * (volume-major, slab order), 8 doubles {B00, B01, B11, c0, c1, u0, u1, rank}
 * of the 2x2 system of its last update (B = D^T A D, c = D^T grad f,
 * u = -B^+ c).  info must hold 8 * (total slabs) doubles.  Synchronises. */
bd3mg_status bd3mg_last_step(bd3mg_ctx *ctx, double *info);

/* Apply the blur H or its adjoint H^T of this context to a device volume
 * (in and out: device pointers, nx*ny*nz floats, must not alias).  Used to
 * check the operators; does not touch the iterate. */
bd3mg_status bd3mg_apply_H(bd3mg_ctx *ctx, const float *in, float *out);
bd3mg_status bd3mg_apply_HT(bd3mg_ctx *ctx, const float *in, float *out);

/* Slab colouring chosen at creation: colour[s] for each slab of each volume
 * (volume-major; total-slab ints, host) and the number of colours.  Slabs of
 * one colour are at least max(pz-1, 1) slices apart, so their steps do not
 * interact. */
bd3mg_status bd3mg_slab_colours(bd3mg_ctx *ctx, int *colour, int *ncolours);

/* Host-only planning helpers (no GPU needed).
 * bd3mg_plan_slab_colours: greedy colouring, in increasing z, of the slabs
 * [bounds[s], bounds[s+1]) so that two slabs of one colour are at least
 * max(pz-1, 1) slices apart (a slab's step reads r on its slices +- (pz-1)/2
 * and x one slice beyond; its update changes r on the same reach), which makes
 * a colour's simultaneous steps equal to the sequential block order of
 * Section 3.1.  colour: nslabs ints out; returns BD3MG_EINVAL on bad bounds.
 * bd3mg_factor_psf: rank-1 factoring h_z(a,b,c) = fx_z(a) fy_z(b) fz_z(c) of
 * each depth's PSF in FP64; fx [nz*px], fy [nz*py], fz [nz*pz] out (may be
 * NULL); *residual = max over depths of max|h - fx fy fz| / max|h|; returns
 * BD3MG_EUNSUPPORTED when that exceeds 1e-6. */
bd3mg_status bd3mg_plan_slab_colours(int nslabs, const int *bounds, int pz, int *colour, int *ncolours);
bd3mg_status bd3mg_factor_psf(int nz, int px, int py, int pz, const float *psf, float *fx, float *fy, float *fz,
                              double *residual);

/* Kernel classes reported by bd3mg_profile_iteration. */
enum {
    BD3MG_K_OBJECTIVE = 0,   /* objective pass (one per sweep) */
    BD3MG_K_RESIDUAL = 1,    /* exact r = H x - y and H d_S (refreshes only: not part of an iteration) */
    BD3MG_K_GRADIENT = 2,    /* g = H^T r + box + penalty gradient */
    BD3MG_K_CURVATURE = 3,   /* H g_S, weights, inner products, 2x2 solve */
    BD3MG_K_UPDATE = 4,      /* x_S += D u, d_S = D u; H d_S and r on the slab's zone */
    BD3MG_K_DENSE = 5,       /* dense-PSF convolutions (H^T r and H g_S of the dense path) */
    BD3MG_K_CLASSES = 6
};

/* Run ONE iteration without the CUDA graph, with CUDA events recorded on the
 * context stream around every launch, and synchronise.  ms[k] receives the
 * summed device time of class k and launches[k] its launch count (arrays of
 * BD3MG_K_CLASSES; either may be NULL).  The iterate advances exactly as with
 * bd3mg_iterate_async(ctx, 1). */
bd3mg_status bd3mg_profile_iteration(bd3mg_ctx *ctx, double *ms, int *launches);

/* Number of kernel launches one iteration enqueues (a persistent context:
 * 1, an upper bound, since one launch runs up to refresh_every iterations). */
int bd3mg_launches_per_iteration(bd3mg_ctx *ctx);

/* Precision escalation of the BF16 forms (Section 2.3's subspace D = [-g, d]
 * with g, or g, d, H g and H d, stored in BF16).  With tol > 0, bd3mg_iterate
 * runs in chunks of 4 iterations and reads the objective trace between chunks;
 * once some volume's objective decreases by at most tol * |f| from one
 * iteration to the next, the context switches for good to FP32 storage (g
 * recomputed by the next iteration; d and H d widened from their BF16 values,
 * then r and H d recomputed exactly) and a new iteration graph.
 * bd3mg_iterate_async never escalates.  tol = 0 turns it off (the default);
 * no effect on FP32 contexts.  bd3mg_escalated: *at = the iteration count at
 * which the switch happened, -1 if it has not.  Errors: BD3MG_EINVAL for a
 * negative or non-finite tol or a NULL at. */
bd3mg_status bd3mg_set_escalation(bd3mg_ctx *ctx, double tol);
bd3mg_status bd3mg_escalated(bd3mg_ctx *ctx, long long *at);

/* Fault injection for testing failure detection (no counterpart in the paper).
 * BD3MG_FAULT_SKIP_COPY: from the next iteration on, the first CTA of every
 * curvature launch leaves the copy of one input slice out, so nothing
 * completes the shared-memory barrier it then waits on; that bounded wait runs
 * out after barrier_timeout_ms, the CTA waits (again bounded) for its other
 * copies and returns, and the call reports BD3MG_ETIMEOUT (the context is then
 * poisoned; the CUDA context stays usable).  Nothing traps, faults or hangs.
 * BD3MG_FAULT_SKIP_ARRIVE (persistent contexts): CTA 0 of the persistent
 * launch leaves without arriving at its first grid-wide barrier; every other
 * CTA's barrier wait runs out after barrier_timeout_ms and the call reports
 * BD3MG_ETIMEOUT in the same way.
 * BD3MG_FAULT_NONE turns it off.  Takes effect at the next launch. */
enum { BD3MG_FAULT_NONE = 0, BD3MG_FAULT_SKIP_COPY = 1, BD3MG_FAULT_SKIP_ARRIVE = 2 };
bd3mg_status bd3mg_inject_fault(bd3mg_ctx *ctx, int kind);

/* Checkpoint / resume.  bd3mg_save writes the state an iteration starts from
 * (x, the memory direction d and the residual r of every volume, the images
 * H d_S of every slab, the iteration count and the refresh schedule) to the
 * file `path` (overwritten); bd3mg_load reads such a file into a context
 * created with the same volumes, slabs and precision, and clears the stopping
 * state.  Everything else an iteration needs (gradient, 2x2 system) is
 * recomputed, so a loaded context continues bit for bit like the one that was
 * saved.
 * Errors: BD3MG_EINVAL (unreadable or mismatching file; the message says
 * which), BD3MG_ECUDA. */
bd3mg_status bd3mg_save(bd3mg_ctx *ctx, const char *path);
bd3mg_status bd3mg_load(bd3mg_ctx *ctx, const char *path);

/* Autotuner of the tile kernels' work shape.  Times `iters` lockstep
 * iterations (after 2 untimed ones) of contexts built like
 * bd3mg_batch_create(nvol, p, y, NULL, data_on_device, stream, NULL, ...) for
 * every pair of a z-chunk (0 = the library's cost model, and 4, 6, 8, 12, 16,
 * 24, 32, 48 output slices per work item) and a curvature tile height (16 and
 * 32 rows with an FP32 gradient, 32 with BF16), and returns the fastest pair in
 * *zchunk and *curv_rows (give them to bd3mg_params.zchunk and .curv_rows;
 * curv_rows may be NULL) and its device time per iteration in
 * *ms_per_iteration (may be NULL).  Candidates that do not fit in device memory
 * are skipped.  cache_path (may be NULL): a JSON-lines file; when it holds an
 * entry for the same shape class (SM count, precision, every volume's extents,
 * PSF extents and slab bounds) that entry is returned without timing
 * (*ms_per_iteration = -1), otherwise the result is appended.  The contexts are
 * created and destroyed on `stream`; the caller's data is only read. */
bd3mg_status bd3mg_autotune(int nvol, const bd3mg_params *p, const float *const *y, int data_on_device, void *stream,
                            int iters, const char *cache_path, int *zchunk, int *curv_rows, double *ms_per_iteration);

/* Size of the device array behind bd3mg_objective_noalloc (bytes). */
#define BD3MG_STATIC_SCRATCH_BYTES (1u << 20)

/* Objective f(x) without allocating device memory (the paper has no
 * counterpart; this is a deployment variant of bd3mg_objective).
 *
 * For callers that cannot allocate where they need the objective: plug-ins
 * inside a host framework that owns all device memory and forbids private
 * allocations, and latency-critical loops that must not take the allocator's
 * locks or pay the device-wide synchronisation that cudaFree implies.  The
 * call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine): its device state lives in one file-scope device array of
 * BD3MG_STATIC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.
 *
 * p: problem as for bd3mg_create (nslabs, precision and pinv_rtol are
 *    ignored; psf is a host pointer, read during the call).
 * x, y: DEVICE volumes [nz][ny][nx], read in place; nx must be a multiple of 4
 *    and both pointers 16-byte aligned.
 * f_out: DEVICE pointer to 4 doubles, written with {f, data term, box term,
 *    penalty term}.  The call first fills them with NaN, so a NaN f means the
 *    kernel did not finish (a timed-out wait) or the input was not finite;
 *    the status returned says which.
 * stream: cudaStream_t as void*; the call enqueues one host-to-device copy of
 *    its plan (from pageable host memory, so the call may wait while the
 *    driver stages it), a fill of f_out and one kernel, then synchronises the
 *    stream to read the kernel's status word back.  Returns BD3MG_ETIMEOUT
 *    when a wait of the kernel ran out and BD3MG_ENONFINITE for a non-finite
 *    objective; f_out is NaN or non-finite then.
 * err, err_len: optional buffer that receives a one-line message.
 *
 * The first call on each device performs that device's set-up (it looks up
 * the array's device address with that device current); make that first call
 * before any stream capture.  All calls share the array and each overwrites
 * it (the completion ticket and status words are cleared at every call), so
 * calls that overlap on the GPU race: order them on one stream.  Returns
 * BD3MG_EINVAL, with a message, when the volume's work list and PSF factor rows
 * do not fit the array (roughly: more than ~20 000 tiles of 32x32 voxels times
 * z-chunks, or more than a few thousand depth slices). */
bd3mg_status bd3mg_objective_noalloc(const bd3mg_params *p, const float *x, const float *y, double *f_out,
                                     void *stream, char *err, size_t err_len);

/* The metric constant L of each volume (nvol doubles): the caller's lipschitz
 * or the library's bound for BD3MG_METRIC_LIPSCHITZ (computed at creation from
 * the factored PSF), and that bound also when the volume uses the majorant. */
bd3mg_status bd3mg_lipschitz(bd3mg_ctx *ctx, double *L);

const char *bd3mg_error_string(bd3mg_ctx *ctx);
const char *bd3mg_status_string(bd3mg_status s);

/* Release the context and its device memory (NULL is a no-op). */
void bd3mg_destroy(bd3mg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* BD3MG_H */
