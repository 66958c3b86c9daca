/*
 * muster.h -- C ABI of the GB300 registration engine for MUSTER
 * (Grodem et al., "MUSTER: Longitudinal Deformable Registration by Composition
 * of Consecutive Deformations", arXiv 2412.14671).
 *
 * The engine registers an N-session 3D image series: it optimises N-1
 * stationary velocity fields phi_{i,i+1} (Sec. Parameterization of consecutive
 * diffeomorphism), exponentiates them by scaling and squaring (Alg. 1), composes
 * them into the deformations between every ordered pair of sessions
 * (Eq. cum_deformation), warps every session onto every other one, and minimises
 * sum_i sum_{j != i} Sim(I_i, I_j o Phi_ji^i) + L_reg (Sec. MUSTER overview) with
 * Sim = SiLNCC or LNCC (Sec. Image Similarity Metric) and L_reg of Eq. reg_sum,
 * by Adam with warm-up and cosine decay over a multi-resolution pyramid
 * (Sec. Implementation Details). Every step runs in CUDA kernels on one GPU.
 *
 * Conventions
 *   - Return value: MUSTER_OK (0) or a negative MUSTER_E* code; the message of
 *     the last failure is muster_last_error(ctx). A failed call leaves the
 *     context usable unless it returned MUSTER_ECUDA from a kernel launch.
 *   - Volumes are float32, row-major (D, H, W), W contiguous. Sessions are
 *     0-based. Vector fields are planar (3, D, H, W); component c is the
 *     displacement along axis c (0 = D, 1 = H, 2 = W) in voxel units of the grid
 *     the field lives on.
 *   - Pair (j, i) means the deformation Phi_ji^i that pulls image j onto the grid
 *     of image i (Sec. Background: I_j o Phi_ji^i ~ I_i).
 *   - Velocities live on a grid flow_factor times coarser than the images of the
 *     current pyramid level (Sec. Implementation Details).
 *   - Pointers marked "device" are CUDA device pointers valid on the current
 *     device; "host" pointers are ordinary host memory. Input buffers are never
 *     retained after a call returns; output buffers belong to the caller.
 *   - All work is issued on the context's stream (muster_set_stream; default:
 *     the legacy default stream). Calls that return numbers to host memory
 *     synchronise that stream. One context must not be used by two host threads
 *     at once.
 */
#ifndef MUSTER_H
#define MUSTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define MUSTER_OK 0
#define MUSTER_EINVAL (-1)   /* bad argument: NULL, shape, range, NaN input */
#define MUSTER_ESTATE (-2)   /* call out of order, e.g. step before set_images */
#define MUSTER_EOOM (-3)     /* device allocation failed */
#define MUSTER_ECUDA (-4)    /* CUDA runtime error (message has the CUDA error string) */
#define MUSTER_ETIMEOUT (-5) /* a bounded wait ran out: on the host (MUSTER_SYNC_TIMEOUT_S seconds,
                                 default 1800), or in a kernel waiting for its own input copies.
                                 The results of that call are not valid; work it issued may
                                 still be running, and a host output buffer of that call may
                                 still be written until the stream drains. The context stays
                                 usable: a later call that synchronises waits for that work. */
#define MUSTER_ENUMERIC (-6) /* the loss became NaN or Inf */

/* similarity (Sec. Image Similarity Metric) */
#define MUSTER_SILNCC 0 /* the paper's scale-invariant LNCC, its default */
#define MUSTER_LNCC 1   /* 1 - local normalised cross-correlation, Eq. LNCC */

/* optimiser (Sec. Implementation Details) */
#define MUSTER_ADAM 0
#define MUSTER_SGD 1 /* plain gradient steps with the same schedule (for parity tests) */

/* field kinds for muster_get_fields */
#define MUSTER_VELOCITY 0  /* phi_{i,i+1}: (3,d,h,w) on the flow grid (S(theta) when smoothing); j ignored */
#define MUSTER_PAIR_FLOW 1 /* displacement of Phi_ji^i on the flow grid (3,d,h,w) */
#define MUSTER_PAIR_DISP 2 /* displacement of Phi_ji^i on the image grid (3,D,H,W), image voxels
                              (with rigid registration: the total deformation of Sec. Rigid Registration) */
#define MUSTER_WARPED 3    /* I_j o Phi_ji^i on the image grid (D,H,W) */
#define MUSTER_IMAGE 4     /* pyramid image I_i at the current level (D,H,W); j ignored */
#define MUSTER_GRADIENT 5  /* gradient of the last step or eval with respect to the parameters
                              theta_{i,i+1} (3,d,h,w) (dL/dphi unless smooth_omega > 0); j ignored */
#define MUSTER_JACOBIAN 6  /* det of the spatial Jacobian of Phi_ji^i on the image grid (D,H,W)
                              (Fig. 1c; central differences, one-sided at the edges; the deformable
                              part only, without the rigid adjustment) */
#define MUSTER_PARAMETERS 7 /* theta_{i,i+1} (3,d,h,w): the optimised parameters; equal to the
                               velocity unless smooth_omega > 0 (then VELOCITY is S(theta)) */

typedef struct muster_ctx muster_ctx;

typedef struct {
  int n_levels;           /* 1..8 pyramid levels; level l has images down-sampled 2^(n_levels-1-l) times */
  int steps_per_level[8]; /* gradient steps per level, coarsest first (paper: 200,200,100) */
  int flow_factor;        /* image-to-flow grid factor; must be 2 (Sec. Implementation Details) */
  int n_squarings;        /* K of Alg. 1: 0..20 */
  int window;             /* odd window edge w, 3..11 (paper: 3) */
  int similarity;         /* MUSTER_SILNCC or MUSTER_LNCC */
  float alpha_ss;         /* weight of L_ss (Eq. reg_sum; value not given in the paper) */
  float alpha_l2;         /* weight of L_L2 */
  float alpha_ts;         /* weight of L_ts */
  float sim_eps;          /* guard added to S_FF (SiLNCC) or to S_FF*S_WW (LNCC); >= 0 */
  int optimizer;          /* MUSTER_ADAM or MUSTER_SGD */
  float lr;               /* peak learning rate, flow voxels per step */
  float beta1, beta2, adam_eps;
  float warmup_frac;      /* fraction of each level's steps spent in linear warm-up (paper: 0.2) */
  int deterministic;      /* 1: the scatter halves of the squaring and composition adjoints add
                             fixed-point terms whose sums are exact, so every run (alone or beside
                             other work) gives the same bits; 0: floating-point vector reductions,
                             whose sums depend on the order in which they arrive */
  int recompute_squaring; /* 1: keep only u_0 and u_K of each exponential, recompute the rest */
  int pair_batch;         /* ordered pairs per image-grid launch; 0 = automatic (all pairs whose
                             image-grid scratch fits in 16 GiB); always capped so that a launch's
                             depth planes or chunks times pairs fit the 65535 grid rows of CUDA */
  float smooth_omega;     /* Gaussian parameterisation (Sec. Regularization, Appendix Gaussian
                             Smoothing): > 0 optimises theta with velocity phi = S(theta), S the
                             multiplication of the DFT of each component by exp(-1/2 (f/omega)^2),
                             f in cycles per mm on the flow grid (periodic); 0 = off (phi = theta) */
  int rigid;              /* 1: rigid registration in parallel (Sec. Rigid Registration): every pair
                             pulled onto grid i >= 1 also moves by r_i(p) = R_i (p - c) + c + t_i - p,
                             R_i = R_0(a0) R_1(a1) R_2(a2) (R_k rotates the plane of the two other
                             axes), c the centre of the image grid, t_i in voxels of the finest
                             level; the six parameters of each session follow the velocity schedule */
  float rigid_lr;         /* step of the translations (voxels); the angles step rigid_lr divided by
                             half the largest image extent (radians) */
  /* launch configuration (not in the paper; chosen by the autotuner of the Python package or
     left at 0 for the defaults) */
  int flow_nf;            /* fields per thread of the flow-grid gather kernels: 1 or 2 (0 = 2); the
                             results do not depend on it */
  int chunk_pct;          /* D-chunk rule of the image-grid kernels: the CTA count up to which a
                             pair's depth is split, in percent of the default (1..800; 0 = 100).
                             Chunks change where the window sums restart and the order of the
                             loss partial sums, so results differ in the last bits between values
                             (each value is reproducible) */
  /* optional device allocator (e.g. a framework's caching allocator); both or neither */
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* alloc_user;
} muster_params;

/* Fills *p with the library defaults: 1 level of 100 steps, flow_factor 2, K 7,
   window 3, SiLNCC, alpha = (1, 0.01, 0), sim_eps 1e-6, Adam(lr 0.05, 0.9, 0.999,
   1e-8), warmup 0.2, atomic adjoint, stored squarings, automatic batching, no Gaussian
   parameterisation, no rigid registration (rigid_lr 0.5). */
void muster_default_params(muster_params* p);

/* Creates a context for n_sessions (>= 2) images of shape[3] = (D, H, W) voxels
   with spacing[3] mm (recorded and reported; the objective is in voxel units).
   Allocates every device buffer of the whole schedule up front; MUSTER_EOOM if
   they do not fit. *out is NULL on failure. */
int muster_create(const int64_t shape[3], int n_sessions, const double spacing[3],
                  const muster_params* params, muster_ctx** out);

/* Issue all further work on this cudaStream_t (NULL = legacy default stream). Work
   issued after the switch is ordered after the work issued before it (the new stream
   waits on an event of the old one); nothing waits on the host. */
int muster_set_stream(muster_ctx* ctx, void* cuda_stream);

/* Copies the N images (N*D*H*W floats, host or device per on_device) into the
   context and builds the pyramid. times: N acquisition times (host, strictly
   increasing; only L_ts uses them) or NULL for t_i = i. Rejects NaN/Inf images.
   Resets the optimisation state (no level selected). */
int muster_set_images(muster_ctx* ctx, const float* imgs, int on_device, const double* times);

/* Selects pyramid level `level`. If the context currently holds level-1, the
   velocities are prolonged (trilinear, doubled; Sec. Implementation Details),
   otherwise they start at zero. Resets Adam and the step counter. */
int muster_set_level(muster_ctx* ctx, int level);

/* Replaces the parameters theta of the current level (the velocities unless smooth_omega
   > 0): v = (N-1, 3, d, h, w) floats, host or device per on_device. Does not reset Adam. */
int muster_set_velocity(muster_ctx* ctx, const float* v, int on_device);

/* One gradient step at the current level: forward, hand-written adjoint and
   optimiser update. loss_out (host, nullable) receives the loss before the
   update; passing it synchronises the stream. MUSTER_ESTATE past the level's
   last step or without a level. */
int muster_step(muster_ctx* ctx, double* loss_out);

/* The whole schedule: every level from the coarsest, steps_per_level[l] steps
   each. final_loss (host, nullable) = loss of the last step. Returns
   MUSTER_ENUMERIC if any step's loss was not finite. Steps after the first of each
   level replay a CUDA graph of one step (environment MUSTER_GRAPHS=0 disables it). */
int muster_run(muster_ctx* ctx, double* final_loss);

/* Advances the same schedule by up to max_steps gradient steps, entering the next
   level (with prolongation) when a level is done, and returns without waiting for
   the GPU. The first call after set_images (or after run) starts at level 0.
   finished (host, nullable) = 1 once every level has run. Lets one host thread
   interleave many contexts, each on its own stream. */
int muster_advance(muster_ctx* ctx, int max_steps, int* finished);

/* Device bytes that muster_create would allocate for this problem (for admission
   control of concurrent registrations). No device is needed. */
int muster_footprint(const int64_t shape[3], int n_sessions, const muster_params* params, size_t* bytes);

/* Loss and gradient at `level` for parameters v (device, (N-1,3,d,h,w) of that level's
   flow grid: the velocities, or theta with smooth_omega > 0, where the gradient is taken
   with respect to theta; NULL = the current parameters, only if level is current).
   loss (host, nullable) = total; grad (device, nullable) same layout as v.
   Does not change the velocities, the optimiser state or the step counter. */
int muster_eval(muster_ctx* ctx, const float* v, int level, double* loss, float* grad);

/* Copies field `kind` (MUSTER_VELOCITY ...) of session i, or of pair (j, i), at
   the current level into out (host or device per on_device). Pair fields are
   recomputed from the current velocities. */
int muster_get_fields(muster_ctx* ctx, int kind, int i, int j, float* out, int on_device);

/* Loss terms of the last step or eval (host): {total, Sim summed over pairs,
   L_ss, L_L2, L_ts}, the last three unweighted. Synchronises. */
int muster_get_loss_split(muster_ctx* ctx, double out[5]);

/* Losses of the schedule's steps up to the current one (host), in schedule order:
   entry steps_per_level[0] + ... + steps_per_level[l-1] + s is the loss of step s
   of level l (levels entered by set_level without running the earlier ones leave
   those entries unspecified). *n in: capacity, out: count. Synchronises. */
int muster_get_loss_history(muster_ctx* ctx, double* out, size_t* n);

/* Rigid parameters (host, (N-1) x 6 doubles: angles a0, a1, a2 in radians, translation in
   voxels of the finest level) of sessions 1..N-1, and (grad, nullable) their gradient of
   the last step or eval. MUSTER_ESTATE when rigid registration is off. Synchronises. */
int muster_get_rigid(muster_ctx* ctx, double* rho, double* grad);
/* Replaces the rigid parameters (same layout); run / advance start from zero at the
   coarsest level, so set them after set_level to evaluate or continue from them. */
int muster_set_rigid(muster_ctx* ctx, const double* rho);

/* Image and flow dims of a pyramid level (host outputs). */
int muster_level_dims(const muster_ctx* ctx, int level, int64_t img[3], int64_t flow[3]);

/* The paper has no counterpart (bookkeeping of the schedule): the current pyramid level
   (-1 while none is selected, e.g. right after set_images) and the gradient steps issued
   at it so far (host outputs, nullable). No device work, no synchronisation. */
int muster_get_level(const muster_ctx* ctx, int* level, int* step);

/* Checkpoint: level, step, velocities and Adam moments. With buf NULL, *n gets
   the size needed. set_state requires a context of the same shape, sessions and
   parameters. */
int muster_get_state(muster_ctx* ctx, void* buf, size_t* n);
int muster_set_state(muster_ctx* ctx, const void* buf, size_t n);

/* Per-kernel timing with CUDA events on the context's stream, for roofline
   reports. Between begin and end, launches made outside a step graph (the first step
   of a level, muster_step, muster_eval, level set-up) are bracketed by events. Of the
   steps that muster_run / muster_advance replay as CUDA graphs, steps 0, 8, 16, ... of
   each level replay a copy of the step graph with an event record node around every
   kernel, and the others replay the plain graph and are only counted; so the window runs
   at close to the speed of an unprofiled one. The events are read at muster_profile_end
   (which synchronises; it also runs at a later muster_profile_begin if end was skipped). */
int muster_profile_begin(muster_ctx* ctx);
int muster_profile_end(muster_ctx* ctx);
/* Entry k of the kernel table: name, timed launches, their summed device milliseconds
   and algorithmic bytes (compulsory reads + writes) in the profiled window.
   Returns MUSTER_EINVAL when k is past the end. */
int muster_kernel_stat(const muster_ctx* ctx, int k, const char** name, int64_t* launches,
                       double* ms, double* bytes);
/* Every launch of kernel k in the profiled window, timed or not (*launches >= the
   timed count of muster_kernel_stat). MUSTER_EINVAL when k is past the end or
   launches is NULL. */
int muster_kernel_launches(const muster_ctx* ctx, int k, int64_t* launches);

/* Last error message of this context ("" if none); ctx may be NULL for errors
   of muster_create. */
const char* muster_last_error(const muster_ctx* ctx);

/* Frees the context and its device memory; NULL-safe. */
void muster_destroy(muster_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
