/*
 * muster_oracle.h -- FP64 CPU oracle of MUSTER's registration loop.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use this library. The product (the CUDA library) neither
 * includes this header nor links this code, and this code includes nothing of
 * the product.
 *
 * Conventions (shared by every function below):
 *   - a scalar volume has dims n[3] = (D, H, W), row-major, W contiguous;
 *   - a vector field is planar: 3 consecutive scalar volumes, component c is the
 *     displacement along axis c (0 = D, 1 = H, 2 = W), in voxel units of its grid;
 *   - sessions are 0-based; phi[m] (m = 0..N-2) is the velocity phi_{m,m+1};
 *   - U[k][i] is the displacement of Phi_{ki}^i: it pulls image k onto grid i.
 */
#ifndef MUSTER_ORACLE_H
#define MUSTER_ORACLE_H
#include <stddef.h>

#define OR_SILNCC 0
#define OR_LNCC 1
#define OR_ADAM 0
#define OR_SGD 1

typedef struct {
  int n_levels;          /* pyramid levels, coarsest first */
  int steps[8];          /* gradient steps per level */
  int flow_factor;       /* image-to-flow grid factor (2) */
  int K;                 /* scaling-and-squaring steps */
  int window;            /* odd window edge w */
  int sim_kind;          /* OR_SILNCC or OR_LNCC */
  int optimizer;         /* OR_ADAM or OR_SGD */
  int pad_;
  double alpha_ss, alpha_l2, alpha_ts;
  double sim_eps;
  double lr, beta1, beta2, adam_eps, warmup_frac;
  /* Gaussian parameterisation (Sec. Regularization, Appendix Gaussian Smoothing):
     phi = S(theta), S multiplies the DFT of each component by exp(-1/2 (f/omega)^2) with f
     the frequency in cycles per mm; smooth_omega <= 0 turns it off. spacing = voxel size
     (mm) of the images handed to or_loss_grad (or_run: of the finest level); the flow grid
     voxel is flow_factor times larger. */
  double smooth_omega;
  double spacing[3];
  /* rigid registration in parallel (Sec. Rigid Registration): rigid = 1 adds, for every pair
     pulled onto grid i >= 1, the displacement r_i(p) = R_i (p - c) + c + t_i - p of session i
     (Euler angles rho[0..2] in radians, R = R_0 R_1 R_2 with R_a the rotation in the plane of
     the two other axes; translation rho[3..5] in voxels of the finest level; c the centre
     of the level's image grid). rigid_lr: step of the translations (voxels); the angles
     step rigid_lr / (half the largest finest extent). */
  int rigid;
  int pad2_;
  double rigid_lr;
} or_params;

/* trilinear sampling with clamp-to-edge; grad (nullable) = d value / d q */
double or_sample(const double* g, const int n[3], const double q[3], double grad[3]);

/* Alg. 1 (displacement form): u = Exp(sign*phi) - identity; inter (nullable) gets u_0..u_K */
void or_exp(const double* phi, const int n[3], int K, double sign, double* u, double* inter);
/* adjoint of or_exp: g_phi = (d u / d phi)^T g_u */
void or_exp_adjoint(const double* phi, const int n[3], int K, double sign,
                    const double* g_u, double* g_phi);

/* Eq. cum_deformation: all N*N pair displacements (diagonal = 0) from the
   consecutive forward (up[m] = Exp(phi_m)) and backward (um[m] = Exp(-phi_m)) maps */
void or_compose(const double* up, const double* um, int N, const int n[3], double* U);
void or_compose_adjoint(const double* up, const double* um, int N, const int n[3],
                        const double* gU, double* g_up, double* g_um);

/* flow grid -> image grid displacement (voxel-centre alignment), and its adjoint */
void or_upsample(const double* U, const int nf[3], const int ni[3], int f, double* Ut);
void or_upsample_adjoint(const double* gUt, const int nf[3], const int ni[3], int f, double* gU);

/* W(p) = I(p + Ut(p)), and gUt(p) = gW(p) * grad I(p + Ut(p)) */
void or_warp(const double* I, const int ni[3], const double* Ut, double* W);
void or_warp_adjoint(const double* I, const int ni[3], const double* Ut, const double* gW,
                     double* gUt);

/* Eq. sum_lncc / Eq. sim_loss: mean over valid windows; dW (nullable) = gradient */
double or_similarity(const double* F, const double* W, const int n[3], int w, int kind,
                     double eps, double* dW);
/* per-window statistics for tests: centred sums of every valid window, row-major
   over the (n - w + 1) centre grid; any output pointer may be NULL */
void or_window_stats(const double* F, const double* W, const int n[3], int w, double* muF,
                     double* muW, double* Sff, double* Sww, double* Sfw);

/* Eq. reg_ss, the L2 term, Eq. reg_ts: L[3] = unweighted (L_ss, L_L2, L_ts);
   grad (nullable) = gradient of alpha_ss L_ss + alpha_l2 L_L2 + alpha_ts L_ts */
void or_regulariser(const double* phi, int N, const int n[3], const double* t,
                    double a_ss, double a_l2, double a_ts, double L[3], double* grad);

/* 2x2x2 mean (odd sizes replicate the last plane) and velocity prolongation */
void or_downsample2(const double* in, const int n[3], double* out);
void or_prolong(const double* v, const int nc[3], const int nf[3], double* out);

/* Appendix Gaussian Smoothing on a periodic grid: out = S(in) for one scalar volume with
   voxel size h[3] (mm): the DFT along each axis multiplied by exp(-1/2 (f/omega)^2), f in
   cycles per mm, written as the equivalent circular convolution whose taps are the inverse
   DFT of that response. S is symmetric, so it is also its own adjoint.
   parity pinned by: numpy.fft, single Fourier modes, constants, symmetry. */
void or_smooth(const double* in, const int n[3], const double h[3], double omega, double* out);

/* total loss (Sec. MUSTER overview) and its gradient at one pyramid level.
   split = (sim, L_ss, L_L2, L_ts); returns the weighted total. grad nullable.
   With p->smooth_omega > 0, phi holds the parameters theta, the loss is taken at S(theta)
   and grad is the gradient with respect to theta. */
double or_loss_grad(const double* imgs, int N, const int ni[3], const double* phi,
                    const int nf[3], const or_params* p, const double* t, double split[4],
                    double* grad);

/* the loss of or_loss_grad with rigid parameters rho[(N-1)*6] of sessions 1..N-1 (NULL:
   none); tscale = finest-level voxels per voxel of this level (2^(levels-1-l)); grad_rho
   (nullable) = dL/drho (angles, translation in finest voxels) */
double or_loss_grad_rigid(const double* imgs, int N, const int ni[3], const double* theta,
                          const int nf[3], const or_params* p, const double* t, const double* rho,
                          double tscale, double split[4], double* grad, double* grad_rho);
/* the rotation R_0(a0) R_1(a1) R_2(a2) and its derivatives dR[k] = dR / da_k (nullable) */
void or_rotation(const double a[3], double R[9], double dR[27]);

/* optimiser (Sec. Implementation Details) */
double or_lr(int step, int T, double lr, double warmup_frac);
void or_adam_step(double* theta, double* m, double* v, const double* g, size_t n, int step,
                  double lr_t, double b1, double b2, double eps);

/* whole multi-level registration; theta_out = finest-level velocities;
   loss_hist (nullable) gets the loss of every step, in order */
double or_run(const double* imgs, int N, const int n[3], const or_params* p, const double* t,
              double* theta_out, double* loss_hist);
/* or_run that also returns the rigid parameters (rho_out (N-1)*6, nullable) */
double or_run_rigid(const double* imgs, int N, const int n[3], const or_params* p, const double* t,
                    double* theta_out, double* loss_hist, double* rho_out);

/* Determinant of the spatial Jacobian of the map x -> x + u(x) on u's grid (the maps of
   Sec. Sensitivity to clinical outcomes, Fig. 1c): det(I + grad u), each derivative by a
   central difference, one-sided on the first and last plane of an axis, 0 along an axis
   of one plane. parity pinned by: affine fields (exact), numpy gradient on random fields. */
void or_jacobian_det(const double* u, const int n[3], double* J);

/* Sec. Evaluation Metrics over the voxels with roi != 0 (roi NULL: every voxel), for two
   displacement fields: out[0] = Eu (mean Euclidean distance), out[1] = PCC of the
   mean-centred vector fields, out[2] = B = trace(A)/3 of the least-squares fit
   u_est = A u_true + b, out[3..11] = A (row-major), out[12..14] = b, out[15] = ROI voxels */
void or_deformation_metrics(const double* u_true, const double* u_est, const unsigned char* roi,
                            const int n[3], double out[16]);

/* grid sizes used by or_run: level l image dims and flow dims */
void or_level_dims(const int n[3], int n_levels, int level, int flow_factor, int ni[3],
                   int nf[3]);
#endif
