// kernels.h -- host-side launchers of the MUSTER kernels (internal to the library).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace muster {

// ---- descriptor tables (device arrays built by the engine) ----
struct ComposeDesc {  // Unew = Uprev + S[u](x + Uprev)
  const float4* Uprev;
  const float4* u;
  float4* Unew;
};
struct ComposeBwdDesc {  // Gprev += G + J^T G ; gfield += scatter(G) at x + Uprev
  const float4* G;
  const float4* Uprev;
  const float4* u;
  float4* Gprev;
  float4* gfield;
  float4* gacc;     // deterministic mode: fixed-point accumulator pair of gfield (hi, lo)
};
struct AddDesc {  // dst += src
  const float4* src;
  float4* dst;
};
// descriptor tables passed by value as kernel parameters (constant bank): the kernels read
// their operands' addresses without a dependent global load. Launchers split longer lists.
constexpr int kMaxDescPerLaunch = 64;
struct ComposeTab {
  ComposeDesc d[kMaxDescPerLaunch];
};
struct ComposeBwdTab {
  ComposeBwdDesc d[kMaxDescPerLaunch];
};
struct AddTab {
  AddDesc d[kMaxDescPerLaunch];
};
// gradients of the single-step pair maps that complete the input of the first squaring
// adjoint step: field slot f adds G[slot_pair[f] * V + v] (G null: none). Up to
// kMaxDescPerLaunch slots (N <= 33 sessions); longer series add them with launch_add.
struct PairGradTab {
  const float4* G;
  int slot_pair[kMaxDescPerLaunch];
};
struct PairDesc {   // ordered pair (k -> i): pulls image k onto grid i
  const float* Ik;  // moving image (level grid)
  const float* Ii;  // fixed image
  const float* Fs;  // window statistics of the fixed image: mu_F then S_FF planes
  const float4* U;  // pair displacement on the flow grid
  float4* G;        // dL/dU on the flow grid (output of the adjoint)
  int fi;           // index of the fixed image in the image tensor map (SimMaps::F)
};

// TMA descriptors of the window-sum inputs, 4-D (x, y, z, volume) over float32 volumes
// of one level (rows of n2 floats, n2 a multiple of 4; out-of-range boxes read zeros):
//   W: warped images of a pair batch (volume = batch-local pair)
//   F: fixed images (volume = PairDesc::fi)
//   C: similarity coefficients (volume = pair * NC + m)
// Built on the host by make_sim_maps; the kernels fall back to plain loads when a map is
// not valid (odd widths, misaligned bases, no driver entry point).
// n_vol float32 volumes of dims n, one after the other, as a 4-D tensor map (x, y, z,
// volume) read in boxes of box_x x box_y x box_z x 1; false (map unusable) when the width
// or box_x is not a multiple of 4, base is not 16-byte aligned, a box edge is outside
// 1..256 or the driver has no tensor-map encoder
bool encode_volumes(CUtensorMap* m, const float* base, Dims n, int n_vol, int box_x, int box_y, int box_z);

struct SimMaps {
  CUtensorMap W, F, C;
  int fwd_ok, bwd_ok;
};

// deterministic mode: the scatter halves of the squaring and composition adjoints add
// fixed-point terms into accumulator pairs (hi, lo: two float4 fields of V nodes per field)
// whose sums are exact, hence the same in any order (common.cuh)
struct FxArgs {
  float4* ain;           // accumulators completing the input gradient; read and cleared (nullable)
  float4* aout;          // accumulators of this launch's scatter
  const unsigned* gmax;  // bits of the largest |dL/dU| of the step's pair fields
  int off_in, off_out;   // quantum offsets of aout (fx_quantum); off_in is not used by readers
  int* oflow;            // set when a term is too large for the accumulator's headroom
};

struct RegArgs {
  float alpha_ss, alpha_l2, alpha_ts;
  float inv_dt[32];  // 1 / (t_{m+1} - t_m)
  int n_fields;      // N - 1
  int n_sessions;
  float inv2K;       // 1 / 2^K
};

// ---- flow-grid kernels (field_kernels.cu) ----
void launch_prolong(const float4* coarse, Dims nc, float4* fine, Dims nf, int n_fields, cudaStream_t s);
// zero (nullable): a word set to 0 by the launch (the step's largest-gradient word of the
// deterministic adjoint, which later kernels of the step raise)
void launch_exp_init(const float4* theta, float4* u0, int n_fields, Dims n, float scale, cudaStream_t s,
                     unsigned* zero = nullptr);
// nf: fields (or chains) per thread of the flow-grid gather kernels, 1 or 2 (launch
// configuration only: the results are the same)
void launch_squaring(const float4* u, float4* un, int n_fields2, Dims n, cudaStream_t s, int nf = 2);
// exp_init and the first squaring in one launch: u0 = +-scale theta (2 n_fields fields, the
// second half negated) and u1 = its first squaring (scale a power of two)
void launch_squaring_first(const float4* theta, float4* u0, float4* u1, int n_fields, Dims n, float scale,
                           cudaStream_t s, int nf = 2, unsigned* zero = nullptr);
// fx null: Gout (zeroed) += own part and scatter, with vector reductions; fx given
// (deterministic): G_in = fx->ain (+ Gin if not null), own part and scatter into fx->aout.
// pg (nullable): pair gradients added to G_in (PairGradTab). clear_in (atomic mode): each
// node of Gin is cleared after its read
void launch_squaring_bwd(const float4* u, const float4* Gin, float4* Gout, int n_fields2, Dims n, const FxArgs* fx,
                         cudaStream_t s, int nf = 2, const PairGradTab* pg = nullptr, bool clear_in = false);
// d: host arrays of descriptors (copied into the launch's parameters)
void launch_compose(const ComposeDesc* d, int n_chains, Dims n, cudaStream_t s, int nf = 2);
void launch_compose_bwd(const ComposeBwdDesc* d, int n_chains, Dims n, const FxArgs* fx, cudaStream_t s,
                        int nf = 2);
void launch_add(const AddDesc* d, int n, Dims dims, cudaStream_t s);  // d: host array
// gradient of the similarity part + regulariser into grad; loss partials (3 per block);
// fx (nullable, deterministic mode): G0 completed with fx->ain (off_in)
int reg_blocks(Dims n);
void launch_reg_grad(const float4* theta, const float4* G0, float4* grad, double* partials, Dims n,
                     const RegArgs& a, const FxArgs* fx, cudaStream_t s,
                     bool clear_g0 = false);
void launch_adam(float4* theta, float4* m, float4* v, const float4* grad, size_t count,
                 const float* sched, const int* step, int sgd, float beta1, float beta2, float eps,
                 cudaStream_t s);
void launch_f4_to_planar(const float4* in, float* out, int n_fields, size_t V, cudaStream_t s);
void launch_planar_to_f4(const float* in, float4* out, int n_fields, size_t V, cudaStream_t s);

// ---- image-grid kernels (image_kernels.cu) ----
void launch_down2(const float* in, Dims n, float* out, Dims m, int n_images, cudaStream_t s);
// warp_kernels.cu; both require nf = ceil(ni / 2) per axis
// W: n_pairs volumes at stride Wstride; gI (nullable): grad I_k at the sample points, 3 planes per pair
void launch_warp(const PairDesc* pd, int n_pairs, Dims ni, Dims nf, float* W, float* gI, size_t Wstride,
                 const float* rigid, cudaStream_t s);
void launch_upsample_disp(const float4* U, Dims nf, Dims ni, float* out_planar, cudaStream_t s);
// *count += number of NaN/Inf values in x[0, n)
void launch_count_nonfinite(const float* x, size_t n, int* count, cudaStream_t s);
// windowed similarity: forward (coefficients + loss partials) and adjoint (dL/dW)
struct SimGeom {
  int nzc;   // z-chunks
  int tz;    // corner planes per chunk
  int ctas;  // CTAs per pair
};
// batch: the most pairs one launch of the caller takes; it sets the D chunking (fewer,
// longer chunks for larger batches), so every launch of a context must pass the same value
SimGeom sim_geom(Dims ni, int window, int batch);  // sim_kernels.cu
// kernel attributes (dynamic shared memory limits), set once per device; call with the
// device current before any launch or capture on it
cudaError_t prepare_kernels();
// mu_F and S_FF of every window corner of each image: stats = n_images x 2 planes; with
// kind 0 (SiLNCC) the second plane holds 1 / (S_FF + eps) instead of S_FF
void launch_fixed_stats(const float* imgs, int n_images, Dims ni, int window, int kind, float eps, float* stats,
                        cudaStream_t s);
int sim_ncoef(int kind);
// maps for W (capacity n_pairs volumes), the n_images fixed images and the coefficient
// buffer (n_pairs * NC volumes), all with stride nvox(ni) between volumes
void make_sim_maps(SimMaps* m, const float* W, int n_pairs, const float* imgs, int n_images, const float* coef,
                   Dims ni, int window, int kind);
// maps (nullable): TMA staging of the inputs when maps->fwd_ok / bwd_ok; err (nullable) is
// set to 1 if a bounded wait for a copy ran out (the results are then not valid)
void launch_sim_fwd(const PairDesc* pd, int n_pairs, int batch, const float* W, size_t Wstride, float* coef,
                    size_t coef_stride, double* partials, Dims ni, int window, int kind, float eps,
                    const SimMaps* maps, int* err, cudaStream_t s);
void launch_sim_bwd(const PairDesc* pd, int n_pairs, int batch, const float* W, size_t Wstride, const float* coef,
                    size_t coef_stride, float* dLdW, Dims ni, int window, int kind, float scale,
                    const SimMaps* maps, int* err, cudaStream_t s);
// batch: the most pairs one launch of this context takes (n_pairs <= batch); it sets the
// D chunking, so every launch of a context splits a pair the same way.
// rigid_part (nullable): per-CTA sums (12 floats) of dL/dq and dL/dq p^T for the rigid
// gradient, warp_bwd_ctas_per_pair(nf, batch) CTAs per pair, pairs of the launch in order
// maps (nullable): TMA staging of dL/dW and grad I_k when maps->ok and stride is the
// volume of ni (make_warp_bwd_maps over the same buffers); err (nullable) is set when a
// bounded wait for a staged copy runs out
struct WarpBwdMaps {
  CUtensorMap dW, gI;
  int ok;
};
void make_warp_bwd_maps(WarpBwdMaps* m, const float* dLdW, const float* gI, int batch, Dims ni);
cudaError_t prepare_warp_kernels();  // dynamic shared memory limits, once per device
int warp_bwd_ctas_per_pair(Dims nf, int batch);
int warp_bwd_zchunks(Dims nf, int batch);  // D chunks of one pair (grid z = chunks x pairs)
// gmax (nullable): atomicMax of the float bits of the largest |component| of every G written
void launch_warp_bwd(const PairDesc* pd, int n_pairs, int batch, const float* dLdW, const float* gI, size_t stride,
                     Dims ni, Dims nf, float* rigid_part, const WarpBwdMaps* maps, int* err, unsigned* gmax,
                     cudaStream_t s);
// rigid_kernels.cu: rigid registration in parallel (Sec. Rigid Registration)
struct RigidArgs {
  int N, per_pair, sgd;
  float c0, c1, c2;  // centre of the level's image grid
  float tscale;      // finest voxels per voxel of the level
  float lr_base, rigid_lr, rmax, b1, b2, eps;
};
void launch_rigid_table(const float* rho, float* tab, const RigidArgs& a, cudaStream_t s);
void launch_rigid_grad(const float* rpart, const float* rho, float* grad, const RigidArgs& a, cudaStream_t s);
void launch_rigid_step(float* rho, float* m, float* v, const float* grad, const float* sched, const int* step,
                       float* tab, const RigidArgs& a, cudaStream_t s);
void launch_add_rigid(float* u, Dims n, const float* row, cudaStream_t s);
// Gaussian smoothing of float4 flow fields (Appendix Gaussian Smoothing): circular
// convolution along axes 0, 1, 2 with device taps; out may be in (tmp_a, tmp_b distinct)
struct SmoothAxis {
  const float* taps;  // m taps of the axis (device), symmetric
  int lo, hi;         // offsets summed: lo..hi
};
void launch_smooth(const float4* in, float4* out, float4* tmp_a, float4* tmp_b, int n_fields, Dims n,
                   const SmoothAxis axes[3], cudaStream_t s);
// metrics_kernels.cu: det(I + grad u) of a planar displacement, and the deformation
// metrics (out: 16 doubles on the device) with scratch of metrics_scratch_doubles()
void launch_jacobian_det(const float* u, Dims n, float* J, cudaStream_t s);
size_t metrics_scratch_doubles();
void launch_deformation_metrics(const float* ut, const float* ue, const unsigned char* roi, Dims n, double* scratch,
                                double* out, cudaStream_t s);
// single-CTA deterministic loss reduction; writes out[0..4], hist[*step], flag, ++*step
void launch_loss_reduce(const double* sim_part, int n_sim, const double* reg_part, int n_reg,
                        double inv_NR, double inv_F, double inv_Nm2, float a_ss, float a_l2,
                        float a_ts, double* out, double* hist, int* step, int* flag, int advance,
                        cudaStream_t s);

}  // namespace muster
