/*
 * muster_ops.h -- stateless entry points of single steps of MUSTER's
 * registration loop (arXiv 2412.14671), on caller-owned device buffers.
 *
 * They run the same kernels as the engine of muster.h and exist so that each
 * step can be used, and checked, on its own. Conventions are those of muster.h:
 * float32, row-major (D, H, W), vector fields planar (3, D, H, W). Every pointer
 * is a device pointer unless marked host. `stream` is a cudaStream_t (NULL = the
 * legacy default stream). Functions returning host values synchronise `stream`.
 * Return value: MUSTER_OK or a negative MUSTER_E* code of muster.h; the message
 * is muster_ops_last_error() (per thread).
 */
#ifndef MUSTER_OPS_H
#define MUSTER_OPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Multi-resolution pyramid step (Sec. Implementation Details; the down-sampling
   method is not given in the paper): out = 2x2x2 mean of `in`, out dims
   ceil(D/2) x ceil(H/2) x ceil(W/2), the last plane replicated for odd sizes.
   n_images volumes of the same shape, back to back. */
int muster_op_downsample(const float* in, int n_images, int64_t D, int64_t H, int64_t W,
                         float* out, void* stream);

/* Exp of Alg. 1 in the displacement form of its comment: u = Exp(sign * phi) - identity
   after K squarings u <- u + u o (x + u) from u = sign * phi / 2^K, trilinear
   sampling with clamp-to-edge. phi, u: (3, D, H, W); sign is +1 or -1.
   Allocates and frees device scratch of 20 * D*H*W floats on `stream`. */
int muster_op_exp(const float* phi, int64_t D, int64_t H, int64_t W, int K, float sign,
                  float* u, void* stream);

/* Windowed similarity of Eq. sum_lncc / Eq. sim_loss: the mean over the valid
   w^3 windows of SiLNCC_R (kind MUSTER_SILNCC) or LNCC_R (MUSTER_LNCC) between
   fixed F and moving W, and (dLdW, nullable) its gradient with respect to W.
   loss: host double. eps: the guard of muster_params.sim_eps. Returns 0 loss and
   a zero gradient when no window fits. Allocates and frees device scratch of
   about 5 * D*H*W floats on `stream`. */
int muster_op_similarity(const float* F, const float* W, int64_t D, int64_t H, int64_t Wd,
                         int window, int kind, float eps, double* loss, float* dLdW,
                         void* stream);

/* Largest volume (voxels) accepted by muster_op_similarity_noalloc: 128^3. */
#define MUSTER_NOALLOC_MAX_VOXELS 2097152

/* The paper has no counterpart to this entry point: it exists for callers that
   must not allocate device memory at call time -- code running under a fixed
   memory budget, inside a host framework that owns every allocation, or on a
   path where cudaMalloc/cudaFree (or a caching allocator) would stall or is not
   permitted. It computes exactly what muster_op_similarity computes, with the
   same kernels, but its scratch (about 43 MB: coefficient and window-statistics
   volumes for up to MUSTER_NOALLOC_MAX_VOXELS voxels and the partial sums) is one fixed device
   array inside this library, which every GPU that loads the library holds
   until the process exits. It calls no cudaMalloc, cudaFree or allocating
   library routine; the caller still passes F, W and dLdW.
   - Volumes larger than MUSTER_NOALLOC_MAX_VOXELS, or shapes that need more than
     2^17 partial sums, return MUSTER_EINVAL with a message.
   - The first call on a device looks up the array's device address with that
     device current (cudaGetSymbolAddress) and caches it; make that first call
     before any stream capture.
   - All calls share the one array, and it keeps the last call's contents; the
     call clears what must start at zero. Calls that overlap on the GPU (on
     different streams, or from different host threads) race on the array:
     serialise them.
   Errors are reported by muster_ops_last_error(). */
int muster_op_similarity_noalloc(const float* F, const float* W, int64_t D, int64_t H, int64_t Wd,
                                 int window, int kind, float eps, double* loss, float* dLdW,
                                 void* stream);

/* Determinant of the spatial Jacobian of x -> x + u(x) (the Jacobian determinant maps of
   Sec. Sensitivity to clinical outcomes and Fig. 1c): J = det(I + grad u) with central
   differences, one-sided on the first and last plane of an axis and 0 along an axis of
   one plane. u: (3, D, H, W) displacement in voxels; J: (D, H, W). No scratch. */
int muster_op_jacobian_det(const float* u, int64_t D, int64_t H, int64_t W, float* J, void* stream);

/* Deformation metrics of Sec. Evaluation Metrics between a reference displacement
   u_true and an estimate u_est, both (3, D, H, W), over the voxels where roi (uint8,
   (D, H, W), nullable = every voxel) is non-zero. out (host, 16 doubles): [0] Eu, the
   mean Euclidean distance; [1] PCC of the mean-centred vector fields; [2] B =
   trace(A)/3 of the least-squares fit u_est = A u_true + b; [3..11] A row-major;
   [12..14] b; [15] the number of ROI voxels (all 0 when it is 0). Each voxel's terms and
   each thread's running sums are double-float values (a pair of floats, about 48
   significant bits); the per-CTA and final sums are FP64 in a fixed order over a grid of
   three CTAs per SM (at most 768), so a device gives the same result on every run.
   Allocates and frees about 150 KB of device scratch on `stream`; synchronises it. */
int muster_op_deformation_metrics(const float* u_true, const float* u_est, const uint8_t* roi, int64_t D,
                                  int64_t H, int64_t W, double out[16], void* stream);

/* Per-thread message of the last failed muster_op_* call. */
const char* muster_ops_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
