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

/* Per-thread message of the last failed muster_op_* call. */
const char* muster_ops_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
