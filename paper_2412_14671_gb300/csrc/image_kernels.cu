// image_kernels.cu -- small kernels on the image grid of a pyramid level: the
// 2x2x2 pyramid, the displacement upsample for output, the non-finite input
// check and the deterministic loss reduction. The warp and its adjoint are in
// warp_kernels.cu, the windowed similarity and its adjoint in sim_kernels.cu.
#include <algorithm>
#include <cfloat>

#include "kernels.h"

namespace muster {

namespace {
constexpr int kThreads = 256;

__host__ __device__ inline unsigned blocks_for(size_t V) { return (unsigned)((V + kThreads - 1) / kThreads); }

// ---- pyramid: 2x2x2 mean, last plane replicated for odd sizes
__global__ void k_down2(const float* __restrict__ in, Dims n, float* __restrict__ out, Dims m) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int Vm = (int)vox(m);
  if (v >= Vm) return;
  const float* I = in + (size_t)blockIdx.y * vox(n);
  int z, y, x;
  unflat(m, v, z, y, x);
  const int z0 = 2 * z, z1 = min(2 * z + 1, n.n0 - 1), y0 = 2 * y, y1 = min(2 * y + 1, n.n1 - 1);
  const int x0 = 2 * x, x1 = min(2 * x + 1, n.n2 - 1);
  auto at = [&](int a, int b, int c) { return I[((size_t)a * n.n1 + b) * n.n2 + c]; };
  const float s = ((at(z0, y0, x0) + at(z0, y0, x1)) + (at(z0, y1, x0) + at(z0, y1, x1))) +
                  ((at(z1, y0, x0) + at(z1, y0, x1)) + (at(z1, y1, x0) + at(z1, y1, x1)));
  out[(size_t)blockIdx.y * Vm + v] = 0.125f * s;
}

// voxel-centre map from image index p to flow coordinate: (p + 1/2)/2 - 1/2
__device__ __forceinline__ float centre(int p) { return 0.5f * (float)p - 0.25f; }

__global__ void k_upsample_disp(const float4* __restrict__ U, Dims nf, Dims ni, float* __restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int Vi = (int)vox(ni);
  if (v >= Vi) return;
  int z, y, x;
  unflat(ni, v, z, y, x);
  const float4 u = sample4(U, nf, centre(z), centre(y), centre(x));
  out[v] = 2.f * u.x;
  out[(size_t)Vi + v] = 2.f * u.y;
  out[2 * (size_t)Vi + v] = 2.f * u.z;
}

__global__ void k_count_nonfinite(const float* __restrict__ x, size_t n, int* __restrict__ count) {
  int bad = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad += isfinite(x[i]) ? 0 : 1;
  bad = __reduce_add_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(count, bad);
}


// ---- deterministic loss reduction (fixed order), one CTA
__global__ void k_loss_reduce(const double* __restrict__ sp, int nsp, const double* __restrict__ rp, int nrp,
                              double inv_NR, double inv_F, double inv_Nm2, float ass, float al2, float ats,
                              double* __restrict__ out, double* __restrict__ hist, int* __restrict__ step,
                              int* __restrict__ flag, int advance) {
  __shared__ double sh[4][kThreads];
  double a = 0.0, b = 0.0, c = 0.0, e = 0.0;
  for (int i = threadIdx.x; i < nsp; i += kThreads) a += sp[i];
  for (int i = threadIdx.x; i < nrp; i += kThreads) {
    b += rp[3 * i];
    c += rp[3 * i + 1];
    e += rp[3 * i + 2];
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  sh[2][threadIdx.x] = c;
  sh[3][threadIdx.x] = e;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sim = sh[0][0] * inv_NR, lss = sh[1][0] * inv_F, ll2 = sh[2][0] * inv_F, lts = sh[3][0] * inv_Nm2;
    const double tot = sim + (double)ass * lss + (double)al2 * ll2 + (double)ats * lts;
    out[0] = tot;
    out[1] = sim;
    out[2] = lss;
    out[3] = ll2;
    out[4] = lts;
    if (!isfinite(tot)) *flag = 1;
    if (hist) hist[*step] = tot;
    if (advance) *step += 1;
  }
}

}  // namespace

void launch_down2(const float* in, Dims n, float* out, Dims m, int n_images, cudaStream_t s) {
  k_down2<<<dim3(blocks_for(vox(m)), n_images), kThreads, 0, s>>>(in, n, out, m);
}
void launch_count_nonfinite(const float* x, size_t n, int* count, cudaStream_t s) {
  const unsigned b = (unsigned)std::min<size_t>((n + kThreads - 1) / kThreads, (size_t)16 * device_sm_count());
  if (b) k_count_nonfinite<<<b, kThreads, 0, s>>>(x, n, count);
}
void launch_upsample_disp(const float4* U, Dims nf, Dims ni, float* out, cudaStream_t s) {
  k_upsample_disp<<<blocks_for(vox(ni)), kThreads, 0, s>>>(U, nf, ni, out);
}

void launch_loss_reduce(const double* sim_part, int n_sim, const double* reg_part, int n_reg, double inv_NR,
                        double inv_F, double inv_Nm2, float a_ss, float a_l2, float a_ts, double* out, double* hist,
                        int* step, int* flag, int advance, cudaStream_t s) {
  k_loss_reduce<<<1, kThreads, 0, s>>>(sim_part, n_sim, reg_part, n_reg, inv_NR, inv_F, inv_Nm2, a_ss, a_l2, a_ts,
                                       out, hist, step, flag, advance);
}

}  // namespace muster
