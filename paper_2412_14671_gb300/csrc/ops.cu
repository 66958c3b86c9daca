// ops.cu -- stateless entry points of include/muster_ops.h: single steps of the
// registration loop on caller-owned device buffers, running the engine's kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "kernels.h"
#include "muster.h"
#include "muster_ops.h"

using namespace muster;

namespace {
thread_local std::string g_err;

int op_fail(int code, const std::string& m) {
  g_err = m;
  return code;
}
int op_cuda(cudaError_t e, const char* what) {
  return op_fail(MUSTER_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define OK_(call)                                    \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return op_cuda(e_, #call); \
  } while (0)

bool dims_ok(int64_t D, int64_t H, int64_t W) {
  return D >= 1 && H >= 1 && W >= 1 && D <= 4096 && H <= 4096 && W <= 4096 && (double)D * H * W < 2147483647.0;
}
}  // namespace

namespace muster {
void set_ops_error(const std::string& m) { g_err = m; }
}  // namespace muster

extern "C" {

const char* muster_ops_last_error(void) { return g_err.c_str(); }

int muster_op_downsample(const float* in, int n_images, int64_t D, int64_t H, int64_t W, float* out, void* stream) {
  if (!in || !out || n_images < 1) return op_fail(MUSTER_EINVAL, "bad arguments");
  if (!dims_ok(D, H, W)) return op_fail(MUSTER_EINVAL, "bad shape");
  const Dims n{(int)D, (int)H, (int)W}, m{(int)(D + 1) / 2, (int)(H + 1) / 2, (int)(W + 1) / 2};
  launch_down2(in, n, out, m, n_images, (cudaStream_t)stream);
  OK_(cudaGetLastError());
  return MUSTER_OK;
}

int muster_op_exp(const float* phi, int64_t D, int64_t H, int64_t W, int K, float sign, float* u, void* stream) {
  if (!phi || !u) return op_fail(MUSTER_EINVAL, "NULL pointer");
  if (!dims_ok(D, H, W)) return op_fail(MUSTER_EINVAL, "bad shape");
  if (K < 0 || K > 20) return op_fail(MUSTER_EINVAL, "K must be 0..20");
  if (sign != 1.f && sign != -1.f) return op_fail(MUSTER_EINVAL, "sign must be +1 or -1");
  cudaStream_t s = (cudaStream_t)stream;
  const Dims n{(int)D, (int)H, (int)W};
  const size_t V = vox(n);
  float4* buf = nullptr;
  OK_(cudaMallocAsync((void**)&buf, sizeof(float4) * 5 * V, s));
  float4 *th = buf, *a = buf + V, *b = buf + 3 * V;
  launch_planar_to_f4(phi, th, 1, V, s);
  launch_exp_init(th, a, 1, n, ldexpf(1.f, -K), s);  // a[0] = +phi/2^K, a[1] = -phi/2^K
  for (int t = 0; t < K; ++t) {
    launch_squaring(a, b, 2, n, s);
    float4* tmp = a;
    a = b;
    b = tmp;
  }
  launch_f4_to_planar(a + (sign > 0.f ? 0 : V), u, 1, V, s);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(buf, s);
  if (e != cudaSuccess) return op_cuda(e, "exp launches");
  return MUSTER_OK;
}

int muster_op_similarity(const float* F, const float* W, int64_t D, int64_t H, int64_t Wd, int window, int kind,
                         float eps, double* loss, float* dLdW, void* stream) {
  if (!F || !W) return op_fail(MUSTER_EINVAL, "NULL image");
  if (!dims_ok(D, H, Wd)) return op_fail(MUSTER_EINVAL, "bad shape");
  if (window < 3 || window > 11 || window % 2 == 0) return op_fail(MUSTER_EINVAL, "window must be odd, 3..11");
  if (kind != MUSTER_SILNCC && kind != MUSTER_LNCC) return op_fail(MUSTER_EINVAL, "unknown similarity");
  if (!(eps >= 0.f)) return op_fail(MUSTER_EINVAL, "eps must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const Dims n{(int)D, (int)H, (int)Wd};
  const size_t V = vox(n);
  const int64_t NR = (D - window + 1) < 1 || (H - window + 1) < 1 || (Wd - window + 1) < 1
                         ? 0
                         : (D - window + 1) * (H - window + 1) * (Wd - window + 1);
  if (NR == 0) {
    if (dLdW) OK_(cudaMemsetAsync(dLdW, 0, sizeof(float) * V, s));
    if (loss) {
      OK_(cudaStreamSynchronize(s));
      *loss = 0.0;
    }
    return MUSTER_OK;
  }
  const int NC = sim_ncoef(kind);
  const SimGeom g = sim_geom(n, window, 1);
  // scratch: [out 8 doubles | step, flag ints | partials | descriptor | coefficients | F statistics]
  const size_t off_part = 64, off_desc = off_part + sizeof(double) * (size_t)g.ctas;
  const size_t off_coef = (off_desc + sizeof(PairDesc) + 255) / 256 * 256;
  const size_t off_stat = off_coef + sizeof(float) * NC * V;
  const size_t bytes = off_stat + sizeof(float) * 2 * V;
  char* buf = nullptr;
  OK_(cudaMallocAsync((void**)&buf, bytes, s));
  double* out = (double*)buf;
  int* ints = (int*)(buf + 48);
  double* part = (double*)(buf + off_part);
  PairDesc* pd = (PairDesc*)(buf + off_desc);
  float* coef = (float*)(buf + off_coef);
  float* stat = (float*)(buf + off_stat);
  PairDesc h{};
  h.Ii = F;
  h.Fs = stat;
  cudaError_t e = cudaMemsetAsync(buf, 0, 64, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pd, &h, sizeof(h), cudaMemcpyHostToDevice, s);
  SimMaps maps;
  make_sim_maps(&maps, W, 1, F, 1, coef, n, window, kind);
  if (e == cudaSuccess) e = prepare_kernels();
  if (e == cudaSuccess) {
    launch_fixed_stats(F, 1, n, window, kind, eps, stat, s);
    launch_sim_fwd(pd, 1, 1, W, V, coef, V, part, n, window, kind, eps, &maps, ints + 2, s);
    launch_loss_reduce(part, g.ctas, nullptr, 0, 1.0 / (double)NR, 0.0, 0.0, 0.f, 0.f, 0.f, out, nullptr, ints,
                       ints + 1, 0, s);
    if (dLdW) {
      const int nw = window * window * window;
      const float scale = kind == MUSTER_SILNCC ? (float)(2.0 / ((double)nw * (double)NR)) : (float)(1.0 / (double)NR);
      launch_sim_bwd(pd, 1, 1, W, V, coef, V, dLdW, n, window, kind, scale, &maps, ints + 2, s);
    }
    e = cudaGetLastError();
  }
  double host_out[2] = {0.0, 0.0};
  int host_err = 0;
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(host_out, out, sizeof(double) * 2, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(&host_err, ints + 2, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(buf, s);
  if (e != cudaSuccess) return op_cuda(e, "similarity launches");
  if (loss) {
    OK_(cudaStreamSynchronize(s));
    if (host_err) return op_fail(MUSTER_ETIMEOUT, "a bounded wait for an input copy ran out");
    *loss = host_out[1];
  }
  return MUSTER_OK;
}

int muster_op_jacobian_det(const float* u, int64_t D, int64_t H, int64_t Wd, float* J, void* stream) {
  if (!u || !J) return op_fail(MUSTER_EINVAL, "NULL field");
  if (!dims_ok(D, H, Wd)) return op_fail(MUSTER_EINVAL, "bad shape");
  launch_jacobian_det(u, Dims{(int)D, (int)H, (int)Wd}, J, (cudaStream_t)stream);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return op_cuda(e, "jacobian launch");
  return MUSTER_OK;
}

int muster_op_deformation_metrics(const float* u_true, const float* u_est, const uint8_t* roi, int64_t D, int64_t H,
                                  int64_t Wd, double out[16], void* stream) {
  if (!u_true || !u_est || !out) return op_fail(MUSTER_EINVAL, "NULL argument");
  if (!dims_ok(D, H, Wd)) return op_fail(MUSTER_EINVAL, "bad shape");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nd = metrics_scratch_doubles();
  double* buf = nullptr;
  OK_(cudaMallocAsync((void**)&buf, sizeof(double) * (nd + 16), s));
  launch_deformation_metrics(u_true, u_est, roi, Dims{(int)D, (int)H, (int)Wd}, buf, buf + nd, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, buf + nd, sizeof(double) * 16, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(buf, s);
  if (e != cudaSuccess) return op_cuda(e, "metrics launches");
  OK_(cudaStreamSynchronize(s));
  return MUSTER_OK;
}

}  // extern "C"
