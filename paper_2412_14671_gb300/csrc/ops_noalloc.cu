// ops_noalloc.cu -- muster_op_similarity_noalloc: the windowed similarity of
// muster_op_similarity for callers that cannot allocate device memory (for
// example code running where cudaMalloc is forbidden or unavailable, such as a
// real-time pipeline with a frozen memory budget, or a host library that may
// only use memory it was handed). Its scratch is one fixed, file-scope device
// array that every GPU loading this library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels.h"
#include "muster.h"
#include "muster_ops.h"

using namespace muster;

namespace muster {
void set_ops_error(const std::string& m);  // ops.cu
}

namespace {

// layout of the scratch: [8 doubles of results | ints | CTA partial sums | descriptor | coefficients |
// window statistics of F]
constexpr size_t kMaxCtas = (size_t)1 << 17;                           // partial sums of the forward kernel
constexpr size_t kHead = (64 + 8 * kMaxCtas + 64 + 255) / 256 * 256;  // results, counters, partials, descriptor
constexpr size_t kCoefBytes = (size_t)3 * 4 * MUSTER_NOALLOC_MAX_VOXELS;  // up to 3 coefficient volumes
constexpr size_t kStatBytes = (size_t)2 * 4 * MUSTER_NOALLOC_MAX_VOXELS;  // mu_F and S_FF volumes
constexpr size_t kScratchBytes = kHead + kCoefBytes + kStatBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

int na_fail(int code, const std::string& m) {
  set_ops_error(m);  // reported by muster_ops_last_error()
  return code;
}

// Device address of the scratch on the current device. In host code the name
// g_noalloc_scratch is only a host-side stand-in, so the address is looked up
// once per device, with that device current, and cached.
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(MUSTER_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(MUSTER_ECUDA, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(MUSTER_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return MUSTER_OK;
}

}  // namespace

extern "C" {

int muster_op_similarity_noalloc(const float* F, const float* W, int64_t D, int64_t H, int64_t Wd, int window,
                                 int kind, float eps, double* loss, float* dLdW, void* stream) {
  if (!F || !W) return na_fail(MUSTER_EINVAL, "NULL image");
  if (D < 1 || H < 1 || Wd < 1) return na_fail(MUSTER_EINVAL, "bad shape");
  if ((double)D * (double)H * (double)Wd > (double)MUSTER_NOALLOC_MAX_VOXELS)
    return na_fail(MUSTER_EINVAL, "volume exceeds MUSTER_NOALLOC_MAX_VOXELS (" +
                                      std::to_string((long long)MUSTER_NOALLOC_MAX_VOXELS) +
                                      " voxels); use muster_op_similarity");
  if (window < 3 || window > 11 || window % 2 == 0) return na_fail(MUSTER_EINVAL, "window must be odd, 3..11");
  if (kind != MUSTER_SILNCC && kind != MUSTER_LNCC) return na_fail(MUSTER_EINVAL, "unknown similarity");
  if (!(eps >= 0.f)) return na_fail(MUSTER_EINVAL, "eps must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const Dims n{(int)D, (int)H, (int)Wd};
  const size_t V = vox(n);
  const int64_t NR = (D - window + 1) < 1 || (H - window + 1) < 1 || (Wd - window + 1) < 1
                         ? 0
                         : (D - window + 1) * (H - window + 1) * (Wd - window + 1);
  cudaError_t e;
  if (NR == 0) {
    if (dLdW && (e = cudaMemsetAsync(dLdW, 0, sizeof(float) * V, s)) != cudaSuccess)
      return na_fail(MUSTER_ECUDA, cudaGetErrorString(e));
    if (loss) {
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return na_fail(MUSTER_ECUDA, cudaGetErrorString(e));
      *loss = 0.0;
    }
    return MUSTER_OK;
  }
  const SimGeom g = sim_geom(n, window, 1);
  const size_t off_part = 64, off_desc = off_part + sizeof(double) * (size_t)g.ctas;
  if ((size_t)g.ctas > kMaxCtas || off_desc + sizeof(PairDesc) > kHead)
    return na_fail(MUSTER_EINVAL, "volume shape needs more partial sums than the fixed scratch holds");
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  char* buf = (char*)base;
  double* out = (double*)buf;
  int* ints = (int*)(buf + 48);
  double* part = (double*)(buf + off_part);
  PairDesc* pd = (PairDesc*)(buf + off_desc);
  float* coef = (float*)(buf + kHead);
  float* stat = (float*)(buf + kHead + kCoefBytes);
  PairDesc h{};
  h.Ii = F;
  h.Fs = stat;
  // results and counters must start at zero: the array keeps the previous call's contents
  e = cudaMemsetAsync(buf, 0, 64, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pd, &h, sizeof(h), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return na_fail(MUSTER_ECUDA, cudaGetErrorString(e));
  SimMaps maps;
  make_sim_maps(&maps, W, 1, F, 1, coef, n, window, kind);
  if ((e = prepare_kernels()) != cudaSuccess) return na_fail(MUSTER_ECUDA, cudaGetErrorString(e));
  launch_fixed_stats(F, 1, n, window, kind, eps, stat, s);
  launch_sim_fwd(pd, 1, 1, W, V, coef, V, part, n, window, kind, eps, &maps, ints + 2, s);
  launch_loss_reduce(part, g.ctas, nullptr, 0, 1.0 / (double)NR, 0.0, 0.0, 0.f, 0.f, 0.f, out, nullptr, ints,
                     ints + 1, 0, s);
  if (dLdW) {
    const int nw = window * window * window;
    const float scale = kind == MUSTER_SILNCC ? (float)(2.0 / ((double)nw * (double)NR)) : (float)(1.0 / (double)NR);
    launch_sim_bwd(pd, 1, 1, W, V, coef, V, dLdW, n, window, kind, scale, &maps, ints + 2, s);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(MUSTER_ECUDA, cudaGetErrorString(e));
  if (loss) {
    double host_out[2] = {0.0, 0.0};
    int host_err = 0;
    if ((e = cudaMemcpyAsync(host_out, out, sizeof(double) * 2, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&host_err, ints + 2, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return na_fail(MUSTER_ECUDA, cudaGetErrorString(e));
    if (host_err) return na_fail(MUSTER_ETIMEOUT, "a bounded wait for an input copy ran out");
    *loss = host_out[1];
  }
  return MUSTER_OK;
}

}  // extern "C"
