// metrics_kernels.cu -- determinant maps of the spatial Jacobian of x -> x + u(x) (the maps
// of Sec. Sensitivity to clinical outcomes, Fig. 1c) and the deformation metrics of Sec.
// Evaluation Metrics: mean Euclidean distance Eu, vector Pearson correlation PCC of the
// centred fields and the slope B = trace(A)/3 of the least-squares fit u_est = A u_true + b.
//
// The determinant uses central differences, one-sided on the first and last plane of an
// axis and 0 along an axis of one plane. The metrics take two passes over the fields
// (means, then centred second moments) and a final single-CTA kernel that adds the partial
// sums in a fixed order and solves the 3x3 normal equations: the results are the same on
// every run. GB300 runs FP64 arithmetic far slower than FP32, so the per-voxel terms and each thread's
// running sums are double-float values (an unevaluated sum hi + lo of two floats, about 48
// significant bits) built from error-free transformations: Knuth's TwoSum for sums and the
// FMA form of Dekker's product (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005)
// for products. FP64 is used only for the per-CTA and final sums.
#include <algorithm>

#include "kernels.h"

namespace muster {

namespace {
constexpr int kJX = 32, kJY = 8;         // Jacobian: CTA tile (W x H) of one plane
// metrics: threads per CTA, and the most CTAs of the grid-stride passes (3 per SM of the
// device; kMCtas bounds the scratch of the per-CTA partial sums)
constexpr int kMT = 256, kMCtas = 3 * 256, kMCtasPerSM = 3;
constexpr int kP1 = 8, kP2 = 16;         // partial sums per CTA of pass 1 and pass 2

// one derivative from the values below (lo) and above (hi) index p of an axis of m planes:
// central inside, one-sided on the first and last plane, 0 on an axis of one plane
__device__ __forceinline__ float dstep(float lo, float mid, float hi, int p, int m) {
  if (m == 1) return 0.f;
  if (p == 0) return hi - mid;
  if (p == m - 1) return mid - lo;
  return 0.5f * (hi - lo);
}

// Streams along D: each thread owns one (y, x) column of a 32 x 8 tile and keeps the three
// components at planes z-1, z, z+1 in registers; plane z of the tile with a 1-voxel halo
// in W and H is staged in shared memory for the in-plane differences.
__global__ void __launch_bounds__(kJX* kJY) k_jacobian_det(const float* __restrict__ u, Dims n, float* __restrict__ J,
                                                           int zchunk) {
  __shared__ float tile[3][kJY + 2][kJX + 2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = blockIdx.x * kJX + tx, y = blockIdx.y * kJY + ty;
  const int z0 = blockIdx.z * zchunk, z1 = min(z0 + zchunk, n.n0);
  const size_t V = vox(n);
  const int plane = n.n1 * n.n2;
  const bool in = x < n.n2 && y < n.n1;
  const int xc = min(x, n.n2 - 1), yc = min(y, n.n1 - 1);
  const float* col = u + (size_t)yc * n.n2 + xc;
  // halo loaders: threads of the first/last column and row also fetch the neighbour cell
  const int hx = tx == 0 ? max(blockIdx.x * kJX - 1, 0) : (tx == kJX - 1 ? min(x + 1, n.n2 - 1) : -1);
  const int hy = ty == 0 ? max(blockIdx.y * kJY - 1, 0) : (ty == kJY - 1 ? min(y + 1, n.n1 - 1) : -1);
  float prv[3], cur[3], nxt[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* f = col + (size_t)c * V;
    cur[c] = __ldg(f + (size_t)z0 * plane);
    prv[c] = z0 > 0 ? __ldg(f + (size_t)(z0 - 1) * plane) : cur[c];
  }
  for (int z = z0; z < z1; ++z) {
#pragma unroll
    for (int c = 0; c < 3; ++c) nxt[c] = z + 1 < n.n0 ? __ldg(col + (size_t)c * V + (size_t)(z + 1) * plane) : cur[c];
    __syncthreads();  // the previous plane's reads of the tile are done
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float* f = u + (size_t)c * V + (size_t)z * plane;
      tile[c][ty + 1][tx + 1] = cur[c];
      if (hx >= 0) tile[c][ty + 1][tx == 0 ? 0 : kJX + 1] = __ldg(f + (size_t)yc * n.n2 + hx);
      if (hy >= 0) tile[c][ty == 0 ? 0 : kJY + 1][tx + 1] = __ldg(f + (size_t)hy * n.n2 + xc);
    }
    __syncthreads();
    if (in) {
      float M[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        M[c][0] = (c == 0 ? 1.f : 0.f) + dstep(prv[c], cur[c], nxt[c], z, n.n0);
        M[c][1] = (c == 1 ? 1.f : 0.f) + dstep(tile[c][ty][tx + 1], cur[c], tile[c][ty + 2][tx + 1], y, n.n1);
        M[c][2] = (c == 2 ? 1.f : 0.f) + dstep(tile[c][ty + 1][tx], cur[c], tile[c][ty + 1][tx + 2], x, n.n2);
      }
      J[(size_t)z * plane + (size_t)y * n.n2 + x] =
          M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
          M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      prv[c] = cur[c];
      cur[c] = nxt[c];
    }
  }
}

// ---- double-float arithmetic. The _rn intrinsics keep the compiler from fusing a product
// into a later addition, which would break the error-free transformations.
struct DF {
  float hi, lo;
};
// a + b = s + e exactly (Knuth)
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return DF{s, e};
}
// s + e with |e| <= ulp(s) / 2 (requires |a| >= |b| or a == 0)
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const DF s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float e = fmaf(x.hi, y.hi, -p);  // a b - p exactly
  return fast_two_sum(p, __fadd_rn(e, __fadd_rn(__fmul_rn(x.hi, y.lo), __fmul_rn(x.lo, y.hi))));
}
// a - (m_hi + m_lo) for a float a and a split double m
__device__ __forceinline__ DF df_sub_split(float a, float m_hi, float m_lo) {
  const DF s = two_sum(a, -m_hi);
  return fast_two_sum(s.hi, __fsub_rn(s.lo, m_lo));
}
// square root of x >= 0: r = sqrt(hi), then one Newton correction (x - r^2) / (2 r)
__device__ __forceinline__ DF df_sqrt(DF x) {
  if (!(x.hi > 0.f)) return DF{0.f, 0.f};
  const float r = sqrtf(x.hi);
  const float res = __fadd_rn(fmaf(-r, r, x.hi), x.lo);
  return fast_two_sum(r, res * (0.5f / r));
}
__device__ __forceinline__ double df_val(DF x) { return (double)x.hi + (double)x.lo; }

// fixed-order sum of one double over the CTA (result valid in thread 0)
__device__ __forceinline__ double cta_sum(double x, double* sh) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = x;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  return r;
}

// pass 1: count, sum |ut - ue|, sum ut, sum ue
__global__ void __launch_bounds__(kMT) k_metrics_pass1(const float* __restrict__ ut, const float* __restrict__ ue,
                                                       const unsigned char* __restrict__ roi, size_t V,
                                                       double* __restrict__ part) {
  __shared__ double sh[kMT / 32];
  int count = 0;
  DF acc[kP1 - 1];  // sum |d|, sum ut (3), sum ue (3)
#pragma unroll
  for (int k = 0; k < kP1 - 1; ++k) acc[k] = DF{0.f, 0.f};
  for (size_t v = (size_t)blockIdx.x * kMT + threadIdx.x; v < V; v += (size_t)gridDim.x * kMT) {
    if (roi && !roi[v]) continue;
    DF d2{0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float a = ut[(size_t)c * V + v], b = ue[(size_t)c * V + v];
      const DF d = two_sum(a, -b);  // a - b exactly
      d2 = df_add(d2, df_mul(d, d));
      acc[1 + c] = df_add(acc[1 + c], DF{a, 0.f});
      acc[4 + c] = df_add(acc[4 + c], DF{b, 0.f});
    }
    ++count;
    acc[0] = df_add(acc[0], df_sqrt(d2));
  }
  {
    const double s = cta_sum((double)count, sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * kP1] = s;
  }
#pragma unroll
  for (int k = 0; k < kP1 - 1; ++k) {
    const double s = cta_sum(df_val(acc[k]), sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * kP1 + 1 + k] = s;
  }
}

// means from the pass-1 partials: stats = {count, sum |d|, mt[3], me[3]} with means in place
__global__ void __launch_bounds__(kMT) k_metrics_means(const double* __restrict__ part, int nparts,
                                                       double* __restrict__ stats) {
  __shared__ double sh[kMT / 32];
  for (int k = 0; k < kP1; ++k) {
    double a = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kMT) a += part[(size_t)i * kP1 + k];
    const double s = cta_sum(a, sh);
    if (threadIdx.x == 0) stats[k] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0 && stats[0] > 0.0)
    for (int k = 2; k < kP1; ++k) stats[k] /= stats[0];
}

// pass 2: centred moments Ctt (6 unique), Cet (9), see
__global__ void __launch_bounds__(kMT) k_metrics_pass2(const float* __restrict__ ut, const float* __restrict__ ue,
                                                       const unsigned char* __restrict__ roi, size_t V,
                                                       const double* __restrict__ stats, double* __restrict__ part) {
  __shared__ double sh[kMT / 32];
  // the means as double-float pairs (hi = nearest float, lo = the float of the remainder)
  float mh[6], ml[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double m = stats[2 + k];
    mh[k] = (float)m;
    ml[k] = (float)(m - (double)mh[k]);
  }
  DF acc[kP2];
#pragma unroll
  for (int k = 0; k < kP2; ++k) acc[k] = DF{0.f, 0.f};
  for (size_t v = (size_t)blockIdx.x * kMT + threadIdx.x; v < V; v += (size_t)gridDim.x * kMT) {
    if (roi && !roi[v]) continue;
    DF a[3], b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a[c] = df_sub_split(ut[(size_t)c * V + v], mh[c], ml[c]);
      b[c] = df_sub_split(ue[(size_t)c * V + v], mh[3 + c], ml[3 + c]);
    }
    acc[0] = df_add(acc[0], df_mul(a[0], a[0]));
    acc[1] = df_add(acc[1], df_mul(a[0], a[1]));
    acc[2] = df_add(acc[2], df_mul(a[0], a[2]));
    acc[3] = df_add(acc[3], df_mul(a[1], a[1]));
    acc[4] = df_add(acc[4], df_mul(a[1], a[2]));
    acc[5] = df_add(acc[5], df_mul(a[2], a[2]));
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[6 + 3 * r + c] = df_add(acc[6 + 3 * r + c], df_mul(b[r], a[c]));
    acc[15] = df_add(acc[15], df_add(df_add(df_mul(b[0], b[0]), df_mul(b[1], b[1])), df_mul(b[2], b[2])));
  }
#pragma unroll
  for (int k = 0; k < kP2; ++k) {
    const double s = cta_sum(df_val(acc[k]), sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * kP2 + k] = s;
  }
}

// final: fixed-order sums of the pass-2 partials, then Eu, PCC, A = Cet Ctt^-1, b, B
__global__ void __launch_bounds__(kMT) k_metrics_final(const double* __restrict__ part, int nparts,
                                                       const double* __restrict__ stats, double* __restrict__ out) {
  __shared__ double sh[kMT / 32];
  __shared__ double S[kP2];
  for (int k = 0; k < kP2; ++k) {
    double a = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kMT) a += part[(size_t)i * kP2 + k];
    const double s = cta_sum(a, sh);
    if (threadIdx.x == 0) S[k] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int k = 0; k < 16; ++k) out[k] = 0.0;
  const double cnt = stats[0];
  out[15] = cnt;
  if (cnt == 0.0) return;
  const double C[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
  const double E[3][3] = {{S[6], S[7], S[8]}, {S[9], S[10], S[11]}, {S[12], S[13], S[14]}};
  const double stt = C[0][0] + C[1][1] + C[2][2], ste = E[0][0] + E[1][1] + E[2][2];
  out[0] = stats[1] / cnt;
  out[1] = ste / (sqrt(stt) * sqrt(S[15]));
  const double det = C[0][0] * (C[1][1] * C[2][2] - C[1][2] * C[2][1]) -
                     C[0][1] * (C[1][0] * C[2][2] - C[1][2] * C[2][0]) +
                     C[0][2] * (C[1][0] * C[2][1] - C[1][1] * C[2][0]);
  double inv[3][3];
  inv[0][0] = (C[1][1] * C[2][2] - C[1][2] * C[2][1]) / det;
  inv[0][1] = (C[0][2] * C[2][1] - C[0][1] * C[2][2]) / det;
  inv[0][2] = (C[0][1] * C[1][2] - C[0][2] * C[1][1]) / det;
  inv[1][0] = (C[1][2] * C[2][0] - C[1][0] * C[2][2]) / det;
  inv[1][1] = (C[0][0] * C[2][2] - C[0][2] * C[2][0]) / det;
  inv[1][2] = (C[0][2] * C[1][0] - C[0][0] * C[1][2]) / det;
  inv[2][0] = (C[1][0] * C[2][1] - C[1][1] * C[2][0]) / det;
  inv[2][1] = (C[0][1] * C[2][0] - C[0][0] * C[2][1]) / det;
  inv[2][2] = (C[0][0] * C[1][1] - C[0][1] * C[1][0]) / det;
  double tr = 0.0;
  for (int r = 0; r < 3; ++r) {
    double Ar[3];
    for (int c = 0; c < 3; ++c) Ar[c] = E[r][0] * inv[0][c] + E[r][1] * inv[1][c] + E[r][2] * inv[2][c];
    for (int c = 0; c < 3; ++c) out[3 + 3 * r + c] = Ar[c];
    out[12 + r] = stats[5 + r] - (Ar[0] * stats[2] + Ar[1] * stats[3] + Ar[2] * stats[4]);
    tr += Ar[r];
  }
  out[2] = tr / 3.0;
}
}  // namespace

void launch_jacobian_det(const float* u, Dims n, float* J, cudaStream_t s) {
  // D chunks so that the grid has at least 8 CTAs per SM of the device
  const int gx = (n.n2 + kJX - 1) / kJX, gy = (n.n1 + kJY - 1) / kJY;
  const long want = 8L * device_sm_count();
  int zc = n.n0;
  while (zc > 4 && (long)gx * gy * ((n.n0 + zc - 1) / zc) < want) zc = (zc + 1) / 2;
  k_jacobian_det<<<dim3(gx, gy, (n.n0 + zc - 1) / zc), dim3(kJX, kJY), 0, s>>>(u, n, J, zc);
}

size_t metrics_scratch_doubles() { return (size_t)kMCtas * (kP1 + kP2) + kP1; }

void launch_deformation_metrics(const float* ut, const float* ue, const unsigned char* roi, Dims n, double* scratch,
                                double* out, cudaStream_t s) {
  const size_t V = vox(n);
  const size_t per_device = (size_t)std::min(kMCtas, kMCtasPerSM * device_sm_count());
  const int ctas = (int)std::max<size_t>(1, std::min<size_t>(per_device, (V + kMT - 1) / kMT));
  double* p1 = scratch;
  double* p2 = scratch + (size_t)kMCtas * kP1;
  double* stats = p2 + (size_t)kMCtas * kP2;
  k_metrics_pass1<<<ctas, kMT, 0, s>>>(ut, ue, roi, V, p1);
  k_metrics_means<<<1, kMT, 0, s>>>(p1, ctas, stats);
  k_metrics_pass2<<<ctas, kMT, 0, s>>>(ut, ue, roi, V, stats, p2);
  k_metrics_final<<<1, kMT, 0, s>>>(p2, ctas, stats, out);
}

}  // namespace muster
