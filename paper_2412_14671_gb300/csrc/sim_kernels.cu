// sim_kernels.cu -- the windowed similarity of Eq. LNCC / the SiLNCC equation,
// averaged over the valid windows (Eq. sum_lncc, Eq. sim_loss), and its adjoint.
//
// Window R has lower corner c (centre c + R); the valid corners are
// 0 <= c_a <= n_a - w. Both kernels stream along D: a CTA of 256 threads owns a
// 32 (W) x 16 (H) tile of windows (forward) or voxels (adjoint) and a chunk of D.
// Per plane the (32 + 2R) x (16 + 2R) halo region of the inputs is staged in
// shared memory, summed along W by running sums over float4 runs, along H by
// running sums (two rows per thread), and along D through a shared-memory ring of
// the last 2R+1 plane sums with a running total that is re-summed exactly every
// 2R+1 planes. When the width is a multiple of 4 the halo planes are copied by
// the tensor memory accelerator (two stages, mbarrier completion, zero fill
// outside the volume); otherwise each thread loads its share of the plane.
//
// The fixed image's window statistics (mu_F, S_FF) depend on the session only and
// are computed once per level (k_fixed_stats); the forward per pair then needs
// the box sums of W', W'^2 and F'W' only.
// Forward: for every corner of the image grid it writes the coefficients of
//   dSim_R/dW(p) = A_R W(p) - B_R F(p) - C_R   (zero for invalid corners)
//   SiLNCC: A = 1 (implicit; 2/|R| is applied by the adjoint), B = beta = S_FW/(S_FF+eps),
//           C = mu_W - beta mu_F;
//   LNCC:   A = S_FW S_FF / Q^{3/2}, B = 1/sqrt(Q), C = A mu_W - B mu_F, Q = S_FF S_WW + eps,
// and adds Sim_R to a per-CTA partial sum. Sums are taken on values shifted by
// one voxel of the tile (variance is shift invariant) to limit cancellation.
// Adjoint: dL/dW(p) = scale * (W(p) sum A - F(p) sum B - sum C) over the
// windows containing p (corners p - 2R .. p).
#include <cudaTypedefs.h>
#include <string.h>

#include <mutex>

#include "kernels.h"
#include "tma.cuh"

namespace muster {

namespace {
constexpr int kThreads = 256, TX = 32;

// The CTA's sum of the per-thread compensated sums (hi + lo), valid in thread 0: float-float
// sums within each warp, then the warp sums in double.
__device__ __forceinline__ double block_sum(FF x, float* sh) {
  x = warp_sum_ff(x);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    sh[2 * w] = x.hi;
    sh[2 * w + 1] = x.lo;
  }
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += (double)sh[2 * i] + (double)sh[2 * i + 1];
  return r;
}

// Statistics of the fixed image of every window, once per session and level:
// out[0][c] = mu_F and out[1][c] = S_FF (centred sum of squares) at corner c, or for SiLNCC
// (KIND 0, which needs S_FF only in beta = S_FW / (S_FF + eps)) out[1][c] = 1 / (S_FF + eps).
template <int R, int KIND>
__global__ void __launch_bounds__(kThreads) k_fixed_stats(const float* __restrict__ imgs, float* __restrict__ stats,
                                                          Dims n, int tz, int nzc, float eps) {
  constexpr int WW = 2 * R + 1, TY = 8, RX = TX + 2 * R, RY = TY + 2 * R;
  constexpr int NE = RY * RX, NSLOT = (NE + kThreads - 1) / kThreads;
  __shared__ float sF[NE];
  __shared__ float sx[2][RY][TX];
  const int img = blockIdx.z / nzc, zc = blockIdx.z - img * nzc;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = zc * tz;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int plane = n.n1 * n.n2;
  const size_t V = (size_t)plane * n.n0;
  const float* __restrict__ F = imgs + (size_t)img * V;
  float* __restrict__ out = stats + (size_t)img * 2 * V;
  int soff[NSLOT];
  bool sok[NSLOT];
#pragma unroll
  for (int k = 0; k < NSLOT; ++k) {
    const int e = tid + kThreads * k;
    const int ry = e / RX, rx = e - ry * RX;
    const int gy = y0 + ry, gx = x0 + rx;
    sok[k] = e < NE && gy < n.n1 && gx < n.n2;
    soff[k] = gy * n.n2 + gx;
  }
  const float shF = F[min(z0 + R, n.n0 - 1) * plane + min(y0 + R, n.n1 - 1) * n.n2 + min(x0 + R, n.n2 - 1)];
  const float inv_nw = 1.f / (float)(WW * WW * WW);
  float ring[2][WW] = {}, S[2] = {0.f, 0.f};
  const int zend = min(z0 + tz, n.n0);
  const int niter = (zend - z0) + 2 * R;
  for (int base = 0; base < niter; base += WW) {
#pragma unroll
    for (int j = 0; j < WW; ++j) {
      const int it = base + j;
      if (it >= niter) break;
      const int zin = z0 + it;
#pragma unroll
      for (int k = 0; k < NSLOT; ++k) {
        const int e = tid + kThreads * k;
        if (e < NE) sF[e] = (zin < n.n0 && sok[k]) ? F[zin * plane + soff[k]] - shF : 0.f;
      }
      __syncthreads();
      for (int ry = ty; ry < RY; ry += kThreads / 32) {
        float a0 = 0.f, a1 = 0.f;
        const float* pf = sF + ry * RX + tx;
#pragma unroll
        for (int k = 0; k < WW; ++k) {
          a0 += pf[k];
          a1 = fmaf(pf[k], pf[k], a1);
        }
        sx[0][ry][tx] = a0;
        sx[1][ry][tx] = a1;
      }
      __syncthreads();
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < WW; ++k) v += sx[m][ty + k][tx];
        S[m] += v - ring[m][j];
        ring[m][j] = v;
        if (j == WW - 1) {
          float t = 0.f;
#pragma unroll
          for (int k = 0; k < WW; ++k) t += ring[m][k];
          S[m] = t;
        }
      }
      if (it >= 2 * R) {
        const int cz = zin - 2 * R, cy = y0 + ty, cx = x0 + tx;
        if (cx < n.n2 && cy < n.n1) {
          const int o = cz * plane + cy * n.n2 + cx;
          out[o] = S[0] * inv_nw + shF;
          const float sff = fmaxf(S[1] - S[0] * S[0] * inv_nw, 0.f);
          out[V + o] = KIND == 0 ? 1.f / (sff + eps) : sff;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Streaming box sums, version with running sums in all three directions.
// CTA tile: 32 (W) x 16 (H) windows (forward) or voxels (adjoint), 256 threads
// (16 output rows against 2R halo rows keep the W pass's share of halo work small).
//  - W pass: 8 tasks per halo row, each 4 consecutive outputs from one float4
//    run of 4 + 2R inputs (running sum along W);
//  - H pass: one thread per column and pair of rows (running sum);
//  - D pass: a ring of the last 2R+1 plane sums in shared memory, one owner
//    thread per output, running sum re-summed exactly every 2R+1 planes.
constexpr int T3X = 32, T3Y = 16, YO = 2, NT3 = T3X * T3Y / YO;  // 256 threads
static_assert(YO == 2, "the D ring of the TMA-staged kernels keeps a thread's two rows as a float2");
// a tensor copy must start on a 16-byte boundary: the forward's box starts at x0 = 32 * blockIdx.x
static_assert(T3X % 4 == 0, "the staged forward box must start at a multiple of 4 floats");

template <int R, int NM>
struct Geo3 {
  static constexpr int WW = 2 * R + 1;
  static constexpr int RX = T3X + 2 * R, RY = T3Y + 2 * R;
  static constexpr int NV = (4 + 2 * R + 3) / 4;  // float4 per W-pass run
  static constexpr int RXS = ((RX + 3) / 4) * 4 > 28 + 4 * NV ? ((RX + 3) / 4) * 4 : 28 + 4 * NV;
  static constexpr int NE = RY * RX, NSLOT = (NE + NT3 - 1) / NT3;
  // shared memory (floats): inputs [NIN][RY][RXS], W sums [NM][RY][T3X], ring [WW][NM][T3Y][T3X]
  __host__ __device__ static constexpr size_t in_floats(int nin) { return (size_t)nin * RY * RXS; }
  __host__ __device__ static constexpr size_t sx_floats() { return (size_t)NM * RY * T3X; }
  __host__ __device__ static constexpr size_t ring_floats() { return (size_t)WW * NM * T3Y * T3X; }
};

// pairwise sum of v[0..N-1]: a dependency chain of depth log2(N) instead of N - 1
template <int N>
struct TreeSum {
  __device__ __forceinline__ static float of(const float* v) {
    return TreeSum<N / 2>::of(v) + TreeSum<N - N / 2>::of(v + N / 2);
  }
};
template <>
struct TreeSum<1> {
  __device__ __forceinline__ static float of(const float* v) { return v[0]; }
};

// running box sum of one run: out[i] = sum_{k<WW} v[i + k], i < NO
template <int WW, int NO>
__device__ __forceinline__ void runsum(const float* v, float* out) {
  float s = TreeSum<WW>::of(v);
  out[0] = s;
#pragma unroll
  for (int i = 1; i < NO; ++i) {
    s += v[i + WW - 1] - v[i - 1];
    out[i] = s;
  }
}

template <int R, int KIND>
__global__ void __launch_bounds__(NT3) k_sim_fwd3(const PairDesc* __restrict__ pd, const float* __restrict__ Wb,
                                                       size_t Wstride, float* __restrict__ coef, size_t cstride,
                                                       double* __restrict__ part, Dims n, float eps, int tz, int nzc) {
  using G = Geo3<R, 3>;
  constexpr int WW = G::WW, RX = G::RX, RY = G::RY, RXS = G::RXS, NV = G::NV, NE = G::NE, NSLOT = G::NSLOT;
  constexpr int NC = KIND == 0 ? 2 : 3;
  extern __shared__ __align__(16) float smem[];
  float* sF = smem;
  float* sW = sF + RY * RXS;
  float* sx = sW + RY * RXS;                 // [3][RY][T3X]
  float* ring = sx + G::sx_floats();         // [WW][3][T3Y][T3X]
  __shared__ float sh[2 * (NT3 / 32)];
  const int pair = blockIdx.z / nzc, zc = blockIdx.z - pair * nzc;
  const int x0 = blockIdx.x * T3X, y0 = blockIdx.y * T3Y, z0 = zc * tz;
  const int tid = threadIdx.x;
  const PairDesc d = pd[pair];
  const float* __restrict__ F = d.Ii;
  const float* __restrict__ Fs = d.Fs;
  const float* __restrict__ W = Wb + (size_t)pair * Wstride;
  float* __restrict__ C = coef + (size_t)pair * NC * cstride;
  const int plane = n.n1 * n.n2;
  int soff[NSLOT], sidx[NSLOT];
  bool sok[NSLOT];
#pragma unroll
  for (int k = 0; k < NSLOT; ++k) {
    const int e = tid + NT3 * k;
    const int ry = e / RX, rx = e - ry * RX;
    const int gy = y0 + ry, gx = x0 + rx;
    sok[k] = e < NE && gy < n.n1 && gx < n.n2;
    soff[k] = gy * n.n2 + gx;
    sidx[k] = e < NE ? ry * RXS + rx : -1;
  }
  const int so = min(z0 + R, n.n0 - 1) * plane + min(y0 + R, n.n1 - 1) * n.n2 + min(x0 + R, n.n2 - 1);
  const float shF = F[so], shW = W[so];
  const float inv_nw = 1.f / (float)(WW * WW * WW);
  const int mx = n.n2 - WW, my = n.n1 - WW, mz = n.n0 - WW;
  // roles: W pass (8 tasks per halo row), H/D pass and outputs (thread = column, YO rows)
  const int col = tid & 31, yseg = tid >> 5;
  float S[YO][3];
#pragma unroll
  for (int i = 0; i < YO; ++i)
#pragma unroll
    for (int m = 0; m < 3; ++m) S[i][m] = 0.f;
  for (int j = 0; j < WW; ++j)
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int i = 0; i < YO; ++i) ring[((j * 3 + m) * T3Y + YO * yseg + i) * T3X + col] = 0.f;
  float lsum = 0.f, lcomp = 0.f;
  const int zend = min(z0 + tz, n.n0);
  const int niter = (zend - z0) + 2 * R;
  float pf[NSLOT], pw[NSLOT];
  auto fetch = [&](int zin) {
    const bool zok = zin < n.n0;
    const int zo = zin * plane;
#pragma unroll
    for (int k = 0; k < NSLOT; ++k) {
      pf[k] = 0.f;
      pw[k] = 0.f;
      if (zok && sok[k]) {
        pf[k] = F[zo + soff[k]] - shF;
        pw[k] = W[zo + soff[k]] - shW;
      }
    }
  };
  // mu_F and S_FF of this thread's windows in the next output plane (loaded one plane ahead)
  float pmu[YO], psf[YO];
  const bool xin = x0 + col <= mx;
  auto fetch_stats = [&](int cz) {
#pragma unroll
    for (int i = 0; i < YO; ++i) {
      const int cy = y0 + YO * yseg + i;
      pmu[i] = 0.f;
      psf[i] = 0.f;
      if (xin && cy <= my && cz <= mz) {
        const int o = cz * plane + cy * n.n2 + x0 + col;
        pmu[i] = Fs[o];
        psf[i] = Fs[(size_t)plane * n.n0 + o];
      }
    }
  };
  fetch(z0);
  int j = 0;  // ring slot of this plane
  for (int it = 0; it < niter; ++it) {
    const int zin = z0 + it;
#pragma unroll
    for (int k = 0; k < NSLOT; ++k)
      if (sidx[k] >= 0) {
        sF[sidx[k]] = pf[k];
        sW[sidx[k]] = pw[k];
      }
    float muF_c[YO], Sff_c[YO];
#pragma unroll
    for (int i = 0; i < YO; ++i) muF_c[i] = pmu[i], Sff_c[i] = psf[i];
    __syncthreads();
    if (it + 1 < niter) {
      fetch(zin + 1);
      if (it + 1 >= 2 * R) fetch_stats(zin + 1 - 2 * R);
    }
    for (int task = tid; task < 8 * RY; task += NT3) {
      const int xrow = task >> 3, xseg = task & 7;
      float f[4 * NV], w[4 * NV];
      const float4* pF = reinterpret_cast<const float4*>(sF + xrow * RXS + 4 * xseg);
      const float4* pW = reinterpret_cast<const float4*>(sW + xrow * RXS + 4 * xseg);
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const float4 a = pF[q], b = pW[q];
        f[4 * q] = a.x, f[4 * q + 1] = a.y, f[4 * q + 2] = a.z, f[4 * q + 3] = a.w;
        w[4 * q] = b.x, w[4 * q + 1] = b.y, w[4 * q + 2] = b.z, w[4 * q + 3] = b.w;
      }
      float ww[4 + 2 * R], fw[4 + 2 * R];
#pragma unroll
      for (int k = 0; k < 4 + 2 * R; ++k) {
        ww[k] = w[k] * w[k];
        fw[k] = f[k] * w[k];
      }
      float o0[4], o1[4], o2[4];
      runsum<WW, 4>(w, o0);
      runsum<WW, 4>(ww, o1);
      runsum<WW, 4>(fw, o2);
      float4* dst = reinterpret_cast<float4*>(sx + xrow * T3X + 4 * xseg);
      dst[0] = make_float4(o0[0], o0[1], o0[2], o0[3]);
      dst[RY * T3X / 4] = make_float4(o1[0], o1[1], o1[2], o1[3]);
      dst[2 * RY * T3X / 4] = make_float4(o2[0], o2[1], o2[2], o2[3]);
    }
    __syncthreads();
    {
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        float v[YO + 2 * R], a[YO];
#pragma unroll
        for (int k = 0; k < YO + 2 * R; ++k) v[k] = sx[(m * RY + YO * yseg + k) * T3X + col];
        runsum<WW, YO>(v, a);
#pragma unroll
        for (int i = 0; i < YO; ++i) {
          float* rp = ring + ((j * 3 + m) * T3Y + YO * yseg + i) * T3X + col;
          S[i][m] += a[i] - *rp;
          *rp = a[i];
        }
      }
      if (j == WW - 1) {  // exact re-sum bounds the drift of the running sums
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
          for (int i = 0; i < YO; ++i) {
            float t = 0.f;
            for (int q = 0; q < WW; ++q) t += ring[((q * 3 + m) * T3Y + YO * yseg + i) * T3X + col];
            S[i][m] = t;
          }
      }
      if (it >= 2 * R) {
        const int cz = zin - 2 * R, cx = x0 + col;
#pragma unroll
        for (int i = 0; i < YO; ++i) {
          const int cy = y0 + YO * yseg + i;
          if (cx >= n.n2 || cy >= n.n1) continue;
          const int o = cz * plane + cy * n.n2 + cx;
          float c0 = 0.f, c1 = 0.f, c2 = 0.f;
          if (cx <= mx && cy <= my && cz <= mz) {
            const float muF = muF_c[i], Sff = Sff_c[i];
            const float Sww = fmaxf(S[i][1] - S[i][0] * S[i][0] * inv_nw, 0.f);
            const float Sfw = S[i][2] - (muF - shF) * S[i][0];
            const float muW = S[i][0] * inv_nw + shW;
            float val;
            if (KIND == 0) {
              const float beta = Sfw * Sff;  // Sff holds 1 / (S_FF + eps) for SiLNCC
              val = (Sww - Sfw * beta) * inv_nw;
              c0 = beta;
              c1 = muW - beta * muF;
            } else {
              const float Q = Sff * Sww + eps;
              const float rq = 1.f / sqrtf(Q);
              val = 1.f - Sfw * rq;
              c0 = Sfw * Sff * rq * rq * rq;
              c1 = rq;
              c2 = c0 * muW - c1 * muF;
            }
            const float yk = val - lcomp;
            const float tk = lsum + yk;
            lcomp = (tk - lsum) - yk;
            lsum = tk;
          }
          C[o] = c0;
          C[cstride + o] = c1;
          if (KIND == 1) C[2 * cstride + o] = c2;
        }
      }
    }
    j = (j + 1 == WW) ? 0 : j + 1;
  }
  const double sum = block_sum(FF{lsum, -lcomp}, sh);
  if (threadIdx.x == 0) part[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = sum;
}

template <int R, int KIND>
__global__ void __launch_bounds__(NT3) k_sim_bwd3(const PairDesc* __restrict__ pd, const float* __restrict__ Wb,
                                                       size_t Wstride, const float* __restrict__ coef, size_t cstride,
                                                       float* __restrict__ dLdW, Dims n, float scale, int tz, int nzc) {
  constexpr int NC = KIND == 0 ? 2 : 3;
  using G = Geo3<R, NC>;
  constexpr int WW = G::WW, RX = G::RX, RY = G::RY, RXS = G::RXS, NV = G::NV, NE = G::NE, NSLOT = G::NSLOT;
  extern __shared__ __align__(16) float smem[];
  float* sc = smem;                            // [NC][RY][RXS]
  float* sx = sc + G::in_floats(NC);           // [NC][RY][T3X]
  float* ring = sx + G::sx_floats();           // [WW][NC][T3Y][T3X]
  const int pair = blockIdx.z / nzc, zc = blockIdx.z - pair * nzc;
  const int x0 = blockIdx.x * T3X, y0 = blockIdx.y * T3Y, z0 = zc * tz;
  const int tid = threadIdx.x;
  const float* __restrict__ F = pd[pair].Ii;
  const float* __restrict__ W = Wb + (size_t)pair * Wstride;
  const float* __restrict__ Cf = coef + (size_t)pair * NC * cstride;
  float* __restrict__ out = dLdW + (size_t)pair * Wstride;
  const int plane = n.n1 * n.n2;
  int soff[NSLOT], sidx[NSLOT];
  bool sok[NSLOT];
#pragma unroll
  for (int k = 0; k < NSLOT; ++k) {
    const int e = tid + NT3 * k;
    const int ry = e / RX, rx = e - ry * RX;
    const int gy = y0 - 2 * R + ry, gx = x0 - 2 * R + rx;
    sok[k] = e < NE && gy >= 0 && gy < n.n1 && gx >= 0 && gx < n.n2;
    soff[k] = gy * n.n2 + gx;
    sidx[k] = e < NE ? ry * RXS + rx : -1;
  }
  const int mx = n.n2 - WW, my = n.n1 - WW, mz = n.n0 - WW;
  const int col = tid & 31, yseg = tid >> 5;
  const int px = x0 + col;
  float cnt_xy[YO];
#pragma unroll
  for (int i = 0; i < YO; ++i) {
    const int py = y0 + YO * yseg + i;
    const int cxn = max(0, min(px, mx) - max(0, px - 2 * R) + 1);
    const int cyn = max(0, min(py, my) - max(0, py - 2 * R) + 1);
    cnt_xy[i] = (float)(cxn * cyn);
  }
  float S[YO][NC];
#pragma unroll
  for (int i = 0; i < YO; ++i)
#pragma unroll
    for (int m = 0; m < NC; ++m) S[i][m] = 0.f;
  for (int j = 0; j < WW; ++j)
#pragma unroll
    for (int m = 0; m < NC; ++m)
#pragma unroll
      for (int i = 0; i < YO; ++i) ring[((j * NC + m) * T3Y + YO * yseg + i) * T3X + col] = 0.f;
  const int zend = min(z0 + tz, n.n0);
  const int niter = (zend - z0) + 2 * R;
  float pc[NC][NSLOT];
  auto fetch = [&](int zin) {
    const bool zok = zin >= 0 && zin < n.n0;
    const int zo = zin * plane;
#pragma unroll
    for (int k = 0; k < NSLOT; ++k) {
      const bool ok = zok && sok[k];
#pragma unroll
      for (int m = 0; m < NC; ++m) pc[m][k] = ok ? Cf[(size_t)m * cstride + zo + soff[k]] : 0.f;
    }
  };
  // W and F at this thread's voxels of the next output plane (loaded one plane ahead)
  float pwv[YO], pfv[YO];
  const bool xin = px < n.n2;
  auto fetch_wf = [&](int pz) {
#pragma unroll
    for (int i = 0; i < YO; ++i) {
      const int py = y0 + YO * yseg + i;
      pwv[i] = 0.f;
      pfv[i] = 0.f;
      if (xin && py < n.n1) {
        const int o = pz * plane + py * n.n2 + px;
        pwv[i] = W[o];
        pfv[i] = F[o];
      }
    }
  };
  fetch(z0 - 2 * R);
  int j = 0;
  for (int it = 0; it < niter; ++it) {
    const int zin = z0 - 2 * R + it;  // corner plane
#pragma unroll
    for (int k = 0; k < NSLOT; ++k)
      if (sidx[k] >= 0) {
#pragma unroll
        for (int m = 0; m < NC; ++m) sc[m * RY * RXS + sidx[k]] = pc[m][k];
      }
    float wv_c[YO], fv_c[YO];
#pragma unroll
    for (int i = 0; i < YO; ++i) wv_c[i] = pwv[i], fv_c[i] = pfv[i];
    __syncthreads();
    if (it + 1 < niter) {
      fetch(zin + 1);
      if (it + 1 >= 2 * R) fetch_wf(zin + 1);
    }
    for (int task = tid; task < 8 * RY; task += NT3) {
      const int xrow = task >> 3, xseg = task & 7;
#pragma unroll
      for (int m = 0; m < NC; ++m) {
        float v[4 * NV];
        const float4* src = reinterpret_cast<const float4*>(sc + (m * RY + xrow) * RXS + 4 * xseg);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const float4 a = src[q];
          v[4 * q] = a.x, v[4 * q + 1] = a.y, v[4 * q + 2] = a.z, v[4 * q + 3] = a.w;
        }
        float o[4];
        runsum<WW, 4>(v, o);
        *reinterpret_cast<float4*>(sx + (m * RY + xrow) * T3X + 4 * xseg) = make_float4(o[0], o[1], o[2], o[3]);
      }
    }
    __syncthreads();
    {
#pragma unroll
      for (int m = 0; m < NC; ++m) {
        float v[YO + 2 * R], a[YO];
#pragma unroll
        for (int k = 0; k < YO + 2 * R; ++k) v[k] = sx[(m * RY + YO * yseg + k) * T3X + col];
        runsum<WW, YO>(v, a);
#pragma unroll
        for (int i = 0; i < YO; ++i) {
          float* rp = ring + ((j * NC + m) * T3Y + YO * yseg + i) * T3X + col;
          S[i][m] += a[i] - *rp;
          *rp = a[i];
        }
      }
      if (j == WW - 1) {
#pragma unroll
        for (int m = 0; m < NC; ++m)
#pragma unroll
          for (int i = 0; i < YO; ++i) {
            float t[WW];
#pragma unroll
            for (int q = 0; q < WW; ++q) t[q] = ring[((q * NC + m) * T3Y + YO * yseg + i) * T3X + col];
            S[i][m] = TreeSum<WW>::of(t);
          }
      }
      if (it >= 2 * R) {
        const int pz = zin;
        const int czn = max(0, min(pz, mz) - max(0, pz - 2 * R) + 1);
#pragma unroll
        for (int i = 0; i < YO; ++i) {
          const int py = y0 + YO * yseg + i;
          if (px >= n.n2 || py >= n.n1) continue;
          const int o = pz * plane + py * n.n2 + px;
          const float wv = wv_c[i], fv = fv_c[i];
          float g;
          if (KIND == 0)
            g = scale * (cnt_xy[i] * (float)czn * wv - fv * S[i][0] - S[i][1]);
          else
            g = scale * (wv * S[i][0] - fv * S[i][1] - S[i][2]);
          out[o] = g;
        }
      }
    }
    j = (j + 1 == WW) ? 0 : j + 1;
  }
}

// ---------------------------------------------------------------------------
// The same two kernels with the input planes staged by the tensor memory
// accelerator: one thread issues a 4-D tile copy (x, y, z, volume) per array and
// plane into one of two shared-memory stages, completion is tracked by an
// mbarrier per stage, and the copy of plane z+2 is issued as soon as every
// thread is past the W pass of plane z (the only reader of a stage). The W sums
// are double-buffered: one iteration runs the W pass of plane z and the H and D
// passes of plane z-1, so a plane costs one barrier. The D ring keeps a thread's two
// rows side by side (one 8-byte load and store per moment and plane). Boxes that
// reach outside a volume are filled with zeros by the copy engine. Waits are
// bounded: a wait that runs out sets *err and the kernel carries on (its results
// are then reported as invalid by the host), so no CTA can hang.
// floats of one staged plane (box RXS x RY), rounded up to 128-byte multiples
template <int R, int NM>
__host__ __device__ constexpr int stage_floats() {
  return ((Geo3<R, NM>::RY * Geo3<R, NM>::RXS) + 31) & ~31;
}

template <int R, int KIND>
__global__ void __launch_bounds__(NT3) k_sim_fwd3t(const __grid_constant__ SimMaps maps, const PairDesc* __restrict__ pd,
                                                   const float* __restrict__ Wb, size_t Wstride,
                                                   float* __restrict__ coef, size_t cstride,
                                                   double* __restrict__ part, Dims n, float eps, int tz, int nzc,
                                                   int* __restrict__ err) {
  using G = Geo3<R, 3>;
  constexpr int WW = G::WW, RY = G::RY, RXS = G::RXS, NV = G::NV;
  constexpr int NC = KIND == 0 ? 2 : 3;
  constexpr int TS = stage_floats<R, 3>();
  constexpr unsigned kBytes = 2u * RY * RXS * 4u;  // F and W boxes of one plane
  extern __shared__ __align__(128) float smem_raw[];
  float* smem = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float* stage = smem;                      // [2 stages][F, W][TS]
  float* sx2 = stage + 4 * TS;              // [2 planes][3][RY][T3X]
  // [WW][3][T3Y / YO][T3X] pairs: a thread's YO = 2 rows side by side (one 8-byte access)
  float2* ring2 = reinterpret_cast<float2*>(sx2 + 2 * G::sx_floats());
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ float sh[2 * (NT3 / 32)];
  const int pair = blockIdx.z / nzc, zc = blockIdx.z - pair * nzc;
  const int x0 = blockIdx.x * T3X, y0 = blockIdx.y * T3Y, z0 = zc * tz;
  const int tid = threadIdx.x;
  const PairDesc d = pd[pair];
  const float* __restrict__ F = d.Ii;
  const float* __restrict__ Fs = d.Fs;
  const float* __restrict__ W = Wb + (size_t)pair * Wstride;
  float* __restrict__ C = coef + (size_t)pair * NC * cstride;
  const int plane = n.n1 * n.n2;
  const int zend = min(z0 + tz, n.n0);
  const int niter = (zend - z0) + 2 * R;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int it) {  // one thread: plane z0 + it of F and W into stage it & 1
    const int st = it & 1;
    mbar_expect_tx(&bar[st], kBytes);
    tma_load4(stage + (2 * st) * TS, &maps.F, x0, y0, z0 + it, d.fi, &bar[st]);
    tma_load4(stage + (2 * st + 1) * TS, &maps.W, x0, y0, z0 + it, pair, &bar[st]);
  };
  if (tid == 0) {
    issue(0);
    if (niter > 1) issue(1);
  }
  const int so = min(z0 + R, n.n0 - 1) * plane + min(y0 + R, n.n1 - 1) * n.n2 + min(x0 + R, n.n2 - 1);
  const float shF = F[so], shW = W[so];
  const float inv_nw = 1.f / (float)(WW * WW * WW);
  const int mx = n.n2 - WW, my = n.n1 - WW, mz = n.n0 - WW;
  const int col = tid & 31, yseg = tid >> 5;
  float S[YO][3];
#pragma unroll
  for (int i = 0; i < YO; ++i)
#pragma unroll
    for (int m = 0; m < 3; ++m) S[i][m] = 0.f;
  for (int j = 0; j < WW; ++j)
#pragma unroll
    for (int m = 0; m < 3; ++m) ring2[((j * 3 + m) * (T3Y / YO) + yseg) * T3X + col] = make_float2(0.f, 0.f);
  float lsum = 0.f, lcomp = 0.f;
  const bool xin = x0 + col <= mx;
  int j = 0;
  bool ok = true;
  // Iteration it runs the W pass of input plane it (into sx buffer it & 1) and the H and
  // D passes of plane it - 1 (from the other buffer): one barrier per plane, and warps
  // without a W-pass task go straight on to their H pass.
  for (int it = 0; it <= niter; ++it) {
    const int h = it - 1;  // plane of the H and D passes
    // mu_F and S_FF of this thread's windows of the output plane (corner plane h - 2R),
    // loaded now and used after the W pass
    float muF_c[YO], Sff_c[YO];
    const bool outp = h >= 2 * R;
#pragma unroll
    for (int i = 0; i < YO; ++i) {
      const int cy = y0 + YO * yseg + i, cz = z0 + h - 2 * R;
      muF_c[i] = 0.f;
      Sff_c[i] = 0.f;
      if (outp && xin && cy <= my && cz <= mz) {
        const int o = cz * plane + cy * n.n2 + x0 + col;
        muF_c[i] = Fs[o];
        Sff_c[i] = Fs[(size_t)plane * n.n0 + o];
      }
    }
    if (it < niter) {
      const int st = it & 1;
      ok = ok && mbar_wait(&bar[st], (unsigned)(it >> 1) & 1u);  // after a failure, stop waiting
      const float* sF = stage + (2 * st) * TS;
      const float* sW = sF + TS;
      float* sx = sx2 + st * G::sx_floats();
      for (int task = tid; task < 8 * RY; task += NT3) {
        const int xrow = task >> 3, xseg = task & 7;
        float f[4 * NV], w[4 * NV];
        const float4* pF = reinterpret_cast<const float4*>(sF + xrow * RXS + 4 * xseg);
        const float4* pW = reinterpret_cast<const float4*>(sW + xrow * RXS + 4 * xseg);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const float4 a = pF[q], b = pW[q];
          f[4 * q] = a.x - shF, f[4 * q + 1] = a.y - shF, f[4 * q + 2] = a.z - shF, f[4 * q + 3] = a.w - shF;
          w[4 * q] = b.x - shW, w[4 * q + 1] = b.y - shW, w[4 * q + 2] = b.z - shW, w[4 * q + 3] = b.w - shW;
        }
        float ww[4 + 2 * R], fw[4 + 2 * R];
#pragma unroll
        for (int k = 0; k < 4 + 2 * R; ++k) {
          ww[k] = w[k] * w[k];
          fw[k] = f[k] * w[k];
        }
        float o0[4], o1[4], o2[4];
        runsum<WW, 4>(w, o0);
        runsum<WW, 4>(ww, o1);
        runsum<WW, 4>(fw, o2);
        float4* dst = reinterpret_cast<float4*>(sx + xrow * T3X + 4 * xseg);
        dst[0] = make_float4(o0[0], o0[1], o0[2], o0[3]);
        dst[RY * T3X / 4] = make_float4(o1[0], o1[1], o1[2], o1[3]);
        dst[2 * RY * T3X / 4] = make_float4(o2[0], o2[1], o2[2], o2[3]);
      }
    }
    if (h >= 0) {
      const float* sx = sx2 + (h & 1) * G::sx_floats();
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        float v[YO + 2 * R], a[YO];
#pragma unroll
        for (int k = 0; k < YO + 2 * R; ++k) v[k] = sx[(m * RY + YO * yseg + k) * T3X + col];
        runsum<WW, YO>(v, a);
        float2* rp = ring2 + ((j * 3 + m) * (T3Y / YO) + yseg) * T3X + col;
        const float2 old = *rp;
        S[0][m] += a[0] - old.x;
        S[1][m] += a[1] - old.y;
        *rp = make_float2(a[0], a[1]);
      }
      if (j == WW - 1) {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          float t0[WW], t1[WW];
#pragma unroll
          for (int q = 0; q < WW; ++q) {
            const float2 r = ring2[((q * 3 + m) * (T3Y / YO) + yseg) * T3X + col];
            t0[q] = r.x;
            t1[q] = r.y;
          }
          S[0][m] = TreeSum<WW>::of(t0);
          S[1][m] = TreeSum<WW>::of(t1);
        }
      }
      if (outp) {
        const int cz = z0 + h - 2 * R, cx = x0 + col;
#pragma unroll
        for (int i = 0; i < YO; ++i) {
          const int cy = y0 + YO * yseg + i;
          if (cx >= n.n2 || cy >= n.n1) continue;
          const int o = cz * plane + cy * n.n2 + cx;
          float c0 = 0.f, c1 = 0.f, c2 = 0.f;
          if (cx <= mx && cy <= my && cz <= mz) {
            const float muF = muF_c[i], Sff = Sff_c[i];
            const float Sww = fmaxf(S[i][1] - S[i][0] * S[i][0] * inv_nw, 0.f);
            const float Sfw = S[i][2] - (muF - shF) * S[i][0];
            const float muW = S[i][0] * inv_nw + shW;
            float val;
            if (KIND == 0) {
              const float beta = Sfw * Sff;  // Sff holds 1 / (S_FF + eps) for SiLNCC
              val = (Sww - Sfw * beta) * inv_nw;
              c0 = beta;
              c1 = muW - beta * muF;
            } else {
              const float Q = Sff * Sww + eps;
              const float rq = 1.f / sqrtf(Q);
              val = 1.f - Sfw * rq;
              c0 = Sfw * Sff * rq * rq * rq;
              c1 = rq;
              c2 = c0 * muW - c1 * muF;
            }
            const float yk = val - lcomp;
            const float tk = lsum + yk;
            lcomp = (tk - lsum) - yk;
            lsum = tk;
          }
          C[o] = c0;
          C[cstride + o] = c1;
          if (KIND == 1) C[2 * cstride + o] = c2;
        }
      }
      j = (j + 1 == WW) ? 0 : j + 1;
    }
    // the W pass of this plane is done with its stage (refilled below) and the H pass of
    // the previous plane with its sx buffer (rewritten by the next W pass)
    __syncthreads();
    if (tid == 0 && it + 2 < niter) {
      fence_proxy_async();
      issue(it + 2);
    }
  }
  if (!ok) {
    // report, then give the copies still in flight into this CTA's stages one more bounded
    // wait (the last use of each stage) before the CTA's shared memory is released
    if (err) atomicOr(err, 1);
    for (int st = 0; st < 2 && st < niter; ++st) {
      const int last = niter - 1 - ((niter - 1 - st) & 1);  // last iteration that used stage st
      mbar_wait(&bar[st], (unsigned)(last >> 1) & 1u);
    }
  }
  const double sum = block_sum(FF{lsum, -lcomp}, sh);
  if (threadIdx.x == 0) part[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = sum;
}

// x offset of the adjoint's staged box: its first column x0 - 2R is rounded down to a
// multiple of 4 (16-byte aligned tile coordinate), so the box starts XOFF columns early
template <int R>
__host__ __device__ constexpr int bwd_xoff() {
  return (2 * R) & 3;
}

template <int R, int KIND>
__global__ void __launch_bounds__(NT3) k_sim_bwd3t(const __grid_constant__ SimMaps maps, const PairDesc* __restrict__ pd,
                                                   const float* __restrict__ Wb, size_t Wstride,
                                                   float* __restrict__ dLdW, Dims n, float scale, int tz, int nzc,
                                                   int* __restrict__ err) {
  constexpr int NC = KIND == 0 ? 2 : 3;
  using G = Geo3<R, NC>;
  constexpr int WW = G::WW, RY = G::RY, RXS = G::RXS;
  constexpr int XOFF = bwd_xoff<R>();
  constexpr int TS = stage_floats<R, NC>();
  constexpr unsigned kBytes = (unsigned)NC * RY * RXS * 4u;
  static_assert(XOFF + 4 * 7 + 4 + 2 * R <= RXS, "staged box too narrow for the W pass");
  static_assert((2 * R + XOFF) % 4 == 0, "the staged adjoint box must start at a multiple of 4 floats");
  extern __shared__ __align__(128) float smem_raw[];
  float* smem = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float* stage = smem;                      // [2 stages][NC][TS]
  float* sx2 = stage + 2 * NC * TS;         // [2 planes][NC][RY][T3X]
  // [WW][NC][T3Y / YO][T3X] pairs: a thread's YO = 2 rows side by side (one 8-byte access)
  float2* ring2 = reinterpret_cast<float2*>(sx2 + 2 * G::sx_floats());
  __shared__ __align__(8) uint64_t bar[2];
  const int pair = blockIdx.z / nzc, zc = blockIdx.z - pair * nzc;
  const int x0 = blockIdx.x * T3X, y0 = blockIdx.y * T3Y, z0 = zc * tz;
  const int tid = threadIdx.x;
  const float* __restrict__ F = pd[pair].Ii;
  const float* __restrict__ W = Wb + (size_t)pair * Wstride;
  float* __restrict__ out = dLdW + (size_t)pair * Wstride;
  const int plane = n.n1 * n.n2;
  const int zend = min(z0 + tz, n.n0);
  const int niter = (zend - z0) + 2 * R;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int it) {  // coefficient planes of corner plane z0 - 2R + it into stage it & 1
    const int st = it & 1;
    mbar_expect_tx(&bar[st], kBytes);
#pragma unroll
    for (int m = 0; m < NC; ++m)
      tma_load4(stage + (st * NC + m) * TS, &maps.C, x0 - 2 * R - XOFF, y0 - 2 * R, z0 - 2 * R + it, pair * NC + m,
                &bar[st]);
  };
  if (tid == 0) {
    issue(0);
    if (niter > 1) issue(1);
  }
  const int mx = n.n2 - WW, my = n.n1 - WW, mz = n.n0 - WW;
  const int col = tid & 31, yseg = tid >> 5;
  const int px = x0 + col;
  float cnt_xy[YO];
#pragma unroll
  for (int i = 0; i < YO; ++i) {
    const int py = y0 + YO * yseg + i;
    const int cxn = max(0, min(px, mx) - max(0, px - 2 * R) + 1);
    const int cyn = max(0, min(py, my) - max(0, py - 2 * R) + 1);
    cnt_xy[i] = (float)(cxn * cyn);
  }
  float S[YO][NC];
#pragma unroll
  for (int i = 0; i < YO; ++i)
#pragma unroll
    for (int m = 0; m < NC; ++m) S[i][m] = 0.f;
  for (int j = 0; j < WW; ++j)
#pragma unroll
    for (int m = 0; m < NC; ++m) ring2[((j * NC + m) * (T3Y / YO) + yseg) * T3X + col] = make_float2(0.f, 0.f);
  const bool xin = px < n.n2;
  int j = 0;
  bool ok = true;
  // Iteration it runs the W pass of corner plane it (into sx buffer it & 1) and the H and
  // D passes of corner plane it - 1 (from the other buffer): one barrier per plane.
  // two planes per loop body: 2 % faster for this kernel (the forward one is faster rolled)
#pragma unroll 2
  for (int it = 0; it <= niter; ++it) {
    const int h = it - 1;               // corner plane of the H and D passes
    const int pz = z0 - 2 * R + h;      // output plane completed by it
    const bool outp = h >= 2 * R;
    // W and F at this thread's voxels of the output plane, loaded now, used after the W pass
    float wv_c[YO], fv_c[YO];
#pragma unroll
    for (int i = 0; i < YO; ++i) {
      const int py = y0 + YO * yseg + i;
      wv_c[i] = 0.f;
      fv_c[i] = 0.f;
      if (outp && xin && py < n.n1) {
        const int o = pz * plane + py * n.n2 + px;
        wv_c[i] = W[o];
        fv_c[i] = F[o];
      }
    }
    if (it < niter) {
      const int st = it & 1;
      ok = ok && mbar_wait(&bar[st], (unsigned)(it >> 1) & 1u);  // after a failure, stop waiting
      float* sx = sx2 + st * G::sx_floats();
      for (int task = tid; task < 8 * RY; task += NT3) {
        const int xrow = task >> 3, xseg = task & 7;
#pragma unroll
        for (int m = 0; m < NC; ++m) {
          float v[4 + 2 * R];  // the 4 + 2R inputs of 4 running outputs, as 2 + R 8-byte loads
          const float2* src =
              reinterpret_cast<const float2*>(stage + (st * NC + m) * TS + xrow * RXS + XOFF + 4 * xseg);
#pragma unroll
          for (int q = 0; q < 2 + R; ++q) {
            const float2 a = src[q];
            v[2 * q] = a.x, v[2 * q + 1] = a.y;
          }
          float o[4];
          runsum<WW, 4>(v, o);
          *reinterpret_cast<float4*>(sx + (m * RY + xrow) * T3X + 4 * xseg) = make_float4(o[0], o[1], o[2], o[3]);
        }
      }
    }
    if (h >= 0) {
      const float* sx = sx2 + (h & 1) * G::sx_floats();
#pragma unroll
      for (int m = 0; m < NC; ++m) {
        float v[YO + 2 * R], a[YO];
#pragma unroll
        for (int k = 0; k < YO + 2 * R; ++k) v[k] = sx[(m * RY + YO * yseg + k) * T3X + col];
        runsum<WW, YO>(v, a);
        float2* rp = ring2 + ((j * NC + m) * (T3Y / YO) + yseg) * T3X + col;
        const float2 old = *rp;
        S[0][m] += a[0] - old.x;
        S[1][m] += a[1] - old.y;
        *rp = make_float2(a[0], a[1]);
      }
      if (j == WW - 1) {
#pragma unroll
        for (int m = 0; m < NC; ++m) {
          float t0[WW], t1[WW];
#pragma unroll
          for (int q = 0; q < WW; ++q) {
            const float2 r = ring2[((q * NC + m) * (T3Y / YO) + yseg) * T3X + col];
            t0[q] = r.x;
            t1[q] = r.y;
          }
          S[0][m] = TreeSum<WW>::of(t0);
          S[1][m] = TreeSum<WW>::of(t1);
        }
      }
      if (outp) {
        const int czn = max(0, min(pz, mz) - max(0, pz - 2 * R) + 1);
#pragma unroll
        for (int i = 0; i < YO; ++i) {
          const int py = y0 + YO * yseg + i;
          if (px >= n.n2 || py >= n.n1) continue;
          const int o = pz * plane + py * n.n2 + px;
          const float wv = wv_c[i], fv = fv_c[i];
          float g;
          if (KIND == 0)
            g = scale * (cnt_xy[i] * (float)czn * wv - fv * S[i][0] - S[i][1]);
          else
            g = scale * (wv * S[i][0] - fv * S[i][1] - S[i][2]);
          out[o] = g;
        }
      }
      j = (j + 1 == WW) ? 0 : j + 1;
    }
    // the W pass of this plane is done with its stage (refilled below) and the H pass of
    // the previous plane with its sx buffer (rewritten by the next W pass)
    __syncthreads();
    if (tid == 0 && it + 2 < niter) {
      fence_proxy_async();
      issue(it + 2);
    }
  }
  if (!ok) {
    // report, then give the copies still in flight into this CTA's stages one more bounded
    // wait (the last use of each stage) before the CTA's shared memory is released
    if (err) atomicOr(err, 1);
    for (int st = 0; st < 2 && st < niter; ++st) {
      const int last = niter - 1 - ((niter - 1 - st) & 1);  // last iteration that used stage st
      mbar_wait(&bar[st], (unsigned)(last >> 1) & 1u);
    }
  }
}

template <typename Kern>
cudaError_t set_smem(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int R>
constexpr size_t fwd3_bytes() {
  return sizeof(float) * (Geo3<R, 3>::in_floats(2) + Geo3<R, 3>::sx_floats() + Geo3<R, 3>::ring_floats());
}
template <int R, int KIND>
constexpr size_t bwd3_bytes() {
  return sizeof(float) * (Geo3<R, KIND == 0 ? 2 : 3>::in_floats(KIND == 0 ? 2 : 3) +
                          Geo3<R, KIND == 0 ? 2 : 3>::sx_floats() + Geo3<R, KIND == 0 ? 2 : 3>::ring_floats());
}
template <int R>
constexpr size_t fwd3t_bytes() {
  return 128 + sizeof(float) * (4 * stage_floats<R, 3>() + 2 * Geo3<R, 3>::sx_floats() + Geo3<R, 3>::ring_floats());
}
template <int R, int KIND>
constexpr size_t bwd3t_bytes() {
  return 128 + sizeof(float) * (2 * (KIND == 0 ? 2 : 3) * stage_floats<R, KIND == 0 ? 2 : 3>() +
                                2 * Geo3<R, KIND == 0 ? 2 : 3>::sx_floats() + Geo3<R, KIND == 0 ? 2 : 3>::ring_floats());
}
template <int R, int KIND>
void fwd3(dim3 g, const PairDesc* pd, const float* W, size_t Ws, float* coef, size_t cs, double* part, Dims n,
          float eps, int tz, int nzc, cudaStream_t s) {
  k_sim_fwd3<R, KIND><<<g, NT3, fwd3_bytes<R>(), s>>>(pd, W, Ws, coef, cs, part, n, eps, tz, nzc);
}
template <int R, int KIND>
void bwd3(dim3 g, const PairDesc* pd, const float* W, size_t Ws, const float* coef, size_t cs, float* dLdW, Dims n,
          float scale, int tz, int nzc, cudaStream_t s) {
  k_sim_bwd3<R, KIND><<<g, NT3, bwd3_bytes<R, KIND>(), s>>>(pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc);
}
template <int R>
cudaError_t prepare_r() {
  const cudaError_t e[8] = {set_smem(k_sim_fwd3<R, 0>, fwd3_bytes<R>()),   set_smem(k_sim_fwd3<R, 1>, fwd3_bytes<R>()),
                            set_smem(k_sim_bwd3<R, 0>, bwd3_bytes<R, 0>()), set_smem(k_sim_bwd3<R, 1>, bwd3_bytes<R, 1>()),
                            set_smem(k_sim_fwd3t<R, 0>, fwd3t_bytes<R>()), set_smem(k_sim_fwd3t<R, 1>, fwd3t_bytes<R>()),
                            set_smem(k_sim_bwd3t<R, 0>, bwd3t_bytes<R, 0>()),
                            set_smem(k_sim_bwd3t<R, 1>, bwd3t_bytes<R, 1>())};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}
template <int R, int KIND>
void fwd3t(dim3 g, const SimMaps& m, const PairDesc* pd, const float* W, size_t Ws, float* coef, size_t cs,
           double* part, Dims n, float eps, int tz, int nzc, int* err, cudaStream_t s) {
  k_sim_fwd3t<R, KIND><<<g, NT3, fwd3t_bytes<R>(), s>>>(m, pd, W, Ws, coef, cs, part, n, eps, tz, nzc, err);
}
template <int R, int KIND>
void bwd3t(dim3 g, const SimMaps& m, const PairDesc* pd, const float* W, size_t Ws, float* dLdW, Dims n,
           float scale, int tz, int nzc, int* err, cudaStream_t s) {
  k_sim_bwd3t<R, KIND><<<g, NT3, bwd3t_bytes<R, KIND>(), s>>>(m, pd, W, Ws, dLdW, n, scale, tz, nzc, err);
}
template <int KIND>
void fwd_dispatch_t(int R, dim3 g, const SimMaps& m, const PairDesc* pd, const float* W, size_t Ws, float* coef,
                    size_t cs, double* part, Dims n, float eps, int tz, int nzc, int* err, cudaStream_t s) {
  switch (R) {
    case 1: fwd3t<1, KIND>(g, m, pd, W, Ws, coef, cs, part, n, eps, tz, nzc, err, s); break;
    case 2: fwd3t<2, KIND>(g, m, pd, W, Ws, coef, cs, part, n, eps, tz, nzc, err, s); break;
    case 3: fwd3t<3, KIND>(g, m, pd, W, Ws, coef, cs, part, n, eps, tz, nzc, err, s); break;
    case 4: fwd3t<4, KIND>(g, m, pd, W, Ws, coef, cs, part, n, eps, tz, nzc, err, s); break;
    case 5: fwd3t<5, KIND>(g, m, pd, W, Ws, coef, cs, part, n, eps, tz, nzc, err, s); break;
    default: break;
  }
}
template <int KIND>
void bwd_dispatch_t(int R, dim3 g, const SimMaps& m, const PairDesc* pd, const float* W, size_t Ws, float* dLdW,
                    Dims n, float scale, int tz, int nzc, int* err, cudaStream_t s) {
  switch (R) {
    case 1: bwd3t<1, KIND>(g, m, pd, W, Ws, dLdW, n, scale, tz, nzc, err, s); break;
    case 2: bwd3t<2, KIND>(g, m, pd, W, Ws, dLdW, n, scale, tz, nzc, err, s); break;
    case 3: bwd3t<3, KIND>(g, m, pd, W, Ws, dLdW, n, scale, tz, nzc, err, s); break;
    case 4: bwd3t<4, KIND>(g, m, pd, W, Ws, dLdW, n, scale, tz, nzc, err, s); break;
    case 5: bwd3t<5, KIND>(g, m, pd, W, Ws, dLdW, n, scale, tz, nzc, err, s); break;
    default: break;
  }
}

}  // namespace

// ---- tensor maps (host): the encoder comes from the driver through the runtime's entry
// point query, so the library needs no link against the driver library
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

bool encode_volumes(CUtensorMap* m, const float* base, Dims n, int n_vol, int box_x, int box_y, int box_z) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !base || n_vol < 1 || box_x > 256 || box_y > 256 || box_z < 1 || box_z > 256 || (box_x & 3))
    return false;
  if ((n.n2 & 3) || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)n.n2, (cuuint64_t)n.n1, (cuuint64_t)n.n0, (cuuint64_t)n_vol};
  const cuuint64_t row = (cuuint64_t)n.n2 * 4;
  const cuuint64_t strides[3] = {row, row * n.n1, row * n.n1 * n.n0};
  const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)box_z, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {
int staged_row(int R) {  // RXS of Geo3<R, *>
  switch (R) {
    case 1: return Geo3<1, 2>::RXS;
    case 2: return Geo3<2, 2>::RXS;
    case 3: return Geo3<3, 2>::RXS;
    case 4: return Geo3<4, 2>::RXS;
    case 5: return Geo3<5, 2>::RXS;
    default: return 0;
  }
}

template <int KIND>
void fwd_dispatch(int R, dim3 g, const PairDesc* pd, const float* W, size_t Ws, float* coef, size_t cs, double* part,
                  Dims n, float eps, int tz, int nzc, cudaStream_t s) {
  switch (R) {
    case 1: fwd3<1, KIND>(g, pd, W, Ws, coef, cs, part, n, eps, tz, nzc, s); break;
    case 2: fwd3<2, KIND>(g, pd, W, Ws, coef, cs, part, n, eps, tz, nzc, s); break;
    case 3: fwd3<3, KIND>(g, pd, W, Ws, coef, cs, part, n, eps, tz, nzc, s); break;
    case 4: fwd3<4, KIND>(g, pd, W, Ws, coef, cs, part, n, eps, tz, nzc, s); break;
    case 5: fwd3<5, KIND>(g, pd, W, Ws, coef, cs, part, n, eps, tz, nzc, s); break;
    default: break;
  }
}
template <int KIND>
void bwd_dispatch(int R, dim3 g, const PairDesc* pd, const float* W, size_t Ws, const float* coef, size_t cs,
                  float* dLdW, Dims n, float scale, int tz, int nzc, cudaStream_t s) {
  switch (R) {
    case 1: bwd3<1, KIND>(g, pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc, s); break;
    case 2: bwd3<2, KIND>(g, pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc, s); break;
    case 3: bwd3<3, KIND>(g, pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc, s); break;
    case 4: bwd3<4, KIND>(g, pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc, s); break;
    case 5: bwd3<5, KIND>(g, pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc, s); break;
    default: break;
  }
}

// D chunk of one CTA: every chunk streams 2R planes more than it covers, so D is split only
// while one pair has fewer than 16384 threads and the launch (batch pairs) fewer than 1824
// CTAs (four waves of three CTAs on each of 152 SMs), and halved only while above min_chunk planes
int chunk_for(int ntiles, int depth, int min_chunk, int threads, int batch) {
  int tz = depth;
  for (;;) {
    const long chunks = (depth + tz - 1) / tz;
    if (tz <= min_chunk || (long)ntiles * chunks * threads >= 16384 || (long)batch * ntiles * chunks >= 1824) break;
    tz = (tz + 1) / 2;
  }
  return tz < 1 ? 1 : tz;
}

dim3 sim_grid(Dims ni, int window, int n_pairs, int batch, SimGeom* geo) {
  (void)window;
  const int gx = (ni.n2 + T3X - 1) / T3X, gy = (ni.n1 + T3Y - 1) / T3Y;
  SimGeom g;
  g.tz = chunk_for(gx * gy, ni.n0, 8, NT3, batch);
  g.nzc = (ni.n0 + g.tz - 1) / g.tz;
  g.ctas = gx * gy * g.nzc;
  if (geo) *geo = g;
  return dim3(gx, gy, g.nzc * n_pairs);
}
}  // namespace

namespace {
template <int KIND>
void fixed_stats(dim3 g, const float* imgs, Dims ni, int window, float eps, float* stats, int tz, int nzc,
                 cudaStream_t s) {
  switch (window / 2) {
    case 1: k_fixed_stats<1, KIND><<<g, kThreads, 0, s>>>(imgs, stats, ni, tz, nzc, eps); break;
    case 2: k_fixed_stats<2, KIND><<<g, kThreads, 0, s>>>(imgs, stats, ni, tz, nzc, eps); break;
    case 3: k_fixed_stats<3, KIND><<<g, kThreads, 0, s>>>(imgs, stats, ni, tz, nzc, eps); break;
    case 4: k_fixed_stats<4, KIND><<<g, kThreads, 0, s>>>(imgs, stats, ni, tz, nzc, eps); break;
    case 5: k_fixed_stats<5, KIND><<<g, kThreads, 0, s>>>(imgs, stats, ni, tz, nzc, eps); break;
    default: break;
  }
}
}  // namespace

void launch_fixed_stats(const float* imgs, int n_images, Dims ni, int window, int kind, float eps, float* stats,
                        cudaStream_t s) {
  const int gx = (ni.n2 + TX - 1) / TX, gy = (ni.n1 + 7) / 8;
  const int tz = chunk_for(gx * gy, ni.n0, 16, 128, 1), nzc = (ni.n0 + tz - 1) / tz;
  const dim3 g(gx, gy, nzc * n_images);
  if (kind == 0)
    fixed_stats<0>(g, imgs, ni, window, eps, stats, tz, nzc, s);
  else
    fixed_stats<1>(g, imgs, ni, window, eps, stats, tz, nzc, s);
}

cudaError_t prepare_kernels() {
  // dynamic shared memory limits of the similarity kernels, once per device
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  return once_per_device(done, mu, [] {
    const cudaError_t e[5] = {prepare_r<1>(), prepare_r<2>(), prepare_r<3>(), prepare_r<4>(), prepare_r<5>()};
    for (cudaError_t x : e)
      if (x != cudaSuccess) return x;
    return cudaSuccess;
  });
}

SimGeom sim_geom(Dims ni, int window, int batch) {
  SimGeom g;
  sim_grid(ni, window, 1, batch, &g);
  return g;
}
int sim_ncoef(int kind) { return kind == 0 ? 2 : 3; }

void make_sim_maps(SimMaps* m, const float* W, int n_pairs, const float* imgs, int n_images, const float* coef,
                   Dims ni, int window, int kind) {
  memset(m, 0, sizeof(*m));
  const int R = window / 2, rxs = staged_row(R), ry = T3Y + 2 * R;
  if (!rxs) return;
  m->fwd_ok =
      encode_volumes(&m->W, W, ni, n_pairs, rxs, ry, 1) && encode_volumes(&m->F, imgs, ni, n_images, rxs, ry, 1);
  m->bwd_ok = encode_volumes(&m->C, coef, ni, n_pairs * sim_ncoef(kind), rxs, ry, 1);
}

void launch_sim_fwd(const PairDesc* pd, int n_pairs, int batch, const float* W, size_t Wstride, float* coef,
                    size_t cs, double* partials, Dims ni, int window, int kind, float eps, const SimMaps* maps,
                    int* err, cudaStream_t s) {
  SimGeom g;
  const dim3 grid = sim_grid(ni, window, n_pairs, batch, &g);
  const int R = window / 2;
  if (maps && maps->fwd_ok) {
    if (kind == 0)
      fwd_dispatch_t<0>(R, grid, *maps, pd, W, Wstride, coef, cs, partials, ni, eps, g.tz, g.nzc, err, s);
    else
      fwd_dispatch_t<1>(R, grid, *maps, pd, W, Wstride, coef, cs, partials, ni, eps, g.tz, g.nzc, err, s);
    return;
  }
  if (kind == 0)
    fwd_dispatch<0>(R, grid, pd, W, Wstride, coef, cs, partials, ni, eps, g.tz, g.nzc, s);
  else
    fwd_dispatch<1>(R, grid, pd, W, Wstride, coef, cs, partials, ni, eps, g.tz, g.nzc, s);
}
void launch_sim_bwd(const PairDesc* pd, int n_pairs, int batch, const float* W, size_t Wstride, const float* coef,
                    size_t cs, float* dLdW, Dims ni, int window, int kind, float scale, const SimMaps* maps, int* err,
                    cudaStream_t s) {
  SimGeom g;
  const dim3 grid = sim_grid(ni, window, n_pairs, batch, &g);
  const int R = window / 2;
  if (maps && maps->bwd_ok) {
    if (kind == 0)
      bwd_dispatch_t<0>(R, grid, *maps, pd, W, Wstride, dLdW, ni, scale, g.tz, g.nzc, err, s);
    else
      bwd_dispatch_t<1>(R, grid, *maps, pd, W, Wstride, dLdW, ni, scale, g.tz, g.nzc, err, s);
    return;
  }
  if (kind == 0)
    bwd_dispatch<0>(R, grid, pd, W, Wstride, coef, cs, dLdW, ni, scale, g.tz, g.nzc, s);
  else
    bwd_dispatch<1>(R, grid, pd, W, Wstride, coef, cs, dLdW, ni, scale, g.tz, g.nzc, s);
}

}  // namespace muster
