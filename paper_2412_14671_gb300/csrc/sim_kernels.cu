// sim_kernels.cu -- the windowed similarity of Eq. LNCC / the SiLNCC equation,
// averaged over the valid windows (Eq. sum_lncc, Eq. sim_loss), and its adjoint.
//
// Window R has lower corner c (centre c + R); the valid corners are
// 0 <= c_a <= n_a - w. Both kernels stream along D: a CTA owns a 32 (W) x 8*CY
// (H) tile of windows (forward) or voxels (adjoint) and a chunk of D. Per plane
// it loads the (32 + 2R) x (8*CY + 2R) halo region into shared memory once
// (per-thread load offsets are fixed for the whole column), sums along W in
// shared memory, along H in registers (CY consecutive rows per thread share the
// H sums), and keeps the last 2R+1 plane sums in registers for the sum along D
// as a running sum that is re-summed exactly every 2R+1 planes.
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
#include "kernels.h"

namespace muster {

namespace {
constexpr int kThreads = 256, TX = 32;

constexpr int cy_for(int R) { return R <= 2 ? 2 : 1; }

__device__ __forceinline__ double block_sum(double x, double* sh) {
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

// Statistics of the fixed image of every window, once per session and level:
// out[0][c] = mu_F, out[1][c] = S_FF (centred sum of squares) at corner c.
template <int R>
__global__ void __launch_bounds__(kThreads) k_fixed_stats(const float* __restrict__ imgs, float* __restrict__ stats,
                                                          Dims n, int tz, int nzc) {
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
          out[V + o] = fmaxf(S[1] - S[0] * S[0] * inv_nw, 0.f);
        }
      }
    }
  }
}

// Forward per pair: box sums of W', W'^2 and F'W' (primes: shifted by a voxel of
// the tile); mu_F and S_FF of the window come from k_fixed_stats.
template <int R, int KIND, int CY>
__global__ void __launch_bounds__(kThreads) k_sim_fwd2(const PairDesc* __restrict__ pd, const float* __restrict__ Wb,
                                                       size_t Wstride, float* __restrict__ coef, size_t cstride,
                                                       double* __restrict__ part, Dims n, float eps, int tz, int nzc) {
  constexpr int WW = 2 * R + 1, TY = 8 * CY, RX = TX + 2 * R, RY = TY + 2 * R;
  constexpr int NE = RY * RX, NSLOT = (NE + kThreads - 1) / kThreads;
  constexpr int NC = KIND == 0 ? 2 : 3;
  constexpr int NM = 3;  // sum W', sum W'^2, sum F'W'
  __shared__ float sF[NE], sW[NE];
  __shared__ float sx[NM][RY][TX];
  __shared__ double sh[kThreads / 32];
  const int pair = blockIdx.z / nzc, zc = blockIdx.z - pair * nzc;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = zc * tz;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const PairDesc d = pd[pair];
  const float* __restrict__ F = d.Ii;
  const float* __restrict__ Fs = d.Fs;
  const float* __restrict__ W = Wb + (size_t)pair * Wstride;
  float* __restrict__ C = coef + (size_t)pair * NC * cstride;
  const int plane = n.n1 * n.n2;
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
  const int so = min(z0 + R, n.n0 - 1) * plane + min(y0 + R, n.n1 - 1) * n.n2 + min(x0 + R, n.n2 - 1);
  const float shF = F[so], shW = W[so];
  const float nw = (float)(WW * WW * WW), inv_nw = 1.f / nw;
  const int mx = n.n2 - WW, my = n.n1 - WW, mz = n.n0 - WW;
  const int cx = x0 + tx;
  float ring[CY][NM][WW], S[CY][NM];
#pragma unroll
  for (int c = 0; c < CY; ++c)
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      S[c][m] = 0.f;
#pragma unroll
      for (int k = 0; k < WW; ++k) ring[c][m][k] = 0.f;
    }
  float lsum = 0.f, lcomp = 0.f;
  const int zend = min(z0 + tz, n.n0);
  const int niter = (zend - z0) + 2 * R;
  // plane loads are issued one plane ahead, into registers
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
  fetch(z0);
  for (int base = 0; base < niter; base += WW) {
#pragma unroll
    for (int j = 0; j < WW; ++j) {
      const int it = base + j;
      if (it >= niter) break;
      const int zin = z0 + it;
#pragma unroll
      for (int k = 0; k < NSLOT; ++k) {
        const int e = tid + kThreads * k;
        if (e < NE) {
          sF[e] = pf[k];
          sW[e] = pw[k];
        }
      }
      __syncthreads();
      if (it + 1 < niter) fetch(zin + 1);
      for (int ry = ty; ry < RY; ry += kThreads / 32) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        const float* qf = sF + ry * RX + tx;
        const float* qw = sW + ry * RX + tx;
#pragma unroll
        for (int k = 0; k < WW; ++k) {
          const float f = qf[k], w = qw[k];
          a0 += w;
          a1 = fmaf(w, w, a1);
          a2 = fmaf(f, w, a2);
        }
        sx[0][ry][tx] = a0;
        sx[1][ry][tx] = a1;
        sx[2][ry][tx] = a2;
      }
      __syncthreads();
      // H sums of this plane for the CY windows of the thread, then the running D sum
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < WW; ++k) v += sx[m][ty * CY + k][tx];
        float a[CY];
        a[0] = v;
        if (CY == 2) a[CY - 1] = v - sx[m][ty * CY][tx] + sx[m][ty * CY + WW][tx];
#pragma unroll
        for (int c = 0; c < CY; ++c) {
          S[c][m] += a[c] - ring[c][m][j];
          ring[c][m][j] = a[c];
          if (j == WW - 1) {  // exact re-sum bounds the drift of the running sum
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < WW; ++k) t += ring[c][m][k];
            S[c][m] = t;
          }
        }
      }
      if (it >= 2 * R) {
        const int cz = zin - 2 * R;
#pragma unroll
        for (int c = 0; c < CY; ++c) {
          const int cy = y0 + ty * CY + c;
          if (cx >= n.n2 || cy >= n.n1) continue;
          const int o = cz * plane + cy * n.n2 + cx;
          float c0 = 0.f, c1 = 0.f, c2 = 0.f;
          if (cx <= mx && cy <= my && cz <= mz) {
            const float muF = Fs[o], Sff = Fs[(size_t)plane * n.n0 + o];
            const float* s = S[c];
            const float Sww = fmaxf(s[1] - s[0] * s[0] * inv_nw, 0.f);
            const float Sfw = s[2] - (muF - shF) * s[0];
            const float muW = s[0] * inv_nw + shW;
            float val;
            if (KIND == 0) {
              const float beta = Sfw / (Sff + eps);
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
  }
  const double sum = block_sum((double)lsum - (double)lcomp, sh);
  if (threadIdx.x == 0) part[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = sum;
}

template <int R, int KIND, int CY>
__global__ void __launch_bounds__(kThreads) k_sim_bwd2(const PairDesc* __restrict__ pd, const float* __restrict__ Wb,
                                                       size_t Wstride, const float* __restrict__ coef, size_t cstride,
                                                       float* __restrict__ dLdW, Dims n, float scale, int tz, int nzc) {
  constexpr int WW = 2 * R + 1, TY = 8 * CY, RX = TX + 2 * R, RY = TY + 2 * R;
  constexpr int NE = RY * RX, NSLOT = (NE + kThreads - 1) / kThreads;
  constexpr int NC = KIND == 0 ? 2 : 3;
  __shared__ float sc[NC][NE];
  __shared__ float sx[NC][RY][TX];
  const int pair = blockIdx.z / nzc, zc = blockIdx.z - pair * nzc;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = zc * tz;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const float* __restrict__ F = pd[pair].Ii;
  const float* __restrict__ W = Wb + (size_t)pair * Wstride;
  const float* __restrict__ Cf = coef + (size_t)pair * NC * cstride;
  float* __restrict__ out = dLdW + (size_t)pair * Wstride;
  const int plane = n.n1 * n.n2;
  int soff[NSLOT];
  bool sok[NSLOT];
#pragma unroll
  for (int k = 0; k < NSLOT; ++k) {
    const int e = tid + kThreads * k;
    const int ry = e / RX, rx = e - ry * RX;
    const int gy = y0 - 2 * R + ry, gx = x0 - 2 * R + rx;
    sok[k] = e < NE && gy >= 0 && gy < n.n1 && gx >= 0 && gx < n.n2;
    soff[k] = gy * n.n2 + gx;
  }
  const int px = x0 + tx;
  const int mx = n.n2 - WW, my = n.n1 - WW, mz = n.n0 - WW;
  float cnt_xy[CY];
#pragma unroll
  for (int c = 0; c < CY; ++c) {
    const int py = y0 + ty * CY + c;
    const int cxn = max(0, min(px, mx) - max(0, px - 2 * R) + 1);
    const int cyn = max(0, min(py, my) - max(0, py - 2 * R) + 1);
    cnt_xy[c] = (float)(cxn * cyn);
  }
  float ring[CY][NC][WW], S[CY][NC];
#pragma unroll
  for (int c = 0; c < CY; ++c)
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      S[c][m] = 0.f;
#pragma unroll
      for (int k = 0; k < WW; ++k) ring[c][m][k] = 0.f;
    }
  const int zend = min(z0 + tz, n.n0);
  const int niter = (zend - z0) + 2 * R;
  // coefficient planes are loaded one plane ahead, into registers
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
  fetch(z0 - 2 * R);
  for (int base = 0; base < niter; base += WW) {
#pragma unroll
    for (int j = 0; j < WW; ++j) {
      const int it = base + j;
      if (it >= niter) break;
      const int zin = z0 - 2 * R + it;  // corner plane
#pragma unroll
      for (int k = 0; k < NSLOT; ++k) {
        const int e = tid + kThreads * k;
        if (e < NE) {
#pragma unroll
          for (int m = 0; m < NC; ++m) sc[m][e] = pc[m][k];
        }
      }
      __syncthreads();
      if (it + 1 < niter) fetch(zin + 1);
      for (int ry = ty; ry < RY; ry += kThreads / 32) {
#pragma unroll
        for (int m = 0; m < NC; ++m) {
          const float* p = sc[m] + ry * RX + tx;
          float a = 0.f;
#pragma unroll
          for (int k = 0; k < WW; ++k) a += p[k];
          sx[m][ry][tx] = a;
        }
      }
      __syncthreads();
#pragma unroll
      for (int m = 0; m < NC; ++m) {
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < WW; ++k) v += sx[m][ty * CY + k][tx];
        float a[CY];
        a[0] = v;
        if (CY == 2) a[CY - 1] = v - sx[m][ty * CY][tx] + sx[m][ty * CY + WW][tx];
#pragma unroll
        for (int c = 0; c < CY; ++c) {
          S[c][m] += a[c] - ring[c][m][j];
          ring[c][m][j] = a[c];
          if (j == WW - 1) {
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < WW; ++k) t += ring[c][m][k];
            S[c][m] = t;
          }
        }
      }
      if (it >= 2 * R) {
        const int pz = zin;
        const int czn = max(0, min(pz, mz) - max(0, pz - 2 * R) + 1);
#pragma unroll
        for (int c = 0; c < CY; ++c) {
          const int py = y0 + ty * CY + c;
          if (px < n.n2 && py < n.n1) {
            const int o = pz * plane + py * n.n2 + px;
            const float wv = W[o], fv = F[o];
            float g;
            if (KIND == 0)
              g = scale * (cnt_xy[c] * (float)czn * wv - fv * S[c][0] - S[c][1]);
            else
              g = scale * (wv * S[c][0] - fv * S[c][1] - S[c][2]);
            out[o] = g;
          }
        }
      }
    }
  }
}

template <int KIND>
void fwd_dispatch(int R, dim3 g, const PairDesc* pd, const float* W, size_t Ws, float* coef, size_t cs, double* part,
                  Dims n, float eps, int tz, int nzc, cudaStream_t s) {
  switch (R) {
    case 1: k_sim_fwd2<1, KIND, cy_for(1)><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, part, n, eps, tz, nzc); break;
    case 2: k_sim_fwd2<2, KIND, cy_for(2)><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, part, n, eps, tz, nzc); break;
    case 3: k_sim_fwd2<3, KIND, cy_for(3)><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, part, n, eps, tz, nzc); break;
    case 4: k_sim_fwd2<4, KIND, cy_for(4)><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, part, n, eps, tz, nzc); break;
    case 5: k_sim_fwd2<5, KIND, cy_for(5)><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, part, n, eps, tz, nzc); break;
    default: break;
  }
}
template <int KIND>
void bwd_dispatch(int R, dim3 g, const PairDesc* pd, const float* W, size_t Ws, const float* coef, size_t cs,
                  float* dLdW, Dims n, float scale, int tz, int nzc, cudaStream_t s) {
  switch (R) {
    case 1: k_sim_bwd2<1, KIND, cy_for(1)><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc); break;
    case 2: k_sim_bwd2<2, KIND, cy_for(2)><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc); break;
    case 3: k_sim_bwd2<3, KIND, cy_for(3)><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc); break;
    case 4: k_sim_bwd2<4, KIND, cy_for(4)><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc); break;
    case 5: k_sim_bwd2<5, KIND, cy_for(5)><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc); break;
    default: break;
  }
}

int chunk_for(int ntiles, int depth, int min_chunk) {
  // split D so that one pair has at least 128 CTAs when the volume allows it
  int tz = depth;
  while (tz > min_chunk && (long)ntiles * ((depth + tz - 1) / tz) < 128) tz = (tz + 1) / 2;
  return tz < 1 ? 1 : tz;
}

dim3 sim_grid(Dims ni, int window, int n_pairs, SimGeom* geo) {
  const int TY = 8 * cy_for(window / 2);
  const int gx = (ni.n2 + TX - 1) / TX, gy = (ni.n1 + TY - 1) / TY;
  SimGeom g;
  g.tz = chunk_for(gx * gy, ni.n0, 16);
  g.nzc = (ni.n0 + g.tz - 1) / g.tz;
  g.ctas = gx * gy * g.nzc;
  if (geo) *geo = g;
  return dim3(gx, gy, g.nzc * n_pairs);
}
}  // namespace

void launch_fixed_stats(const float* imgs, int n_images, Dims ni, int window, float* stats, cudaStream_t s) {
  const int gx = (ni.n2 + TX - 1) / TX, gy = (ni.n1 + 7) / 8;
  const int tz = chunk_for(gx * gy, ni.n0, 16), nzc = (ni.n0 + tz - 1) / tz;
  const dim3 g(gx, gy, nzc * n_images);
  switch (window / 2) {
    case 1: k_fixed_stats<1><<<g, kThreads, 0, s>>>(imgs, stats, ni, tz, nzc); break;
    case 2: k_fixed_stats<2><<<g, kThreads, 0, s>>>(imgs, stats, ni, tz, nzc); break;
    case 3: k_fixed_stats<3><<<g, kThreads, 0, s>>>(imgs, stats, ni, tz, nzc); break;
    case 4: k_fixed_stats<4><<<g, kThreads, 0, s>>>(imgs, stats, ni, tz, nzc); break;
    case 5: k_fixed_stats<5><<<g, kThreads, 0, s>>>(imgs, stats, ni, tz, nzc); break;
    default: break;
  }
}

SimGeom sim_geom(Dims ni, int window) {
  SimGeom g;
  sim_grid(ni, window, 1, &g);
  return g;
}
int sim_ncoef(int kind) { return kind == 0 ? 2 : 3; }

void launch_sim_fwd(const PairDesc* pd, int n_pairs, const float* W, size_t Wstride, float* coef, size_t cs,
                    double* partials, Dims ni, int window, int kind, float eps, cudaStream_t s) {
  SimGeom g;
  const dim3 grid = sim_grid(ni, window, n_pairs, &g);
  const int R = window / 2;
  if (kind == 0)
    fwd_dispatch<0>(R, grid, pd, W, Wstride, coef, cs, partials, ni, eps, g.tz, g.nzc, s);
  else
    fwd_dispatch<1>(R, grid, pd, W, Wstride, coef, cs, partials, ni, eps, g.tz, g.nzc, s);
}
void launch_sim_bwd(const PairDesc* pd, int n_pairs, const float* W, size_t Wstride, const float* coef, size_t cs,
                    float* dLdW, Dims ni, int window, int kind, float scale, cudaStream_t s) {
  SimGeom g;
  const dim3 grid = sim_grid(ni, window, n_pairs, &g);
  const int R = window / 2;
  if (kind == 0)
    bwd_dispatch<0>(R, grid, pd, W, Wstride, coef, cs, dLdW, ni, scale, g.tz, g.nzc, s);
  else
    bwd_dispatch<1>(R, grid, pd, W, Wstride, coef, cs, dLdW, ni, scale, g.tz, g.nzc, s);
}

}  // namespace muster
