// image_kernels.cu -- kernels on the image grid of a pyramid level: the 2x2x2
// pyramid, the warp I_k o Phi_ki^i with the flow-to-image upsample fused in, the
// windowed similarity (Eq. LNCC / the SiLNCC equation, averaged as in Eq.
// sum_lncc) with its adjoint, the warp adjoint fused with the transposed
// upsample, and the deterministic loss reduction.
//
// Windowed sums are separable and streamed along D: a CTA owns a 32 (W) x 8 (H)
// column of windows, loads one plane of the (32+2R) x (8+2R) halo region at a
// time into shared memory, sums along W and H there, and keeps the last 2R+1
// plane sums in registers for the sum along D. Each voxel is loaded once per
// column (plus the H/W halo), never re-read from DRAM for the D direction.
#include <algorithm>
#include <cfloat>

#include "kernels.h"

namespace muster {

namespace {
constexpr int kThreads = 256;
constexpr int TX = 32, TY = 8;  // window tile of the similarity kernels
constexpr int FX = 32, FY = 8;  // flow tile of the warp adjoint

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

// ---- warp: W(p) = S[I_k](p + 2 S[U](q(p)))
__global__ void k_warp(const PairDesc* __restrict__ pd, Dims ni, Dims nf, float* __restrict__ W, size_t stride) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= (int)vox(ni)) return;
  const PairDesc d = pd[blockIdx.y];
  int z, y, x;
  unflat(ni, v, z, y, x);
  const float4 u = sample4(d.U, nf, centre(z), centre(y), centre(x));
  W[(size_t)blockIdx.y * stride + v] = sample1(d.Ik, ni, z + 2.f * u.x, y + 2.f * u.y, x + 2.f * u.z);
}

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

// ---- windowed similarity, forward.
// Window R (centre voxel c + R) has lower corner c; the valid corners are
// 0 <= c_a <= n_a - w. For every corner of the image grid the kernel writes the
// coefficients of dSim_R/dW(p) = A_R W(p) - B_R F(p) - C_R (zero for invalid
// corners) and adds Sim_R to the loss:
//   SiLNCC: A = 2/|R| (implicit), B = beta = S_FW/(S_FF+eps), C = mu_W - beta mu_F
//           (the 2/|R| factor is applied in the adjoint);
//   LNCC:   A = S_FW S_FF / Q^{3/2}, B = 1/sqrt(Q), C = A mu_W - B mu_F, Q = S_FF S_WW + eps.
// Sums are taken on values shifted by one voxel of the tile (variance is shift
// invariant) to limit cancellation in S = sum x^2 - (sum x)^2 / |R|.
template <int R, int KIND>
__global__ void __launch_bounds__(kThreads) k_sim_fwd(const PairDesc* __restrict__ pd, const float* __restrict__ Wb,
                                                      size_t Wstride, float* __restrict__ coef, size_t cstride,
                                                      double* __restrict__ part, Dims n, float eps, int tz, int nzc) {
  constexpr int WW = 2 * R + 1, RX = TX + 2 * R, RY = TY + 2 * R;
  constexpr int NC = KIND == 0 ? 2 : 3;
  __shared__ float sF[RY][RX], sW[RY][RX];
  __shared__ float sx[5][RY][TX];
  __shared__ double sh[kThreads / 32];
  const int pair = blockIdx.z / nzc, zc = blockIdx.z - pair * nzc;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = zc * tz;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const float* __restrict__ F = pd[pair].Ii;
  const float* __restrict__ W = Wb + (size_t)pair * Wstride;
  float* __restrict__ C = coef + (size_t)pair * NC * cstride;
  const int mx = n.n2 - WW, my = n.n1 - WW, mz = n.n0 - WW;
  const int cx = x0 + tx, cy = y0 + ty;
  const size_t so = ((size_t)min(z0 + R, n.n0 - 1) * n.n1 + min(y0 + R, n.n1 - 1)) * n.n2 + min(x0 + R, n.n2 - 1);
  const float shF = F[so], shW = W[so];
  const float inv_nw = 1.f / (float)(WW * WW * WW);
  float ring[5][WW];
  float lsum = 0.f, lcomp = 0.f;
  const int zend = min(z0 + tz, n.n0);
  const int niter = (zend - z0) + 2 * R;
  for (int base = 0; base < niter; base += WW) {
#pragma unroll
    for (int j = 0; j < WW; ++j) {
      const int it = base + j;
      if (it >= niter) break;
      const int zin = z0 + it;
      for (int e = threadIdx.x; e < RY * RX; e += kThreads) {
        const int ry = e / RX, rx = e - ry * RX;
        const int gy = y0 + ry, gx = x0 + rx;
        float f = 0.f, w = 0.f;
        if (zin < n.n0 && gy < n.n1 && gx < n.n2) {
          const size_t o = ((size_t)zin * n.n1 + gy) * n.n2 + gx;
          f = F[o] - shF;
          w = W[o] - shW;
        }
        sF[ry][rx] = f;
        sW[ry][rx] = w;
      }
      __syncthreads();
      for (int ry = ty; ry < RY; ry += kThreads / 32) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
        for (int k = 0; k < WW; ++k) {
          const float f = sF[ry][tx + k], w = sW[ry][tx + k];
          a0 += f;
          a1 += w;
          a2 = fmaf(f, f, a2);
          a3 = fmaf(w, w, a3);
          a4 = fmaf(f, w, a4);
        }
        sx[0][ry][tx] = a0;
        sx[1][ry][tx] = a1;
        sx[2][ry][tx] = a2;
        sx[3][ry][tx] = a3;
        sx[4][ry][tx] = a4;
      }
      __syncthreads();
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < WW; ++k) a += sx[m][ty + k][tx];
        ring[m][j] = a;
      }
      if (it >= 2 * R) {
        const int cz = zin - 2 * R;
        float S[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
          float a = 0.f;
#pragma unroll
          for (int k = 0; k < WW; ++k) a += ring[m][k];
          S[m] = a;
        }
        float c0 = 0.f, c1 = 0.f, c2 = 0.f, val = 0.f;
        if (cx <= mx && cy <= my && cz <= mz) {
          const float Sff = fmaxf(S[2] - S[0] * S[0] * inv_nw, 0.f);
          const float Sww = fmaxf(S[3] - S[1] * S[1] * inv_nw, 0.f);
          const float Sfw = S[4] - S[0] * S[1] * inv_nw;
          const float muF = S[0] * inv_nw + shF, muW = S[1] * inv_nw + shW;
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
        if (cx < n.n2 && cy < n.n1) {
          const size_t o = ((size_t)cz * n.n1 + cy) * n.n2 + cx;
          C[o] = c0;
          C[cstride + o] = c1;
          if (NC == 3) C[2 * cstride + o] = c2;
        }
      }
    }
  }
  const double s = block_sum((double)lsum - (double)lcomp, sh);
  if (threadIdx.x == 0) part[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
}

// ---- windowed similarity, adjoint: dL/dW(p) = scale * (W(p) sum A - F(p) sum B - sum C)
// over the windows containing p (corners p - 2R .. p); for SiLNCC sum A = number
// of valid windows containing p (times the 2/|R| folded into scale).
template <int R, int KIND>
__global__ void __launch_bounds__(kThreads) k_sim_bwd(const PairDesc* __restrict__ pd, const float* __restrict__ Wb,
                                                      size_t Wstride, const float* __restrict__ coef, size_t cstride,
                                                      float* __restrict__ dLdW, Dims n, float scale, int tz, int nzc) {
  constexpr int WW = 2 * R + 1, RX = TX + 2 * R, RY = TY + 2 * R;
  constexpr int NC = KIND == 0 ? 2 : 3;
  __shared__ float sc[NC][RY][RX];
  __shared__ float sx[NC][RY][TX];
  const int pair = blockIdx.z / nzc, zc = blockIdx.z - pair * nzc;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = zc * tz;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const float* __restrict__ F = pd[pair].Ii;
  const float* __restrict__ W = Wb + (size_t)pair * Wstride;
  const float* __restrict__ C = coef + (size_t)pair * NC * cstride;
  float* __restrict__ out = dLdW + (size_t)pair * Wstride;
  const int px = x0 + tx, py = y0 + ty;
  const int mx = n.n2 - WW, my = n.n1 - WW, mz = n.n0 - WW;
  float cnt_xy = 0.f;
  if (KIND == 0) {
    const int cxn = max(0, min(px, mx) - max(0, px - 2 * R) + 1);
    const int cyn = max(0, min(py, my) - max(0, py - 2 * R) + 1);
    cnt_xy = (float)(cxn * cyn);
  }
  float ring[NC][WW];
  const int zend = min(z0 + tz, n.n0);
  const int niter = (zend - z0) + 2 * R;
  for (int base = 0; base < niter; base += WW) {
#pragma unroll
    for (int j = 0; j < WW; ++j) {
      const int it = base + j;
      if (it >= niter) break;
      const int zin = z0 - 2 * R + it;  // corner plane
      for (int e = threadIdx.x; e < RY * RX; e += kThreads) {
        const int ry = e / RX, rx = e - ry * RX;
        const int gy = y0 - 2 * R + ry, gx = x0 - 2 * R + rx;
        const bool ok = zin >= 0 && zin < n.n0 && gy >= 0 && gy < n.n1 && gx >= 0 && gx < n.n2;
        const size_t o = ok ? ((size_t)zin * n.n1 + gy) * n.n2 + gx : 0;
#pragma unroll
        for (int k = 0; k < NC; ++k) sc[k][ry][rx] = ok ? C[k * cstride + o] : 0.f;
      }
      __syncthreads();
      for (int ry = ty; ry < RY; ry += kThreads / 32) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          float a = 0.f;
#pragma unroll
          for (int q = 0; q < WW; ++q) a += sc[k][ry][tx + q];
          sx[k][ry][tx] = a;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        float a = 0.f;
#pragma unroll
        for (int q = 0; q < WW; ++q) a += sx[k][ty + q][tx];
        ring[k][j] = a;
      }
      if (it >= 2 * R) {
        const int pz = zin;
        float S[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          float a = 0.f;
#pragma unroll
          for (int q = 0; q < WW; ++q) a += ring[k][q];
          S[k] = a;
        }
        if (px < n.n2 && py < n.n1) {
          const size_t o = ((size_t)pz * n.n1 + py) * n.n2 + px;
          const float wv = W[o], fv = F[o];
          float g;
          if (KIND == 0) {
            const int czn = max(0, min(pz, mz) - max(0, pz - 2 * R) + 1);
            g = scale * (cnt_xy * (float)czn * wv - fv * S[0] - S[1]);
          } else {
            g = scale * (wv * S[0] - fv * S[1] - S[2]);
          }
          out[o] = g;
        }
      }
    }
  }
}

// ---- warp adjoint fused with the transposed upsample.
// dL/dU~(p) = dL/dW(p) grad S[I_k](p + U~(p)); dL/dU(Y) = 2 sum_p w(Y; q(p)) dL/dU~(p)
// in gather form: a CTA owns a 32 x 8 (W x H) column of flow nodes, streams the
// image planes along D, computes dL/dU~ once per image voxel of its
// (2*32+2) x (2*8+2) halo region, reduces along W and H in shared memory and
// along D in registers. Every flow node is written once: no atomics.
__device__ __forceinline__ float up_weight(int node, int p, int nflow) {
  const Cell c = cell_of(centre(p), nflow);
  return (c.i0 == node ? 1.f - c.t : 0.f) + (c.i1 == node ? c.t : 0.f);
}

__global__ void __launch_bounds__(kThreads) k_warp_bwd(const PairDesc* __restrict__ pd, const float* __restrict__ dLdWb,
                                                       size_t stride, Dims ni, Dims nf, int fz, int nzc) {
  constexpr int RX = 2 * FX + 2, RY = 2 * FY + 2;
  __shared__ float sg[3][RY][RX];
  __shared__ float sgx[3][RY][FX];
  const int pair = blockIdx.z / nzc, zc = blockIdx.z - pair * nzc;
  const PairDesc d = pd[pair];
  const float* __restrict__ dW = dLdWb + (size_t)pair * stride;
  const int X0 = blockIdx.x * FX, Y0 = blockIdx.y * FY, Z0 = zc * fz, Z1 = min(Z0 + fz, nf.n0);
  const int fx = threadIdx.x & 31, fy = threadIdx.x >> 5;
  const int X = X0 + fx, Y = Y0 + fy;
  const int px0 = 2 * X0 - 1, py0 = 2 * Y0 - 1;
  // per-thread weights along W (for its 3 rows of the x-pass) and H
  float wxk[4], wyk[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    wxk[k] = up_weight(X, 2 * X - 1 + k, nf.n2);
    wyk[k] = up_weight(Y, 2 * Y - 1 + k, nf.n1);
  }
  float3 acc0 = make_float3(0.f, 0.f, 0.f), acc1 = make_float3(0.f, 0.f, 0.f);
  int Zb = Z0 - 1;  // acc0 <-> flow plane Zb, acc1 <-> Zb + 1
  const int pz_lo = max(0, 2 * Z0 - 1), pz_hi = min(ni.n0 - 1, 2 * Z1);
  for (int pz = pz_lo; pz <= pz_hi; ++pz) {
    for (int e = threadIdx.x; e < RY * RX; e += kThreads) {
      const int ry = e / RX, rx = e - ry * RX;
      const int py = py0 + ry, px = px0 + rx;
      float g0 = 0.f, g1 = 0.f, g2 = 0.f;
      if (py >= 0 && py < ni.n1 && px >= 0 && px < ni.n2) {
        const size_t o = ((size_t)pz * ni.n1 + py) * ni.n2 + px;
        const float dl = dW[o];
        if (dl != 0.f) {
          const float4 u = sample4(d.U, nf, centre(pz), centre(py), centre(px));
          const float3 gi = sample1_grad(d.Ik, ni, pz + 2.f * u.x, py + 2.f * u.y, px + 2.f * u.z);
          const float s = 2.f * dl;
          g0 = s * gi.x;
          g1 = s * gi.y;
          g2 = s * gi.z;
        }
      }
      sg[0][ry][rx] = g0;
      sg[1][ry][rx] = g1;
      sg[2][ry][rx] = g2;
    }
    __syncthreads();
    for (int ry = fy; ry < RY; ry += kThreads / 32) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) a = fmaf(wxk[k], sg[c][ry][2 * fx + k], a);
        sgx[c][ry][fx] = a;
      }
    }
    __syncthreads();
    float r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float a = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) a = fmaf(wyk[k], sgx[c][2 * fy + k][fx], a);
      r[c] = a;
    }
    const Cell cz = cell_of(centre(pz), nf.n0);
    while (cz.i0 > Zb) {  // flow plane Zb gets no more contributions
      if (Zb >= Z0 && Zb < Z1 && X < nf.n2 && Y < nf.n1)
        d.G[((size_t)Zb * nf.n1 + Y) * nf.n2 + X] = make_float4(acc0.x, acc0.y, acc0.z, 0.f);
      acc0 = acc1;
      acc1 = make_float3(0.f, 0.f, 0.f);
      ++Zb;
    }
    const float w0 = 1.f - cz.t, w1 = cz.t;
    // i0 == Zb here; i1 is Zb or Zb + 1
    acc0.x = fmaf(w0, r[0], acc0.x);
    acc0.y = fmaf(w0, r[1], acc0.y);
    acc0.z = fmaf(w0, r[2], acc0.z);
    if (cz.i1 == Zb) {
      acc0.x = fmaf(w1, r[0], acc0.x);
      acc0.y = fmaf(w1, r[1], acc0.y);
      acc0.z = fmaf(w1, r[2], acc0.z);
    } else {
      acc1.x = fmaf(w1, r[0], acc1.x);
      acc1.y = fmaf(w1, r[1], acc1.y);
      acc1.z = fmaf(w1, r[2], acc1.z);
    }
  }
  // flush the remaining planes of the chunk
  while (Zb < Z1) {
    if (Zb >= Z0 && X < nf.n2 && Y < nf.n1)
      d.G[((size_t)Zb * nf.n1 + Y) * nf.n2 + X] = make_float4(acc0.x, acc0.y, acc0.z, 0.f);
    acc0 = acc1;
    acc1 = make_float3(0.f, 0.f, 0.f);
    ++Zb;
  }
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

template <int KIND>
void sim_fwd_dispatch(int R, dim3 g, const PairDesc* pd, const float* W, size_t Ws, float* coef, size_t cs,
                      double* part, Dims n, float eps, int tz, int nzc, cudaStream_t s) {
  switch (R) {
    case 1: k_sim_fwd<1, KIND><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, part, n, eps, tz, nzc); break;
    case 2: k_sim_fwd<2, KIND><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, part, n, eps, tz, nzc); break;
    case 3: k_sim_fwd<3, KIND><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, part, n, eps, tz, nzc); break;
    case 4: k_sim_fwd<4, KIND><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, part, n, eps, tz, nzc); break;
    case 5: k_sim_fwd<5, KIND><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, part, n, eps, tz, nzc); break;
    default: break;
  }
}
template <int KIND>
void sim_bwd_dispatch(int R, dim3 g, const PairDesc* pd, const float* W, size_t Ws, const float* coef, size_t cs,
                      float* dLdW, Dims n, float scale, int tz, int nzc, cudaStream_t s) {
  switch (R) {
    case 1: k_sim_bwd<1, KIND><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc); break;
    case 2: k_sim_bwd<2, KIND><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc); break;
    case 3: k_sim_bwd<3, KIND><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc); break;
    case 4: k_sim_bwd<4, KIND><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc); break;
    case 5: k_sim_bwd<5, KIND><<<g, kThreads, 0, s>>>(pd, W, Ws, coef, cs, dLdW, n, scale, tz, nzc); break;
    default: break;
  }
}

int chunk_for(int ntiles, int depth, int min_chunk) {
  // split D so that one pair has at least 128 CTAs when the volume allows it
  int tz = depth;
  while (tz > min_chunk && (long)ntiles * ((depth + tz - 1) / tz) < 128) tz = (tz + 1) / 2;
  return tz < 1 ? 1 : tz;
}
}  // namespace

void launch_down2(const float* in, Dims n, float* out, Dims m, int n_images, cudaStream_t s) {
  k_down2<<<dim3(blocks_for(vox(m)), n_images), kThreads, 0, s>>>(in, n, out, m);
}
void launch_warp(const PairDesc* pd, int n_pairs, Dims ni, Dims nf, float* W, size_t Wstride, cudaStream_t s) {
  k_warp<<<dim3(blocks_for(vox(ni)), n_pairs), kThreads, 0, s>>>(pd, ni, nf, W, Wstride);
}
void launch_count_nonfinite(const float* x, size_t n, int* count, cudaStream_t s) {
  const unsigned b = (unsigned)std::min<size_t>((n + kThreads - 1) / kThreads, 152 * 16);
  if (b) k_count_nonfinite<<<b, kThreads, 0, s>>>(x, n, count);
}
void launch_upsample_disp(const float4* U, Dims nf, Dims ni, float* out, cudaStream_t s) {
  k_upsample_disp<<<blocks_for(vox(ni)), kThreads, 0, s>>>(U, nf, ni, out);
}

SimGeom sim_geom(Dims ni) {
  SimGeom g;
  const int gx = (ni.n2 + TX - 1) / TX, gy = (ni.n1 + TY - 1) / TY;
  g.tz = chunk_for(gx * gy, ni.n0, 16);
  g.nzc = (ni.n0 + g.tz - 1) / g.tz;
  g.ctas = gx * gy * g.nzc;
  return g;
}
int sim_ncoef(int kind) { return kind == 0 ? 2 : 3; }

void launch_sim_fwd(const PairDesc* pd, int n_pairs, const float* W, size_t Wstride, float* coef, size_t cs,
                    double* partials, Dims ni, int window, int kind, float eps, cudaStream_t s) {
  const SimGeom g = sim_geom(ni);
  const dim3 grid((ni.n2 + TX - 1) / TX, (ni.n1 + TY - 1) / TY, g.nzc * n_pairs);
  const int R = window / 2;
  if (kind == 0)
    sim_fwd_dispatch<0>(R, grid, pd, W, Wstride, coef, cs, partials, ni, eps, g.tz, g.nzc, s);
  else
    sim_fwd_dispatch<1>(R, grid, pd, W, Wstride, coef, cs, partials, ni, eps, g.tz, g.nzc, s);
}
void launch_sim_bwd(const PairDesc* pd, int n_pairs, const float* W, size_t Wstride, const float* coef, size_t cs,
                    float* dLdW, Dims ni, int window, int kind, float scale, cudaStream_t s) {
  const SimGeom g = sim_geom(ni);
  const dim3 grid((ni.n2 + TX - 1) / TX, (ni.n1 + TY - 1) / TY, g.nzc * n_pairs);
  const int R = window / 2;
  if (kind == 0)
    sim_bwd_dispatch<0>(R, grid, pd, W, Wstride, coef, cs, dLdW, ni, scale, g.tz, g.nzc, s);
  else
    sim_bwd_dispatch<1>(R, grid, pd, W, Wstride, coef, cs, dLdW, ni, scale, g.tz, g.nzc, s);
}
void launch_warp_bwd(const PairDesc* pd, int n_pairs, const float* dLdW, size_t stride, Dims ni, Dims nf,
                     cudaStream_t s) {
  const int gx = (nf.n2 + FX - 1) / FX, gy = (nf.n1 + FY - 1) / FY;
  const int fz = chunk_for(gx * gy, nf.n0, 4);
  const int nzc = (nf.n0 + fz - 1) / fz;
  k_warp_bwd<<<dim3(gx, gy, nzc * n_pairs), kThreads, 0, s>>>(pd, dLdW, stride, ni, nf, fz, nzc);
}
void launch_loss_reduce(const double* sim_part, int n_sim, const double* reg_part, int n_reg, double inv_NR,
                        double inv_F, double inv_Nm2, float a_ss, float a_l2, float a_ts, double* out, double* hist,
                        int* step, int* flag, int advance, cudaStream_t s) {
  k_loss_reduce<<<1, kThreads, 0, s>>>(sim_part, n_sim, reg_part, n_reg, inv_NR, inv_F, inv_Nm2, a_ss, a_l2, a_ts,
                                       out, hist, step, flag, advance);
}

}  // namespace muster
