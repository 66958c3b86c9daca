// warp_kernels.cu -- the trilinear warp I_k o Phi_ki^i with the flow-to-image
// upsample fused in (Sec. Background; flows on the 2x coarser grid of Sec.
// Implementation Details), and its adjoint fused with the transposed upsample.
//
// Both kernels work on 2x2x2 blocks of image voxels: the block at flow node m
// holds image voxels 2m + d, d in {0,1}^3. With voxel-centre alignment
// q = (p + 1/2)/2 - 1/2 and clamp-to-edge sampling, the upsampled displacement
// of image voxel 2m is 0.25 U(m-1) + 0.75 U(m) and of 2m+1 is
// 0.75 U(m) + 0.25 U(m+1) along each axis, with node indices clamped into the
// grid: an exact separable stencil on the 3x3x3 nodes around m (27 vector loads
// per 8 voxels instead of 64). The forward also stores grad I_k at the sample
// point (12 B per voxel), which spares the adjoint the upsample and the 8-corner
// gathers. The adjoint applies the transpose of the stencil, reduced along W with
// warp shuffles, along H in shared memory and along D in registers while
// streaming over D; every flow node is written once. When the image width is a
// multiple of 4 the adjoint's inputs (dL/dW and the three components of grad I_k) are
// staged plane pair by plane pair by the tensor memory accelerator, two stages ahead.
#include <string.h>

#include <mutex>

#include "kernels.h"
#include "tma.cuh"

namespace muster {

namespace {

constexpr int BX = 16, BY = 16;            // forward: threads per CTA in W and H
constexpr int RX = 32, RY = 8;             // adjoint: threads per CTA (W lanes x H)
constexpr int OX = RX - 2, OY = RY - 2;    // adjoint: flow nodes written per CTA
// the staged adjoint's box starts at x = 2 (OX blockIdx.x - 1) - 2, a multiple of 4 floats
// (a tensor copy must start on a 16-byte boundary) only while OX is even
static_assert(OX % 2 == 0, "the staged warp-adjoint box must start at a multiple of 4 floats");

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 comb(float wa, float3 a, float wb, float3 b) {
  return make_float3(fmaf(wa, a.x, wb * b.x), fmaf(wa, a.y, wb * b.y), fmaf(wa, a.z, wb * b.z));
}

// upsampled displacement (image voxels) of the 8 image voxels of block (mz, my, mx)
__device__ __forceinline__ void upsample_block(const float4* __restrict__ U, Dims nf, int mz, int my, int mx,
                                               float3 (&u)[2][2][2]) {
  const int zs[3] = {max(mz - 1, 0), mz, min(mz + 1, nf.n0 - 1)};
  const int ys[3] = {max(my - 1, 0), my, min(my + 1, nf.n1 - 1)};
  const int x0 = max(mx - 1, 0), x2 = min(mx + 1, nf.n2 - 1);
  float3 s[3][2][2];  // [z node][dy][dx] after the W and H passes
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float3 r[3][2];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float4* row = U + (zs[a] * nf.n1 + ys[b]) * nf.n2;
      const float3 A = f3(__ldg(row + x0)), B = f3(__ldg(row + mx)), C = f3(__ldg(row + x2));
      r[b][0] = comb(0.25f, A, 0.75f, B);
      r[b][1] = comb(0.75f, B, 0.25f, C);
    }
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      s[a][0][dx] = comb(0.25f, r[0][dx], 0.75f, r[1][dx]);
      s[a][1][dx] = comb(0.75f, r[1][dx], 0.25f, r[2][dx]);
    }
  }
  // along D, and the factor 2 from flow to image voxel units
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      u[0][dy][dx] = comb(0.5f, s[0][dy][dx], 1.5f, s[1][dy][dx]);
      u[1][dy][dx] = comb(1.5f, s[1][dy][dx], 0.5f, s[2][dy][dx]);
    }
}

// one axis of the image sampling operator: clamp, cell, fraction, stride to the upper node;
// `in` is 1 when q was not clamped (a NaN clamps to 0 and counts as clamped)
struct Ax {
  int i, d;
  float t, in;
};
__device__ __forceinline__ Ax axis(float q, int n, int stride) {
  Ax a;
  const float hi = (float)(n - 1);
  const float c = fminf(fmaxf(q, 0.f), hi);
  a.in = c == q ? 1.f : 0.f;
  const float f = floorf(c);
  a.t = c - f;
  a.i = (int)f;
  a.d = a.i < n - 1 ? stride : 0;
  return a;
}

__device__ __forceinline__ float img_sample(const float* __restrict__ I, Dims n, float qz, float qy, float qx) {
  const Ax z = axis(qz, n.n0, n.n1 * n.n2), y = axis(qy, n.n1, n.n2), x = axis(qx, n.n2, 1);
  const float* p = I + (z.i * n.n1 + y.i) * n.n2 + x.i;
  const float c00 = lerpf(__ldg(p), __ldg(p + x.d), x.t);
  const float c01 = lerpf(__ldg(p + y.d), __ldg(p + y.d + x.d), x.t);
  const float c10 = lerpf(__ldg(p + z.d), __ldg(p + z.d + x.d), x.t);
  const float c11 = lerpf(__ldg(p + z.d + y.d), __ldg(p + z.d + y.d + x.d), x.t);
  return lerpf(lerpf(c00, c01, y.t), lerpf(c10, c11, y.t), z.t);
}


__device__ __forceinline__ float img_sample_grad(const float* __restrict__ I, Dims n, float qz, float qy, float qx,
                                                float3& g) {
  const Ax z = axis(qz, n.n0, n.n1 * n.n2), y = axis(qy, n.n1, n.n2), x = axis(qx, n.n2, 1);
  const float* p = I + (z.i * n.n1 + y.i) * n.n2 + x.i;
  const float v000 = __ldg(p), v001 = __ldg(p + x.d), v010 = __ldg(p + y.d), v011 = __ldg(p + y.d + x.d);
  const float v100 = __ldg(p + z.d), v101 = __ldg(p + z.d + x.d), v110 = __ldg(p + z.d + y.d),
              v111 = __ldg(p + z.d + y.d + x.d);
  const float c00 = lerpf(v000, v001, x.t), c01 = lerpf(v010, v011, x.t);
  const float c10 = lerpf(v100, v101, x.t), c11 = lerpf(v110, v111, x.t);
  const float c0 = lerpf(c00, c01, y.t), c1 = lerpf(c10, c11, y.t);
  g.x = (c1 - c0) * z.in;
  g.y = lerpf(c01 - c00, c11 - c10, z.t) * y.in;
  g.z = lerpf(lerpf(v001 - v000, v011 - v010, y.t), lerpf(v101 - v100, v111 - v110, y.t), z.t) * x.in;
  return lerpf(c0, c1, z.t);
}

// ---- W(p) = S[I_k](p + U~(p)) for every image voxel of the pair batch; with GRAD the
// gradient of the sampled image at the same point (needed by the adjoint) is
// written too, as three planes gI[c * stride + v]
template <bool GRAD, bool RIGID>
__global__ void __launch_bounds__(BX* BY) k_warp2(const PairDesc* __restrict__ pd, Dims ni, Dims nf,
                                                  float* __restrict__ W, float* __restrict__ gI, size_t stride,
                                                  const float* __restrict__ rig) {
  const int pair = blockIdx.z / nf.n0, mz = blockIdx.z - pair * nf.n0;
  const int mx = blockIdx.x * BX + threadIdx.x, my = blockIdx.y * BY + threadIdx.y;
  if (mx >= nf.n2 || my >= nf.n1) return;
  const PairDesc d = pd[pair];
  float3 u[2][2][2];
  upsample_block(d.U, nf, mz, my, mx, u);
  if (RIGID) {
    // Sec. Rigid Registration: the rigid displacement A p + b of the fixed session's grid
    const float* t = rig + 12 * d.fi;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const float pz = (float)(2 * mz + dz), py = (float)(2 * my + dy), px = (float)(2 * mx + dx);
          float3& v = u[dz][dy][dx];
          v.x += fmaf(t[0], pz, fmaf(t[1], py, fmaf(t[2], px, t[9])));
          v.y += fmaf(t[3], pz, fmaf(t[4], py, fmaf(t[5], px, t[10])));
          v.z += fmaf(t[6], pz, fmaf(t[7], py, fmaf(t[8], px, t[11])));
        }
  }
  float* out = W + (size_t)pair * stride;
  float* go = GRAD ? gI + (size_t)pair * 3 * stride : nullptr;
  // both voxels of a W pair in one 8-byte store (even widths and 8-byte aligned outputs:
  // every row, pair and plane offset is then even, so the pair starts on an 8-byte boundary)
  const bool pair_store = (ni.n2 & 1) == 0 && (reinterpret_cast<uintptr_t>(out) & 7) == 0 &&
                          (!GRAD || (reinterpret_cast<uintptr_t>(go) & 7) == 0);
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    const int z = 2 * mz + dz;
    if (z >= ni.n0) continue;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const int y = 2 * my + dy;
      if (y >= ni.n1) continue;
      if (pair_store) {
        const int o = (z * ni.n1 + y) * ni.n2 + 2 * mx;
        const float3 v0 = u[dz][dy][0], v1 = u[dz][dy][1];
        if (GRAD) {
          float3 g0, g1;
          const float w0 = img_sample_grad(d.Ik, ni, z + v0.x, y + v0.y, 2 * mx + v0.z, g0);
          const float w1 = img_sample_grad(d.Ik, ni, z + v1.x, y + v1.y, 2 * mx + 1 + v1.z, g1);
          *reinterpret_cast<float2*>(out + o) = make_float2(w0, w1);
          *reinterpret_cast<float2*>(go + o) = make_float2(g0.x, g1.x);
          *reinterpret_cast<float2*>(go + stride + o) = make_float2(g0.y, g1.y);
          *reinterpret_cast<float2*>(go + 2 * stride + o) = make_float2(g0.z, g1.z);
        } else {
          const float w0 = img_sample(d.Ik, ni, z + v0.x, y + v0.y, 2 * mx + v0.z);
          const float w1 = img_sample(d.Ik, ni, z + v1.x, y + v1.y, 2 * mx + 1 + v1.z);
          *reinterpret_cast<float2*>(out + o) = make_float2(w0, w1);
        }
        continue;
      }
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int x = 2 * mx + dx;
        if (x >= ni.n2) continue;
        const float3 v = u[dz][dy][dx];
        const int o = (z * ni.n1 + y) * ni.n2 + x;
        if (GRAD) {
          float3 g;
          out[o] = img_sample_grad(d.Ik, ni, z + v.x, y + v.y, x + v.z, g);
          go[o] = g.x;
          go[stride + o] = g.y;
          go[2 * stride + o] = g.z;
        } else {
          out[o] = img_sample(d.Ik, ni, z + v.x, y + v.y, x + v.z);
        }
      }
    }
  }
}

// ---- adjoint: g(p) = 2 dL/dW(p) grad S[I_k](p + U~(p)) at every image voxel (the image
// gradient at the sample point was stored by the forward warp), then
// dL/dU(node) = sum over the image voxels of the node's stencil with the same
// 0.25 / 0.75 weights (contributions to clamped node indices fold onto the edge node).
template <bool RIGID>
__global__ void __launch_bounds__(RX* RY) k_warp_bwd2(const PairDesc* __restrict__ pd, const float* __restrict__ dLdWb,
                                                      const float* __restrict__ gIb, size_t stride, Dims ni, Dims nf,
                                                      int fz, int nzc, float* __restrict__ rpart,
                                                      unsigned* __restrict__ gmax) {
  __shared__ float sh[RY][RX][12];
  float gm = 0.f;  // largest |component| of the nodes this thread writes
  // with rpart: sums of dL/dq and dL/dq p^T over the image voxels of the nodes this CTA
  // writes (the rigid gradient, Sec. Rigid Registration), 12 per CTA
  float racc[RIGID ? 12 : 1];
#pragma unroll
  for (int k = 0; k < (RIGID ? 12 : 1); ++k) racc[k] = 0.f;
  const int pair = blockIdx.z / nzc, zc = blockIdx.z - pair * nzc;
  const PairDesc d = pd[pair];
  const float* __restrict__ dW = dLdWb + (size_t)pair * stride;
  const float* __restrict__ gI = gIb + (size_t)pair * 3 * stride;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int mx = blockIdx.x * OX - 1 + lane, my = blockIdx.y * OY - 1 + ty;
  const bool active = mx >= 0 && mx < nf.n2 && my >= 0 && my < nf.n1;
  const bool writer = lane >= 1 && lane <= OX && ty >= 1 && ty <= OY && active;
  const int Z0 = zc * fz, Z1 = min(Z0 + fz, nf.n0);
  // even widths with 8-byte aligned inputs: the two voxels of a W pair start on an
  // 8-byte boundary in every row, pair and plane
  const bool pair_load = (ni.n2 & 1) == 0 && (reinterpret_cast<uintptr_t>(dW) & 7) == 0 &&
                         (reinterpret_cast<uintptr_t>(gI) & 7) == 0 && (stride & 1) == 0;
  float3 pend = make_float3(0.f, 0.f, 0.f), carry = pend;
  for (int mz = max(Z0 - 1, 0); mz <= min(Z1, nf.n0 - 1); ++mz) {
    // per-voxel gradient of the 8 image voxels of block (mz, my, mx)
    float3 g[2][2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c) g[a][b][c] = make_float3(0.f, 0.f, 0.f);
    if (active && pair_load) {
      // the two voxels of a W pair with 8-byte loads
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const int z = 2 * mz + dz, y = 2 * my + dy;
          if (z < ni.n0 && y < ni.n1) {
            const int o = (z * ni.n1 + y) * ni.n2 + 2 * mx;
            const float2 s = *reinterpret_cast<const float2*>(dW + o);
            const float2 a = *reinterpret_cast<const float2*>(gI + o);
            const float2 b = *reinterpret_cast<const float2*>(gI + stride + o);
            const float2 c = *reinterpret_cast<const float2*>(gI + 2 * stride + o);
            g[dz][dy][0] = make_float3(2.f * s.x * a.x, 2.f * s.x * b.x, 2.f * s.x * c.x);
            g[dz][dy][1] = make_float3(2.f * s.y * a.y, 2.f * s.y * b.y, 2.f * s.y * c.y);
          }
        }
    } else if (active) {
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const int z = 2 * mz + dz, y = 2 * my + dy, x = 2 * mx + dx;
            if (z < ni.n0 && y < ni.n1 && x < ni.n2) {
              const int o = (z * ni.n1 + y) * ni.n2 + x;
              const float s = 2.f * dW[o];
              g[dz][dy][dx] = make_float3(s * gI[o], s * gI[stride + o], s * gI[2 * stride + o]);
            }
          }
    }
    if (RIGID && writer && mz >= Z0 && mz < Z1) {
      // g holds 2 dL/dq (the 2 of the flow-to-image scale); image voxels outside the
      // grid were left at 0
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const float3 q = g[dz][dy][dx];
            const float gx = 0.5f * q.x, gy = 0.5f * q.y, gz = 0.5f * q.z;
            const float pz = (float)(2 * mz + dz), py = (float)(2 * my + dy), px = (float)(2 * mx + dx);
            float* r = racc;
            r[0] += gx, r[1 % (RIGID ? 12 : 1)] += gy, r[2 % (RIGID ? 12 : 1)] += gz;
            if (RIGID) {
              r[3] += gx * pz, r[4] += gx * py, r[5] += gx * px;
              r[6] += gy * pz, r[7] += gy * py, r[8] += gy * px;
              r[9] += gz * pz, r[10] += gz * py, r[11] += gz * px;
            }
          }
    }
    // transpose along W: node mx gets 0.75 (g0 + g1) of its block, 0.25 g1 of block mx-1
    // and 0.25 g0 of block mx+1 (neighbouring lanes); edge nodes keep their folded share
    float hx[2][2][3];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const float3 g0 = g[dz][dy][0], g1 = g[dz][dy][1];
        const float e0 = (mx == 0) ? 0.25f : 0.f, e1 = (mx == nf.n2 - 1) ? 0.25f : 0.f;
        const float a0[3] = {g0.x, g0.y, g0.z}, a1[3] = {g1.x, g1.y, g1.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float left = __shfl_up_sync(0xffffffffu, a1[c], 1);
          const float right = __shfl_down_sync(0xffffffffu, a0[c], 1);
          hx[dz][dy][c] = 0.75f * (a0[c] + a1[c]) + 0.25f * (left + right) + e0 * a0[c] + e1 * a1[c];
        }
      }
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int c = 0; c < 3; ++c) sh[ty][lane][(dz * 2 + dy) * 3 + c] = hx[dz][dy][c];
    __syncthreads();
    // transpose along H (neighbouring rows in shared memory)
    float k[2][3];
    {
      const int up = max(ty - 1, 0), dn = min(ty + 1, RY - 1);
      const float e0 = (my == 0) ? 0.25f : 0.f, e1 = (my == nf.n1 - 1) ? 0.25f : 0.f;
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float h0 = hx[dz][0][c], h1 = hx[dz][1][c];
          const float l = ty > 0 ? sh[up][lane][(dz * 2 + 1) * 3 + c] : 0.f;
          const float r = ty < RY - 1 ? sh[dn][lane][(dz * 2 + 0) * 3 + c] : 0.f;
          k[dz][c] = 0.75f * (h0 + h1) + 0.25f * (l + r) + e0 * h0 + e1 * h1;
        }
    }
    __syncthreads();
    // transpose along D, streaming: node mz-1 is complete once block mz added its 0.25 k0
    const float3 k0 = make_float3(k[0][0], k[0][1], k[0][2]), k1 = make_float3(k[1][0], k[1][1], k[1][2]);
    if (mz - 1 >= Z0 && mz - 1 < Z1 && writer)
    {
      const float4 gv = make_float4(pend.x + 0.25f * k0.x, pend.y + 0.25f * k0.y, pend.z + 0.25f * k0.z, 0.f);
      d.G[((mz - 1) * nf.n1 + my) * nf.n2 + mx] = gv;
      gm = fmaxf(gm, fmaxf(fabsf(gv.x), fmaxf(fabsf(gv.y), fabsf(gv.z))));
    }
    const float e0 = (mz == 0) ? 0.25f : 0.f, e1 = (mz == nf.n0 - 1) ? 0.25f : 0.f;
    pend.x = 0.75f * (k0.x + k1.x) + carry.x + e0 * k0.x + e1 * k1.x;
    pend.y = 0.75f * (k0.y + k1.y) + carry.y + e0 * k0.y + e1 * k1.y;
    pend.z = 0.75f * (k0.z + k1.z) + carry.z + e0 * k0.z + e1 * k1.z;
    carry = make_float3(0.25f * k1.x, 0.25f * k1.y, 0.25f * k1.z);
  }
  // the last node of the volume has no block after it
  if (Z1 == nf.n0 && writer) {
    d.G[((nf.n0 - 1) * nf.n1 + my) * nf.n2 + mx] = make_float4(pend.x, pend.y, pend.z, 0.f);
    gm = fmaxf(gm, fmaxf(fabsf(pend.x), fmaxf(fabsf(pend.y), fabsf(pend.z))));
  }
  if (gmax) {  // the scale of the deterministic adjoint's fixed-point sums
    const unsigned b = __reduce_max_sync(0xffffffffu, __float_as_uint(gm));
    if ((threadIdx.x & 31) == 0 && b) atomicMax(gmax, b);
  }
  if (RIGID) {
    // CTA sums in a fixed order: warp shuffles, then the warps in order (through sh)
    __syncthreads();
    float* red = &sh[0][0][0];
    const int tid = ty * RX + lane, w = tid >> 5;
#pragma unroll
    for (int k = 0; k < (RIGID ? 12 : 1); ++k) {
      float v = racc[k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[w * 12 + k] = v;
    }
    __syncthreads();
    if (tid < 12) {
      float t = 0.f;
      for (int i = 0; i < RX * RY / 32; ++i) t += red[i * 12 + tid];
      const int per_pair = gridDim.x * gridDim.y * nzc;
      const int cta = (zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      rpart[((size_t)pair * per_pair + cta) * 12 + tid] = t;
    }
  }
}

// ---- the same adjoint with its inputs staged by the tensor memory accelerator. Per flow
// plane mz one thread copies the 2 image planes 2mz, 2mz+1 of the CTA's region (16 rows,
// 68 columns from a 16-byte aligned start: the 64 columns of the 32 node columns and 4 of
// alignment) of dL/dW and of each component of grad I_k into one of two stages; the copy
// of plane mz+2 is issued once every thread has read plane mz. Voxels outside the image
// arrive as zeros, as the plain loads of k_warp_bwd2 leave them. A wait that runs out sets
// *err and the CTA carries on without waiting (its results are reported as invalid).
constexpr int SXW = 2 * RX + 4, SYH = 2 * RY, SZD = 2;  // staged box: columns, rows, planes
constexpr int SARR = SZD * SYH * SXW;                    // floats of one array in one stage

template <bool RIGID>
__global__ void __launch_bounds__(RX* RY) k_warp_bwd3t(const __grid_constant__ WarpBwdMaps maps,
                                                       const PairDesc* __restrict__ pd, Dims ni, Dims nf, int fz,
                                                       int nzc, float* __restrict__ rpart, int* __restrict__ err,
                                                       unsigned* __restrict__ gmax) {
  float gm = 0.f;  // largest |component| of the nodes this thread writes
  __shared__ __align__(8) uint64_t bar[2];
  extern __shared__ __align__(128) float smem_raw[];
  float* stage = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  // the H transpose's exchange buffer [RY][RX][12] lives in the stage just read (its next
  // copy is issued once the exchange is done), which leaves room for 3 CTAs per SM
  typedef float ShRow[RX][12];
  static_assert(RY * RX * 12 <= 4 * SARR, "exchange buffer larger than a stage");
  float racc[RIGID ? 12 : 1];
#pragma unroll
  for (int k = 0; k < (RIGID ? 12 : 1); ++k) racc[k] = 0.f;
  const int pair = blockIdx.z / nzc, zc = blockIdx.z - pair * nzc;
  const PairDesc d = pd[pair];
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * RX + lane;
  const int mx = blockIdx.x * OX - 1 + lane, my = blockIdx.y * OY - 1 + ty;
  const bool writer = lane >= 1 && lane <= OX && ty >= 1 && ty <= OY && mx >= 0 && mx < nf.n2 && my >= 0 &&
                      my < nf.n1;
  const int Z0 = zc * fz, Z1 = min(Z0 + fz, nf.n0);
  const int m0 = max(Z0 - 1, 0), m1 = min(Z1, nf.n0 - 1), niter = m1 - m0 + 1;
  const int xs = 2 * (blockIdx.x * OX - 1) - 2, ys = 2 * (blockIdx.y * OY - 1);  // xs: multiple of 4
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int k) {  // one thread: flow plane m0 + k into stage k & 1
    const int st = k & 1, zs = 2 * (m0 + k);
    float* dst = stage + st * 4 * SARR;
    mbar_expect_tx(&bar[st], 4u * SARR * 4u);
    tma_load4(dst, &maps.dW, xs, ys, zs, pair, &bar[st]);
#pragma unroll
    for (int c = 0; c < 3; ++c) tma_load4(dst + (1 + c) * SARR, &maps.gI, xs, ys, zs, 3 * pair + c, &bar[st]);
  };
  if (tid == 0) {
    issue(0);
    if (niter > 1) issue(1);
  }
  float3 pend = make_float3(0.f, 0.f, 0.f), carry = pend;
  bool ok = true;
  for (int k = 0; k < niter; ++k) {
    const int mz = m0 + k, st = k & 1;
    ok = ok && mbar_wait(&bar[st], (unsigned)(k >> 1) & 1u);  // after a failure, stop waiting
    const float* sd = stage + st * 4 * SARR;
    ShRow* sh = reinterpret_cast<ShRow*>(stage + st * 4 * SARR);
    // per-voxel gradient of the 8 image voxels of block (mz, my, mx)
    float3 g[2][2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int o = (dz * SYH + 2 * ty + dy) * SXW + 2 + 2 * lane;
        const float2 sv = *reinterpret_cast<const float2*>(sd + o);
        const float2 a = *reinterpret_cast<const float2*>(sd + SARR + o);
        const float2 b = *reinterpret_cast<const float2*>(sd + 2 * SARR + o);
        const float2 c = *reinterpret_cast<const float2*>(sd + 3 * SARR + o);
        g[dz][dy][0] = make_float3(2.f * sv.x * a.x, 2.f * sv.x * b.x, 2.f * sv.x * c.x);
        g[dz][dy][1] = make_float3(2.f * sv.y * a.y, 2.f * sv.y * b.y, 2.f * sv.y * c.y);
      }
    if (RIGID && writer && mz >= Z0 && mz < Z1) {
      // g holds 2 dL/dq (the 2 of the flow-to-image scale); image voxels outside the
      // grid arrived as 0
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const float3 q = g[dz][dy][dx];
            const float gx = 0.5f * q.x, gy = 0.5f * q.y, gz = 0.5f * q.z;
            const float pz = (float)(2 * mz + dz), py = (float)(2 * my + dy), px = (float)(2 * mx + dx);
            float* r = racc;
            r[0] += gx, r[1 % (RIGID ? 12 : 1)] += gy, r[2 % (RIGID ? 12 : 1)] += gz;
            if (RIGID) {
              r[3] += gx * pz, r[4] += gx * py, r[5] += gx * px;
              r[6] += gy * pz, r[7] += gy * py, r[8] += gy * px;
              r[9] += gz * pz, r[10] += gz * py, r[11] += gz * px;
            }
          }
    }
    // transpose along W (neighbouring lanes), as in k_warp_bwd2
    float hx[2][2][3];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const float3 g0 = g[dz][dy][0], g1 = g[dz][dy][1];
        const float e0 = (mx == 0) ? 0.25f : 0.f, e1 = (mx == nf.n2 - 1) ? 0.25f : 0.f;
        const float a0[3] = {g0.x, g0.y, g0.z}, a1[3] = {g1.x, g1.y, g1.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float left = __shfl_up_sync(0xffffffffu, a1[c], 1);
          const float right = __shfl_down_sync(0xffffffffu, a0[c], 1);
          hx[dz][dy][c] = 0.75f * (a0[c] + a1[c]) + 0.25f * (left + right) + e0 * a0[c] + e1 * a1[c];
        }
      }
    __syncthreads();  // every thread is past its reads of stage st, which now takes the exchange
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int c = 0; c < 3; ++c) sh[ty][lane][(dz * 2 + dy) * 3 + c] = hx[dz][dy][c];
    __syncthreads();
    // transpose along H (neighbouring rows in shared memory)
    float kk[2][3];
    {
      const int up = max(ty - 1, 0), dn = min(ty + 1, RY - 1);
      const float e0 = (my == 0) ? 0.25f : 0.f, e1 = (my == nf.n1 - 1) ? 0.25f : 0.f;
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float h0 = hx[dz][0][c], h1 = hx[dz][1][c];
          const float l = ty > 0 ? sh[up][lane][(dz * 2 + 1) * 3 + c] : 0.f;
          const float r = ty < RY - 1 ? sh[dn][lane][(dz * 2 + 0) * 3 + c] : 0.f;
          kk[dz][c] = 0.75f * (h0 + h1) + 0.25f * (l + r) + e0 * h0 + e1 * h1;
        }
    }
    // the exchange is read: refill stage st with plane k + 2 (every thread orders its generic
    // accesses of the stage before the copy engine's writes)
    fence_proxy_async();
    __syncthreads();
    if (tid == 0 && k + 2 < niter) issue(k + 2);
    // transpose along D, streaming: node mz-1 is complete once block mz added its 0.25 k0
    const float3 k0 = make_float3(kk[0][0], kk[0][1], kk[0][2]), k1 = make_float3(kk[1][0], kk[1][1], kk[1][2]);
    if (mz - 1 >= Z0 && mz - 1 < Z1 && writer)
    {
      const float4 gv = make_float4(pend.x + 0.25f * k0.x, pend.y + 0.25f * k0.y, pend.z + 0.25f * k0.z, 0.f);
      d.G[((mz - 1) * nf.n1 + my) * nf.n2 + mx] = gv;
      gm = fmaxf(gm, fmaxf(fabsf(gv.x), fmaxf(fabsf(gv.y), fabsf(gv.z))));
    }
    const float e0 = (mz == 0) ? 0.25f : 0.f, e1 = (mz == nf.n0 - 1) ? 0.25f : 0.f;
    pend.x = 0.75f * (k0.x + k1.x) + carry.x + e0 * k0.x + e1 * k1.x;
    pend.y = 0.75f * (k0.y + k1.y) + carry.y + e0 * k0.y + e1 * k1.y;
    pend.z = 0.75f * (k0.z + k1.z) + carry.z + e0 * k0.z + e1 * k1.z;
    carry = make_float3(0.25f * k1.x, 0.25f * k1.y, 0.25f * k1.z);
  }
  if (Z1 == nf.n0 && writer) {
    d.G[((nf.n0 - 1) * nf.n1 + my) * nf.n2 + mx] = make_float4(pend.x, pend.y, pend.z, 0.f);
    gm = fmaxf(gm, fmaxf(fabsf(pend.x), fmaxf(fabsf(pend.y), fabsf(pend.z))));
  }
  if (gmax) {  // the scale of the deterministic adjoint's fixed-point sums
    const unsigned b = __reduce_max_sync(0xffffffffu, __float_as_uint(gm));
    if ((threadIdx.x & 31) == 0 && b) atomicMax(gmax, b);
  }
  if (!ok) {
    // report, then give the copies still in flight into this CTA's stages one more bounded
    // wait (the last use of each stage) before the CTA's shared memory is released
    if (err) atomicOr(err, 1);
    for (int st = 0; st < 2 && st < niter; ++st) {
      const int last = niter - 1 - ((niter - 1 - st) & 1);
      mbar_wait(&bar[st], (unsigned)(last >> 1) & 1u);
    }
  }
  if (RIGID) {
    __syncthreads();
    float* red = stage;  // every copy into the stages has been waited for
    const int w = tid >> 5;
#pragma unroll
    for (int k = 0; k < (RIGID ? 12 : 1); ++k) {
      float v = racc[k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[w * 12 + k] = v;
    }
    __syncthreads();
    if (tid < 12) {
      float t = 0.f;
      for (int i = 0; i < RX * RY / 32; ++i) t += red[i * 12 + tid];
      const int per_pair = gridDim.x * gridDim.y * nzc;
      const int cta = (zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      rpart[((size_t)pair * per_pair + cta) * 12 + tid] = t;
    }
  }
}
constexpr size_t kWarpBwd3tBytes = 128 + sizeof(float) * 2 * 4 * SARR;

// flow planes per D chunk of the adjoint: every chunk streams two planes more than it
// writes, so chunks are split only until a launch of `batch` pairs has about four waves of
// four CTAs on each of 152 SMs (2432 CTAs), and halved only while above 4 planes
int chunk_nodes(int ntiles, int depth, int batch) {
  int fz = depth;
  while (fz > 4 && (long)batch * ntiles * ((depth + fz - 1) / fz) < 2432) fz = (fz + 1) / 2;
  return fz < 1 ? 1 : fz;
}
}  // namespace

void launch_warp(const PairDesc* pd, int n_pairs, Dims ni, Dims nf, float* W, float* gI, size_t Wstride,
                 const float* rigid, cudaStream_t s) {
  const dim3 grid((nf.n2 + BX - 1) / BX, (nf.n1 + BY - 1) / BY, nf.n0 * n_pairs);
  const dim3 b(BX, BY);
  if (gI) {
    if (rigid)
      k_warp2<true, true><<<grid, b, 0, s>>>(pd, ni, nf, W, gI, Wstride, rigid);
    else
      k_warp2<true, false><<<grid, b, 0, s>>>(pd, ni, nf, W, gI, Wstride, nullptr);
  } else {
    if (rigid)
      k_warp2<false, true><<<grid, b, 0, s>>>(pd, ni, nf, W, nullptr, Wstride, rigid);
    else
      k_warp2<false, false><<<grid, b, 0, s>>>(pd, ni, nf, W, nullptr, Wstride, nullptr);
  }
}

int warp_bwd_ctas_per_pair(Dims nf, int batch) {
  const int gx = (nf.n2 + OX - 1) / OX, gy = (nf.n1 + OY - 1) / OY;
  const int fz = chunk_nodes(gx * gy, nf.n0, batch);
  return gx * gy * ((nf.n0 + fz - 1) / fz);
}
int warp_bwd_zchunks(Dims nf, int batch) {
  const int gx = (nf.n2 + OX - 1) / OX, gy = (nf.n1 + OY - 1) / OY;
  const int fz = chunk_nodes(gx * gy, nf.n0, batch);
  return (nf.n0 + fz - 1) / fz;
}

void make_warp_bwd_maps(WarpBwdMaps* m, const float* dLdW, const float* gI, int batch, Dims ni) {
  memset(m, 0, sizeof(*m));
  m->ok = encode_volumes(&m->dW, dLdW, ni, batch, SXW, SYH, SZD) &&
          encode_volumes(&m->gI, gI, ni, 3 * batch, SXW, SYH, SZD);
}

cudaError_t prepare_warp_kernels() {
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  return once_per_device(done, mu, [] {
    const cudaError_t a =
        cudaFuncSetAttribute(k_warp_bwd3t<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWarpBwd3tBytes);
    const cudaError_t b =
        cudaFuncSetAttribute(k_warp_bwd3t<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWarpBwd3tBytes);
    return a != cudaSuccess ? a : b;
  });
}

void launch_warp_bwd(const PairDesc* pd, int n_pairs, int batch, const float* dLdW, const float* gI, size_t stride,
                     Dims ni, Dims nf, float* rigid_part, const WarpBwdMaps* maps, int* err, unsigned* gmax,
                     cudaStream_t s) {
  const int gx = (nf.n2 + OX - 1) / OX, gy = (nf.n1 + OY - 1) / OY;
  const int fz = chunk_nodes(gx * gy, nf.n0, batch);
  const int nzc = (nf.n0 + fz - 1) / fz;
  const dim3 g(gx, gy, nzc * n_pairs), b(RX, RY);
  if (maps && maps->ok && stride == vox(ni)) {
    if (rigid_part)
      k_warp_bwd3t<true><<<g, b, kWarpBwd3tBytes, s>>>(*maps, pd, ni, nf, fz, nzc, rigid_part, err, gmax);
    else
      k_warp_bwd3t<false><<<g, b, kWarpBwd3tBytes, s>>>(*maps, pd, ni, nf, fz, nzc, nullptr, err, gmax);
    return;
  }
  if (rigid_part)
    k_warp_bwd2<true><<<g, b, 0, s>>>(pd, dLdW, gI, stride, ni, nf, fz, nzc, rigid_part, gmax);
  else
    k_warp_bwd2<false><<<g, b, 0, s>>>(pd, dLdW, gI, stride, ni, nf, fz, nzc, nullptr, gmax);
}

}  // namespace muster
