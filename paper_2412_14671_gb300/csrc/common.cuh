// common.cuh -- device helpers shared by the MUSTER kernels: grid dims, the
// trilinear sampling operator with clamp-to-edge, its derivative and its
// transpose (scatter).
//
// Sampling convention (used by every kernel that interpolates): index
// coordinates with voxel centres at integers; each coordinate q is clamped to
// [0, n-1]; the cell is floor(q_clamped) .. min(floor+1, n-1); weights are
// trilinear; the derivative with respect to q uses that cell and is zero along
// an axis whose coordinate was clamped. The paper states only "trilinear
// interpolation" (Eq. cum_deformation) and prefers the displacement form of
// Alg. 1 "due to boundary effects"; clamp-to-edge makes a constant velocity
// exponentiate to an exact translation.
//
// Vector fields on the flow grid are stored interleaved as float4
// {axis0 (D), axis1 (H), axis2 (W), 0}: one 16-byte load per trilinear corner and
// one vector reduction (red.global.add.v4.f32) per scattered corner.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace muster {

struct Dims {
  int n0, n1, n2;  // D (slowest), H, W (contiguous)
};

__host__ __device__ inline size_t vox(Dims d) { return (size_t)d.n0 * d.n1 * d.n2; }

struct Cell {
  int i0, i1;
  float t;   // fractional position in the cell
  float in;  // 1 if q was inside [0, n-1], else 0 (clamped)
};

__device__ __forceinline__ Cell cell_of(float q, int n) {
  Cell c;
  const float hi = (float)(n - 1);
  c.in = (q >= 0.f && q <= hi) ? 1.f : 0.f;
  const float qc = fminf(fmaxf(q, 0.f), hi);  // NaN -> 0
  const float f = floorf(qc);
  c.i0 = (int)f;
  c.i1 = min(c.i0 + 1, n - 1);
  c.t = qc - f;
  return c;
}

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, 0.f);
}
__device__ __forceinline__ float4 f4sub(float4 a, float4 b) {
  return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, 0.f);
}
__device__ __forceinline__ float4 f4scale(float4 a, float s) {
  return make_float4(a.x * s, a.y * s, a.z * s, 0.f);
}
__device__ __forceinline__ float4 f4lerp(float4 a, float4 b, float t) {
  return make_float4(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y), fmaf(t, b.z - a.z, a.z), 0.f);
}
__device__ __forceinline__ float f4dot3(float4 a, float4 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}
__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

// Corner offsets of the cell containing q (row-major within the volume).
struct Corners {
  int o000, o001, o010, o011, o100, o101, o110, o111;
  float t0, t1, t2, in0, in1, in2;
};

__device__ __forceinline__ Corners corners_of(Dims n, float q0, float q1, float q2) {
  const Cell a = cell_of(q0, n.n0), b = cell_of(q1, n.n1), c = cell_of(q2, n.n2);
  Corners k;
  const int r00 = (a.i0 * n.n1 + b.i0) * n.n2, r01 = (a.i0 * n.n1 + b.i1) * n.n2;
  const int r10 = (a.i1 * n.n1 + b.i0) * n.n2, r11 = (a.i1 * n.n1 + b.i1) * n.n2;
  k.o000 = r00 + c.i0;
  k.o001 = r00 + c.i1;
  k.o010 = r01 + c.i0;
  k.o011 = r01 + c.i1;
  k.o100 = r10 + c.i0;
  k.o101 = r10 + c.i1;
  k.o110 = r11 + c.i0;
  k.o111 = r11 + c.i1;
  k.t0 = a.t;
  k.t1 = b.t;
  k.t2 = c.t;
  k.in0 = a.in;
  k.in1 = b.in;
  k.in2 = c.in;
  return k;
}

// S[g](q) for a float4 vector field
__device__ __forceinline__ float4 sample4(const float4* __restrict__ g, Dims n, float q0, float q1,
                                          float q2) {
  const Corners k = corners_of(n, q0, q1, q2);
  const float4 c00 = f4lerp(__ldg(g + k.o000), __ldg(g + k.o001), k.t2);
  const float4 c01 = f4lerp(__ldg(g + k.o010), __ldg(g + k.o011), k.t2);
  const float4 c10 = f4lerp(__ldg(g + k.o100), __ldg(g + k.o101), k.t2);
  const float4 c11 = f4lerp(__ldg(g + k.o110), __ldg(g + k.o111), k.t2);
  return f4lerp(f4lerp(c00, c01, k.t1), f4lerp(c10, c11, k.t1), k.t0);
}

// S[g](q) and its partial derivatives d/dq_a (each a float4 over components)
struct Samp4 {
  float4 v, d0, d1, d2;
};

__device__ __forceinline__ Samp4 sample4_grad(const float4* __restrict__ g, Dims n, float q0,
                                              float q1, float q2, Corners* out_k = nullptr) {
  const Corners k = corners_of(n, q0, q1, q2);
  const float4 v000 = __ldg(g + k.o000), v001 = __ldg(g + k.o001), v010 = __ldg(g + k.o010),
               v011 = __ldg(g + k.o011), v100 = __ldg(g + k.o100), v101 = __ldg(g + k.o101),
               v110 = __ldg(g + k.o110), v111 = __ldg(g + k.o111);
  // along axis 2 (W)
  const float4 c00 = f4lerp(v000, v001, k.t2), c01 = f4lerp(v010, v011, k.t2);
  const float4 c10 = f4lerp(v100, v101, k.t2), c11 = f4lerp(v110, v111, k.t2);
  const float4 x00 = f4sub(v001, v000), x01 = f4sub(v011, v010);
  const float4 x10 = f4sub(v101, v100), x11 = f4sub(v111, v110);
  // along axis 1 (H)
  const float4 c0 = f4lerp(c00, c01, k.t1), c1 = f4lerp(c10, c11, k.t1);
  const float4 y0 = f4sub(c01, c00), y1 = f4sub(c11, c10);
  const float4 x0 = f4lerp(x00, x01, k.t1), x1 = f4lerp(x10, x11, k.t1);
  Samp4 s;
  s.v = f4lerp(c0, c1, k.t0);
  s.d0 = f4scale(f4sub(c1, c0), k.in0);
  s.d1 = f4scale(f4lerp(y0, y1, k.t0), k.in1);
  s.d2 = f4scale(f4lerp(x0, x1, k.t0), k.in2);
  if (out_k) *out_k = k;
  return s;
}

// S[I](q) for a scalar image, optionally with d/dq
__device__ __forceinline__ float sample1(const float* __restrict__ g, Dims n, float q0, float q1,
                                         float q2) {
  const Corners k = corners_of(n, q0, q1, q2);
  const float c00 = lerpf(__ldg(g + k.o000), __ldg(g + k.o001), k.t2);
  const float c01 = lerpf(__ldg(g + k.o010), __ldg(g + k.o011), k.t2);
  const float c10 = lerpf(__ldg(g + k.o100), __ldg(g + k.o101), k.t2);
  const float c11 = lerpf(__ldg(g + k.o110), __ldg(g + k.o111), k.t2);
  return lerpf(lerpf(c00, c01, k.t1), lerpf(c10, c11, k.t1), k.t0);
}

__device__ __forceinline__ float3 sample1_grad(const float* __restrict__ g, Dims n, float q0,
                                               float q1, float q2) {
  const Corners k = corners_of(n, q0, q1, q2);
  const float v000 = __ldg(g + k.o000), v001 = __ldg(g + k.o001), v010 = __ldg(g + k.o010),
              v011 = __ldg(g + k.o011), v100 = __ldg(g + k.o100), v101 = __ldg(g + k.o101),
              v110 = __ldg(g + k.o110), v111 = __ldg(g + k.o111);
  const float c00 = lerpf(v000, v001, k.t2), c01 = lerpf(v010, v011, k.t2);
  const float c10 = lerpf(v100, v101, k.t2), c11 = lerpf(v110, v111, k.t2);
  const float x0 = lerpf(v001 - v000, v011 - v010, k.t1);
  const float x1 = lerpf(v101 - v100, v111 - v110, k.t1);
  const float c0 = lerpf(c00, c01, k.t1), c1 = lerpf(c10, c11, k.t1);
  float3 d;
  d.x = (c1 - c0) * k.in0;
  d.y = lerpf(c01 - c00, c11 - c10, k.t0) * k.in1;
  d.z = lerpf(x0, x1, k.t0) * k.in2;
  return d;
}

// vector reduction into global memory (red.global.add.v4.f32 on sm_90+)
__device__ __forceinline__ void red4(float4* addr, float4 v) { atomicAdd(addr, v); }

// transpose of sample4 with respect to the sampled values: g[corner] += w * v
__device__ __forceinline__ void scatter4(float4* g, const Corners& k, float4 v) {
  const float a1 = k.t0, a0 = 1.f - k.t0, b1 = k.t1, b0 = 1.f - k.t1, c1 = k.t2, c0 = 1.f - k.t2;
  red4(g + k.o000, f4scale(v, a0 * b0 * c0));
  red4(g + k.o001, f4scale(v, a0 * b0 * c1));
  red4(g + k.o010, f4scale(v, a0 * b1 * c0));
  red4(g + k.o011, f4scale(v, a0 * b1 * c1));
  red4(g + k.o100, f4scale(v, a1 * b0 * c0));
  red4(g + k.o101, f4scale(v, a1 * b0 * c1));
  red4(g + k.o110, f4scale(v, a1 * b1 * c0));
  red4(g + k.o111, f4scale(v, a1 * b1 * c1));
}

// scatter4 with W-neighbours merged across a warp: when lane L+1 samples the cell next to
// lane L's along W, lane L's corners at x+1 (o001, o011, o101, o111) are lane L+1's
// corners at x (o000, o010, o100, o110); lane L+1 then adds lane L's share to its own
// before one reduction and lane L skips those corners. Both lanes decide from the same
// comparison of corner offsets, so any geometry (row ends, clamped edges, folds) is
// handled exactly. Every lane of the warp must call it; valid = false contributes nothing.
__device__ __forceinline__ void scatter4_merged(float4* g, const Corners& k, float4 v, bool valid) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const float a1 = k.t0, a0 = 1.f - k.t0, b1 = k.t1, b0 = 1.f - k.t1, c1 = k.t2, c0 = 1.f - k.t2;
  const float w0[4] = {a0 * b0 * c0, a0 * b1 * c0, a1 * b0 * c0, a1 * b1 * c0};
  const float w1[4] = {a0 * b0 * c1, a0 * b1 * c1, a1 * b0 * c1, a1 * b1 * c1};
  const int o0[4] = {valid ? k.o000 : -1, valid ? k.o010 : -1, valid ? k.o100 : -1, valid ? k.o110 : -1};
  const int o1[4] = {valid ? k.o001 : -1, valid ? k.o011 : -1, valid ? k.o101 : -1, valid ? k.o111 : -1};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float4 own = f4scale(v, w0[e]);
    const float4 mine1 = f4scale(v, w1[e]);
    // the left neighbour's x+1 corner e, if it is my x corner e
    const int lo = __shfl_up_sync(full, o1[e], 1);
    const float lx = __shfl_up_sync(full, mine1.x, 1), ly = __shfl_up_sync(full, mine1.y, 1),
                lz = __shfl_up_sync(full, mine1.z, 1);
    if (lane > 0 && lo >= 0 && lo == o0[e]) {
      own.x += lx;
      own.y += ly;
      own.z += lz;
    }
    // my x+1 corner e is taken by the right neighbour if it is its x corner e
    const int ro = __shfl_down_sync(full, o0[e], 1);
    const bool taken = lane < 31 && o1[e] >= 0 && ro == o1[e];
    if (valid) {
      red4(g + o0[e], own);
      if (!taken) red4(g + o1[e], mine1);
    }
  }
}

// (z, y, x) of a linear voxel index
__device__ __forceinline__ void unflat(Dims n, int v, int& z, int& y, int& x) {
  x = v % n.n2;
  const int r = v / n.n2;
  y = r % n.n1;
  z = r / n.n1;
}

}  // namespace muster
