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

#include <mutex>

namespace muster {

// Host: runs f() (returning cudaError_t) once for the current device. Kernel attributes
// such as the dynamic shared memory limit belong to a device's context, so set-up that
// sets them is repeated on every device the process uses; a failed set-up is retried on
// the next call and its error returned.
constexpr int kMaxDevices = 64;
template <class Fn>
cudaError_t once_per_device(bool (&done)[kMaxDevices], std::mutex& mu, Fn f) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  e = f();
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

// Host: number of SMs of the current device, read once per device (152 on GB300; 152 if
// the query fails, so grid sizing never sees 0).
inline int device_sm_count() {
  static std::mutex mu;
  static int count[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return 152;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!count[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 152;
    }
    count[dev] = n;
  }
  return count[dev];
}

struct Dims {
  int n0, n1, n2;  // D (slowest), H, W (contiguous)
};

// Float-float numbers (the unevaluated sum hi + lo, about 44 significant bits) for the CTA
// sums of loss terms: GB300's FP64 rate is 1/64 of its FP32 rate, so the kernels reduce in
// float-float within warps and leave double arithmetic to one thread per CTA. ff_add is
// Knuth's two-sum of the high parts, the low parts added to its error, then renormalised.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  const float e = ((a.hi - (s - v)) + (b.hi - v)) + (a.lo + b.lo);
  const float h = s + e;
  return FF{h, e - (h - s)};
}
// sum over the warp by a shuffle tree, valid in lane 0 (every lane must call it)
__device__ __forceinline__ FF warp_sum_ff(FF x) {
  for (int o = 16; o > 0; o >>= 1) {
    const FF y{__shfl_down_sync(0xffffffffu, x.hi, o), __shfl_down_sync(0xffffffffu, x.lo, o)};
    x = ff_add(x, y);
  }
  return x;
}

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

// transpose of sample4 with W-neighbours merged across a warp: when lane L+1 samples the
// cell next to lane L's along W, lane L's corners at x+1 (o001, o011, o101, o111) are lane
// L+1's corners at x (o000, o010, o100, o110); lane L+1 then adds lane L's share to its own
// before one reduction and lane L skips those corners. Both lanes decide from the same
// comparison of corner offsets, so any geometry (row ends, clamped edges, folds) is
// handled exactly. emit(offset, value) issues one reduction. Every lane of the warp must
// call it; valid = false contributes nothing. The merge is a fixed pattern of the warp, so
// the value emitted for a corner does not depend on timing. An extra term xv for node xo
// (xo < 0: none; the voxel's own part in the squaring adjoint) joins the first of the
// lane's corners at that node before the merges, and is emitted on its own when no corner
// is there: one reduction fewer per voxel whenever the sample cell touches the voxel's node.
template <class Emit>
__device__ __forceinline__ void scatter_merged(const Corners& k, float4 v, bool valid, Emit emit,
                                               float4 xv = float4{}, int xo = -1) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const float a1 = k.t0, a0 = 1.f - k.t0, b1 = k.t1, b0 = 1.f - k.t1, c1 = k.t2, c0 = 1.f - k.t2;
  const float w0[4] = {a0 * b0 * c0, a0 * b1 * c0, a1 * b0 * c0, a1 * b1 * c0};
  const float w1[4] = {a0 * b0 * c1, a0 * b1 * c1, a1 * b0 * c1, a1 * b1 * c1};
  const int o0[4] = {valid ? k.o000 : -1, valid ? k.o010 : -1, valid ? k.o100 : -1, valid ? k.o110 : -1};
  const int o1[4] = {valid ? k.o001 : -1, valid ? k.o011 : -1, valid ? k.o101 : -1, valid ? k.o111 : -1};
  // corner that takes the extra term: the first match among the x corners, else among the x+1 ones
  int xe = -1, xs = 0;
  if (valid && xo >= 0) {
#pragma unroll
    for (int e = 3; e >= 0; --e)
      if (o1[e] == xo) xe = e, xs = 1;
#pragma unroll
    for (int e = 3; e >= 0; --e)
      if (o0[e] == xo) xe = e, xs = 0;
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float4 own = f4scale(v, w0[e]);
    float4 mine1 = f4scale(v, w1[e]);
    if (xe == e) {
      if (xs == 0)
        own = f4add(own, xv);
      else
        mine1 = f4add(mine1, xv);
    }
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
      emit(o0[e], own);
      if (!taken) emit(o1[e], mine1);
    }
  }
  if (valid && xo >= 0 && xe < 0) emit(xo, xv);
}

// scatter_merged into a float4 field with vector reductions (the atomic adjoint: the
// order in which reductions of different warps arrive changes the last bits of the sums)
__device__ __forceinline__ void scatter4_merged(float4* g, const Corners& k, float4 v, bool valid) {
  scatter_merged(k, v, valid, [&](int o, float4 x) { red4(g + o, x); });
}

// 2-D thread layout of the scatter adjoints: a CTA of 256 threads covers 16 (W) x 16 (H)
// voxels of one plane and each warp an 8 (W) x 4 (H) patch (lane = 8 * row + column), so
// that the corners neighbouring voxels share along W and along H meet inside one warp
struct Tile2 {
  int x, y, lx, ly;
};
constexpr int kT2 = 16;  // tile edge (voxels) of the 2-D layout
__device__ __forceinline__ Tile2 tile2() {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Tile2 t;
  t.lx = lane & 7;
  t.ly = lane >> 3;
  t.x = blockIdx.x * kT2 + (w & 1) * 8 + t.lx;
  t.y = blockIdx.y * kT2 + (w >> 1) * 4 + t.ly;
  return t;
}

// Transpose of sample4 for the 2-D layout, with corners merged along W and then along H
// inside a warp: a voxel's x1 corners are the x0 corners of the voxel to its right when
// both sample neighbouring cells, and its y1 corners the y0 corners of the voxel below; the
// receiving lane adds the share to its own before one reduction and the giving lane skips
// it. Both lanes decide from the same comparison of corner offsets, so every geometry
// (grid ends, clamped edges, folds) is handled exactly. emit(offset, value) issues one
// reduction. Every lane of the warp must call it; valid = false contributes nothing. The
// merges follow a fixed pattern of the warp, so the values emitted do not depend on timing.
// An extra term xv for node xo joins the lane's first corner at that node, as in
// scatter_merged.
// The merges of scatter_merged_2d without the reductions: the lane's corner values and
// offsets after the W and H merges (offset -1: nothing to add there), and whether the extra
// term joined a corner.
__device__ __forceinline__ void merge_2d(const Corners& k, float4 v, bool valid, int lx, int ly, float4 xv, int xo,
                                         float4 (&val)[2][2][2], int (&off)[2][2][2], bool& placed) {
  const unsigned full = 0xffffffffu;
  const float a[2] = {1.f - k.t0, k.t0}, b[2] = {1.f - k.t1, k.t1}, c[2] = {1.f - k.t2, k.t2};
  const int oo[2][2][2] = {{{k.o000, k.o001}, {k.o010, k.o011}}, {{k.o100, k.o101}, {k.o110, k.o111}}};
#pragma unroll
  for (int zi = 0; zi < 2; ++zi)
#pragma unroll
    for (int yi = 0; yi < 2; ++yi)
#pragma unroll
      for (int xi = 0; xi < 2; ++xi) {
        val[zi][yi][xi] = f4scale(v, a[zi] * b[yi] * c[xi]);
        off[zi][yi][xi] = valid ? oo[zi][yi][xi] : -1;
      }
  placed = !(valid && xo >= 0);
#pragma unroll
  for (int zi = 0; zi < 2; ++zi)
#pragma unroll
    for (int yi = 0; yi < 2; ++yi)
#pragma unroll
      for (int xi = 0; xi < 2; ++xi)
        if (!placed && off[zi][yi][xi] == xo) {
          val[zi][yi][xi] = f4add(val[zi][yi][xi], xv);
          placed = true;
        }
  // along W: lanes +-1 within a row of 8
#pragma unroll
  for (int zi = 0; zi < 2; ++zi)
#pragma unroll
    for (int yi = 0; yi < 2; ++yi) {
      const int lo = __shfl_up_sync(full, off[zi][yi][1], 1);
      const float4 m1 = val[zi][yi][1];
      const float lvx = __shfl_up_sync(full, m1.x, 1), lvy = __shfl_up_sync(full, m1.y, 1),
                  lvz = __shfl_up_sync(full, m1.z, 1);
      const int ro = __shfl_down_sync(full, off[zi][yi][0], 1);
      if (lx > 0 && lo >= 0 && lo == off[zi][yi][0]) {
        val[zi][yi][0].x += lvx;
        val[zi][yi][0].y += lvy;
        val[zi][yi][0].z += lvz;
      }
      if (lx < 7 && off[zi][yi][1] >= 0 && ro == off[zi][yi][1]) off[zi][yi][1] = -1;
    }
  // along H: lanes +-8 within a column of 4
#pragma unroll
  for (int zi = 0; zi < 2; ++zi)
#pragma unroll
    for (int xi = 0; xi < 2; ++xi) {
      const int uo = __shfl_up_sync(full, off[zi][1][xi], 8);
      const float4 m1 = val[zi][1][xi];
      const float uvx = __shfl_up_sync(full, m1.x, 8), uvy = __shfl_up_sync(full, m1.y, 8),
                  uvz = __shfl_up_sync(full, m1.z, 8);
      const int bo = __shfl_down_sync(full, off[zi][0][xi], 8);
      if (ly > 0 && uo >= 0 && uo == off[zi][0][xi]) {
        val[zi][0][xi].x += uvx;
        val[zi][0][xi].y += uvy;
        val[zi][0][xi].z += uvz;
      }
      if (ly < 3 && off[zi][1][xi] >= 0 && bo == off[zi][1][xi]) off[zi][1][xi] = -1;
    }
}

template <class Emit>
__device__ __forceinline__ void scatter_merged_2d(const Corners& k, float4 v, bool valid, int lx, int ly, Emit emit,
                                                  float4 xv = float4{}, int xo = -1) {
  float4 val[2][2][2];
  int off[2][2][2];
  bool placed;
  merge_2d(k, v, valid, lx, ly, xv, xo, val, off, placed);
#pragma unroll
  for (int zi = 0; zi < 2; ++zi)
#pragma unroll
    for (int yi = 0; yi < 2; ++yi)
#pragma unroll
      for (int xi = 0; xi < 2; ++xi)
        if (off[zi][yi][xi] >= 0) emit(off[zi][yi][xi], val[zi][yi][xi]);
  if (!placed) emit(xo, xv);
}

// Scatter of a lane's two voxels of one column, (z, y, x) and (z + 1, y, x), merged along D
// as well: after each voxel's W and H merges, a z+1 corner of the first that is the same node
// as the second's z corner at the same (y, x) place joins it before the reduction (in a
// smooth map, neighbouring voxels sample neighbouring cells). dz_first(val, off) is called
// between the two voxels with the first's corners; the z corners of the first are emitted
// there and its z+1 corners kept; dz_second emits the rest. A fixed pattern per lane, so the
// values emitted do not depend on timing.
struct KeepZ1 {
  float4 val[2][2];
  int off[2][2];
};
template <class Emit>
__device__ __forceinline__ void dz_first(const float4 (&val)[2][2][2], const int (&off)[2][2][2], KeepZ1& kp,
                                         Emit emit) {
#pragma unroll
  for (int yi = 0; yi < 2; ++yi)
#pragma unroll
    for (int xi = 0; xi < 2; ++xi) {
      if (off[0][yi][xi] >= 0) emit(off[0][yi][xi], val[0][yi][xi]);
      kp.val[yi][xi] = val[1][yi][xi];
      kp.off[yi][xi] = off[1][yi][xi];
    }
}
template <class Emit>
__device__ __forceinline__ void dz_second(float4 (&val)[2][2][2], const int (&off)[2][2][2], KeepZ1& kp, Emit emit) {
#pragma unroll
  for (int yi = 0; yi < 2; ++yi)
#pragma unroll
    for (int xi = 0; xi < 2; ++xi)
      if (kp.off[yi][xi] >= 0 && kp.off[yi][xi] == off[0][yi][xi]) {
        val[0][yi][xi] = f4add(val[0][yi][xi], kp.val[yi][xi]);
        kp.off[yi][xi] = -1;
      }
#pragma unroll
  for (int zi = 0; zi < 2; ++zi)
#pragma unroll
    for (int yi = 0; yi < 2; ++yi)
#pragma unroll
      for (int xi = 0; xi < 2; ++xi)
        if (off[zi][yi][xi] >= 0) emit(off[zi][yi][xi], val[zi][yi][xi]);
#pragma unroll
  for (int yi = 0; yi < 2; ++yi)
#pragma unroll
    for (int xi = 0; xi < 2; ++xi)
      if (kp.off[yi][xi] >= 0) emit(kp.off[yi][xi], kp.val[yi][xi]);
}

// ---- fixed-point accumulation (the deterministic adjoint). A float sum of terms that are
// all integer multiples of a power of two q is exact as long as every partial sum stays
// below 2^24 q in magnitude, so it is the same in whatever order the terms arrive. Each
// term x is split into x_hi = x rounded to a multiple of q and the remainder (exact, at
// most q/2) rounded to a multiple of q 2^-14, and the two go to two float4 accumulators by
// vector reductions; the reader adds hi + lo. The quantum is chosen per launch
// (fx_quantum): q = 2^(e + off - 10) with M < 2^e the step's largest pair gradient and off
// the expected growth (in bits) of the terms of that launch over M, so expected terms are
// near 2^10 q: a hi sum stays exact for 2^14 of them, a lo sum (terms below 2^13 q 2^-14)
// for 2^11 terms, and the lo quantum resolves 2^-24 of the expected magnitude. A scattered
// value or own part at or above 2^19 q raises *oflow (below that, terms stay below 2^21 q,
// and eight of them below 2^24 q).
struct FxQ {
  float q, mh, ml;  // quantum; 1.5 * 2^23 q and 1.5 * 2^23 q 2^-14 (rounding constants of hi, lo)
};
__device__ __forceinline__ FxQ fx_quantum(const unsigned* gmax, int off) {
  // M < 2^e with e = (biased exponent of M) - 126 for the non-negative float M
  const int e = (int)((*gmax >> 23) & 0xffu) - 126;
  const int k = min(max(e + off - 10, -100), 100);
  // powers of two and 1.5 times powers of two, built from their bits
  return FxQ{__int_as_float((k + 127) << 23), __int_as_float(((k + 23 + 127) << 23) | 0x400000),
             __int_as_float(((k + 9 + 127) << 23) | 0x400000)};
}
// x rounded to the nearest multiple of q (m = 1.5 * 2^23 q, |x| < 2^22 q): adding m leaves
// the float's last place at q, subtracting it is exact
__device__ __forceinline__ float fx_rnd(float x, float m) { return __fsub_rn(__fadd_rn(x, m), m); }
// flags a value too large for the accumulators' headroom: a term of the scatter is at most
// twice the largest value a warp scatters (merged corner weights sum to at most 2) plus the
// voxel's own part that joins a corner, so the check is made once per scattered value and
// own part, at 2^19 q (terms stay below 2^21 q)
__device__ __forceinline__ void fx_guard(float4 x, FxQ Q, int* oflow) {
  if (fmaxf(fabsf(x.x), fmaxf(fabsf(x.y), fabsf(x.z))) >= 0x1p19f * Q.q) atomicOr(oflow, 1);
}
// one term into the accumulator pair (hi at a, lo at a + V)
__device__ __forceinline__ void red4_fx(float4* a, size_t V, int o, float4 x, FxQ Q) {
  const float4 h = make_float4(fx_rnd(x.x, Q.mh), fx_rnd(x.y, Q.mh), fx_rnd(x.z, Q.mh), 0.f);
  // the remainders x - h are exact (Sterbenz), at most q/2
  red4(a + o, h);
  red4(a + V + o, make_float4(fx_rnd(__fsub_rn(x.x, h.x), Q.ml), fx_rnd(__fsub_rn(x.y, h.y), Q.ml),
                              fx_rnd(__fsub_rn(x.z, h.z), Q.ml), 0.f));
}
// the sum at node o of an accumulator pair
__device__ __forceinline__ float4 load_fx(const float4* a, size_t V, int o) {
  const float4 h = a[o], l = a[V + o];
  return make_float4(h.x + l.x, h.y + l.y, h.z + l.z, 0.f);
}
// clears node o of an accumulator pair for its next use; called once the loads of the node
// have been used, so that the stores do not wait behind them
__device__ __forceinline__ void clear_fx(float4* a, size_t V, int o) {
  a[o] = make_float4(0.f, 0.f, 0.f, 0.f);
  a[V + o] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// (z, y, x) of a linear voxel index
__device__ __forceinline__ void unflat(Dims n, int v, int& z, int& y, int& x) {
  x = v % n.n2;
  const int r = v / n.n2;
  y = r % n.n1;
  z = r / n.n1;
}

}  // namespace muster
