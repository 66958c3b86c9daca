// field_kernels.cu -- kernels on the velocity (flow) grid: prolongation between
// pyramid levels, scaling and squaring (Alg. 1) and its adjoint, composition of
// consecutive deformations (Eq. cum_deformation) and its adjoint, the
// regulariser (Eq. reg_ss, the L2 term, Eq. reg_ts) and the optimiser update
// (Sec. Implementation Details).
//
// All of them stream flow-grid fields (float4 per voxel) and gather trilinear
// corners through the read-only cache; scatters of the adjoints are vector
// reductions into L2, or, in the deterministic mode, reductions of fixed-point terms
// whose sums are exact in any order (common.cuh). Grids: x over voxels (256 threads), y over
// fields/chains; the deterministic scatter adjoints take 16 x 16 voxel tiles of a plane (or
// of a pair of planes) in x and y, and planes x fields/chains in z.
#include <algorithm>

#include "kernels.h"

namespace muster {

namespace {
constexpr int kThreads = 256;

__host__ __device__ inline unsigned blocks_for(size_t V) { return (unsigned)((V + kThreads - 1) / kThreads); }

// ---- Sec. Implementation Details: velocity initialised from the previous stage
__global__ void k_prolong(const float4* __restrict__ coarse, Dims nc, float4* __restrict__ fine, Dims nf) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t Vf = vox(nf);
  if (v >= (int)Vf) return;
  const int f = blockIdx.y;
  int z, y, x;
  unflat(nf, v, z, y, x);
  const float4 s = sample4(coarse + (size_t)f * vox(nc), nc, 0.5f * z - 0.25f, 0.5f * y - 0.25f,
                           0.5f * x - 0.25f);
  fine[(size_t)f * Vf + v] = f4scale(s, 2.f);
}

// ---- Alg. 1, first line: u_0 = sign * phi / 2^K; fields [0, F) are +phi, [F, 2F) are -phi
__global__ void k_exp_init(const float4* __restrict__ theta, float4* __restrict__ u0, int F, int V,
                           float scale, unsigned* __restrict__ zero) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (zero && v == 0 && blockIdx.y == 0) *zero = 0u;  // a per-step word the step's later kernels set
  if (v >= V) return;
  const int f = blockIdx.y;
  const float s = f < F ? scale : -scale;
  u0[(size_t)f * V + v] = f4scale(theta[(size_t)(f < F ? f : f - F) * V + v], s);
}

// The four kernels below give each thread NF fields (or chains) of one voxel: the loads of
// the NF fields are independent, so each thread keeps NF gather chains in flight (the
// kernels wait on dependent loads: the field at x, then the 8 corners at x + u(x)).
// Field j of a thread is blockIdx.y * NF + j; fields past `count` are skipped.

// ---- Alg. 1, loop body in displacement form: u(x) <- u(x) + S[u](x + u(x))
template <int NF>
__global__ void k_squaring(const float4* __restrict__ u, float4* __restrict__ un, Dims n, int count) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int V = (int)vox(n);
  if (v >= V) return;
  int z, y, x;
  unflat(n, v, z, y, x);
  float4 a[NF];
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const int f = blockIdx.y * NF + j;
    a[j] = f < count ? u[(size_t)f * V + v] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const int f = blockIdx.y * NF + j;
    if (f >= count) continue;
    const float4* uf = u + (size_t)f * V;
    un[(size_t)f * V + v] = f4add(a[j], sample4(uf, n, z + a[j].x, y + a[j].y, x + a[j].z));
  }
}

// ---- Alg. 1, first line and first loop iteration in one launch: u_0 = sign phi / 2^K is
// written (the adjoint reads it) and u_1 = u_0 + S[u_0](x + u_0(x)) is computed from phi.
// sign / 2^K is a power of two, so scaling commutes with every rounding of the trilinear
// sample: u_1 equals the result of forming u_0 first, bit for bit.
template <int NF>
__global__ void k_squaring_first(const float4* __restrict__ th, float4* __restrict__ u0, float4* __restrict__ u1,
                                 Dims n, int count, int F, float scale, unsigned* __restrict__ zero) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (zero && v == 0 && blockIdx.y == 0) *zero = 0u;  // a per-step word the step's later kernels set
  const int V = (int)vox(n);
  if (v >= V) return;
  int z, y, x;
  unflat(n, v, z, y, x);
  float4 a[NF];
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const int f = blockIdx.y * NF + j;
    a[j] = f < count ? f4scale(th[(size_t)(f < F ? f : f - F) * V + v], f < F ? scale : -scale)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const int f = blockIdx.y * NF + j;
    if (f >= count) continue;
    const float s = f < F ? scale : -scale;
    u0[(size_t)f * V + v] = a[j];
    const float4 g = sample4(th + (size_t)(f < F ? f : f - F) * V, n, z + a[j].x, y + a[j].y, x + a[j].z);
    u1[(size_t)f * V + v] = f4add(a[j], f4scale(g, s));
  }
}

// Thread placement of the scatter adjoints. Atomic mode: consecutive threads on consecutive
// voxels of the flattened grid (x over voxels, y over groups of fields), corners merged along W
// within a warp. Deterministic mode, whose fixed-point terms take two reductions each and
// are bound by the L2's reduction throughput: the 2-D layout of tile2 with two planes per
// lane (k_squaring_bwd_dz, k_compose_bwd_dz: corners merged along W, H and D), or with one
// plane (z over planes x groups, corners merged along W and H) where the plane pairs times
// fields exceed the grid's z limit.
struct Place {
  int x, y, z, v, grp, lx, ly;
  bool vin;
};
template <bool TWO_D>
__device__ __forceinline__ Place place(Dims n) {
  Place p;
  if (TWO_D) {
    p.z = blockIdx.z % n.n0;
    p.grp = blockIdx.z / n.n0;
    const Tile2 t = tile2();
    p.x = t.x;
    p.y = t.y;
    p.lx = t.lx;
    p.ly = t.ly;
    p.vin = p.x < n.n2 && p.y < n.n1;
    p.v = p.vin ? (p.z * n.n1 + p.y) * n.n2 + p.x : 0;
  } else {
    p.grp = blockIdx.y;
    p.v = blockIdx.x * blockDim.x + threadIdx.x;
    p.vin = p.v < (int)vox(n);
    p.x = p.y = p.z = p.lx = p.ly = 0;
    if (p.vin) unflat(n, p.v, p.z, p.y, p.x);
  }
  return p;
}
template <bool TWO_D, class Emit>
__device__ __forceinline__ void scatter_placed(const Place& p, const Corners& k, float4 g, Emit emit,
                                               float4 xv = float4{}, int xo = -1) {
  if (TWO_D)
    scatter_merged_2d(k, g, p.vin, p.lx, p.ly, emit, xv, xo);
  else
    scatter_merged(k, g, p.vin, emit, xv, xo);
}

// ---- adjoint of one squaring: G_in is dL/du_{t+1}; G_out receives dL/du_t:
//   through the sample point  G_out(x) += G + J^T G   (J = dS[u_t]/dq at x + u_t(x))
//   through the sampled field G_out(corner) += w_corner * G
// FX = false: G_out (zeroed) takes both parts by vector reductions.
// FX = true (deterministic): G_in is the fixed-point sums of fx.ain (read and cleared) plus,
// if not null, the float field Gin; both parts go to the fixed-point accumulators fx.aout
// (G_out is not used). In the first step (t = K - 1) G_in also takes the gradient of the
// field's single-step pair map from pg (the chains' adjoint leaves it there).
// CLEAR (atomic mode): G_in read through Gclr (the same buffer) and its node cleared after
// the read, so that the buffer is zero for its next use as an output (small grids, where a
// separate clearing pass costs more than the stores).
template <bool FX, int NF, bool CLEAR = false>
__global__ void k_squaring_bwd(const float4* __restrict__ u, const float4* __restrict__ Gin,
                               float4* __restrict__ Gout, Dims n, int count, FxArgs fx,
                               const __grid_constant__ PairGradTab pg, float4* Gclr) {
  const Place p = place<FX>(n);
  const int x = p.x, y = p.y, z = p.z, v = p.v, grp = p.grp;
  const bool vin = p.vin;
  const int V = (int)vox(n);
  const FxQ qout = FX ? fx_quantum(fx.gmax, fx.off_out) : FxQ{};
  float4 a[NF], G[NF];
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const size_t off = (size_t)(grp * NF + j) * V;
    const bool ok = vin && grp * NF + j < count;
    a[j] = ok ? u[off + v] : make_float4(0.f, 0.f, 0.f, 0.f);
    G[j] = ok && Gin ? (CLEAR ? Gclr[off + v] : Gin[off + v]) : make_float4(0.f, 0.f, 0.f, 0.f);
    if (CLEAR && ok) Gclr[off + v] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ok && pg.G) G[j] = f4add(G[j], pg.G[(size_t)pg.slot_pair[grp * NF + j] * V + v]);
    if (FX && ok) G[j] = f4add(G[j], load_fx(fx.ain + 2 * off, V, v));
  }
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const int f = grp * NF + j;
    if (f >= count) continue;  // uniform over the CTA
    const size_t off = (size_t)f * V;
    Corners k{};
    float4 own = make_float4(0.f, 0.f, 0.f, 0.f);
    if (vin) {
      const Samp4 s = sample4_grad(u + off, n, z + a[j].x, y + a[j].y, x + a[j].z, &k);
      const float4 g = G[j];
      own = make_float4(g.x + f4dot3(s.d0, g), g.y + f4dot3(s.d1, g), g.z + f4dot3(s.d2, g), 0.f);
      if (FX) {
        fx_guard(g, qout, fx.oflow);
        fx_guard(own, qout, fx.oflow);
      }
    }
    // every lane of the warp: merges inside; the own part joins the corner at this voxel's
    // node when the sample cell has one (always while |u| < 1 voxel)
    if (FX) {
      float4* acc = fx.aout + 2 * off;
      scatter_placed<FX>(p, k, G[j], [&](int o, float4 q) { red4_fx(acc, V, o, q, qout); }, own, vin ? v : -1);
    } else {
      float4* g = Gout + off;
      scatter_placed<FX>(p, k, G[j], [&](int o, float4 q) { red4(g + o, q); }, own, vin ? v : -1);
    }
  }
  if (FX && vin) {
#pragma unroll
    for (int j = 0; j < NF; ++j)
      if (grp * NF + j < count) clear_fx(fx.ain + 2 * (size_t)(grp * NF + j) * V, V, v);
  }
}

// ---- the deterministic squaring adjoint with two voxels of one column per lane (planes
// 2 zp and 2 zp + 1 of one field; grid z = planes / 2 x fields), so that the scattered
// corners are merged along D as well as along W and H before their fixed-point reductions
__global__ void k_squaring_bwd_dz(const float4* __restrict__ u, const float4* __restrict__ Gin, Dims n, FxArgs fx,
                                  const __grid_constant__ PairGradTab pg) {
  const int nzp = (n.n0 + 1) / 2;
  const int zp = blockIdx.z % nzp, f = blockIdx.z / nzp;
  const Tile2 tl = tile2();
  const int x = tl.x, y = tl.y;
  const bool inxy = x < n.n2 && y < n.n1;
  const int V = (int)vox(n);
  const size_t off = (size_t)f * V;
  const FxQ qout = fx_quantum(fx.gmax, fx.off_out);
  float4 a[2], G[2];
  int v[2];
  bool vin[2];
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    const int z = 2 * zp + dz;
    vin[dz] = inxy && z < n.n0;
    v[dz] = vin[dz] ? (z * n.n1 + y) * n.n2 + x : 0;
    a[dz] = vin[dz] ? u[off + v[dz]] : make_float4(0.f, 0.f, 0.f, 0.f);
    G[dz] = vin[dz] && Gin ? Gin[off + v[dz]] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (vin[dz] && pg.G) G[dz] = f4add(G[dz], pg.G[(size_t)pg.slot_pair[f] * V + v[dz]]);
    if (vin[dz]) G[dz] = f4add(G[dz], load_fx(fx.ain + 2 * off, V, v[dz]));
  }
  float4* acc = fx.aout + 2 * off;
  auto emit = [&](int o, float4 q) { red4_fx(acc, V, o, q, qout); };
  KeepZ1 kp;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    Corners k{};
    float4 own = make_float4(0.f, 0.f, 0.f, 0.f);
    if (vin[dz]) {
      const Samp4 s = sample4_grad(u + off, n, 2 * zp + dz + a[dz].x, y + a[dz].y, x + a[dz].z, &k);
      const float4 g = G[dz];
      own = make_float4(g.x + f4dot3(s.d0, g), g.y + f4dot3(s.d1, g), g.z + f4dot3(s.d2, g), 0.f);
      fx_guard(g, qout, fx.oflow);
      fx_guard(own, qout, fx.oflow);
    }
    // every lane of the warp: merges inside; the own part joins the corner at the voxel's node
    float4 val[2][2][2];
    int offs[2][2][2];
    bool placed;
    merge_2d(k, G[dz], vin[dz], tl.lx, tl.ly, own, vin[dz] ? v[dz] : -1, val, offs, placed);
    if (dz == 0)
      dz_first(val, offs, kp, emit);
    else
      dz_second(val, offs, kp, emit);
    if (!placed) emit(v[dz], own);
  }
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
    if (vin[dz]) clear_fx(fx.ain + 2 * off, V, v[dz]);
}

// ---- Eq. cum_deformation: U_new(x) = U_prev(x) + S[u](x + U_prev(x))
template <int NF>
__global__ void __launch_bounds__(kThreads, 8) k_compose(const __grid_constant__ ComposeTab t, Dims n, int count) {
  const ComposeDesc* d = t.d;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= (int)vox(n)) return;
  int z, y, x;
  unflat(n, v, z, y, x);
  float4 a[NF];
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const int c = blockIdx.y * NF + j;
    a[j] = c < count ? d[c].Uprev[v] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const int c = blockIdx.y * NF + j;
    if (c >= count) continue;
    d[c].Unew[v] = f4add(a[j], sample4(d[c].u, n, z + a[j].x, y + a[j].y, x + a[j].z));
  }
}

// ---- adjoint of one composition step (unique writer of Gprev per chain and voxel); the
// scatter into the sampled field's gradient goes to gfield by vector reductions, or (FX) to
// its fixed-point accumulator gacc. Thread placement as k_squaring_bwd.
template <bool FX, int NF>
__global__ void __launch_bounds__(kThreads, 4)
    k_compose_bwd(const __grid_constant__ ComposeBwdTab t, Dims n, int count, FxArgs fx) {
  const ComposeBwdDesc* d = t.d;
  const Place p = place<FX>(n);
  const int x = p.x, y = p.y, z = p.z, v = p.v, grp = p.grp;
  const bool vin = p.vin;
  const int V = (int)vox(n);
  const FxQ qout = FX ? fx_quantum(fx.gmax, fx.off_out) : FxQ{};
  // G_prev is read with the chain's other operands, ahead of the gather: this thread is
  // its only writer and the scatter goes to the sampled field's gradient, another buffer
  float4 a[NF], G[NF], P[NF];
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const int c = grp * NF + j;
    const bool ok = vin && c < count;
    a[j] = ok ? d[c].Uprev[v] : make_float4(0.f, 0.f, 0.f, 0.f);
    G[j] = ok ? d[c].G[v] : make_float4(0.f, 0.f, 0.f, 0.f);
    P[j] = ok ? d[c].Gprev[v] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const int ci = grp * NF + j;
    if (ci >= count) continue;  // uniform over the CTA
    const ComposeBwdDesc c = d[ci];
    Corners k{};
    if (vin) {
      const Samp4 s = sample4_grad(c.u, n, z + a[j].x, y + a[j].y, x + a[j].z, &k);
      const float4 g = G[j];
      float4 p = P[j];
      p.x += g.x + f4dot3(s.d0, g);
      p.y += g.y + f4dot3(s.d1, g);
      p.z += g.z + f4dot3(s.d2, g);
      c.Gprev[v] = p;
    }
    // every lane of the warp: merges inside
    if (FX) {
      float4* acc = c.gacc;
      if (vin) fx_guard(G[j], qout, fx.oflow);
      scatter_placed<FX>(p, k, G[j], [&](int o, float4 q) { red4_fx(acc, V, o, q, qout); });
    } else {
      float4* g = c.gfield;
      scatter_placed<FX>(p, k, G[j], [&](int o, float4 q) { red4(g + o, q); });
    }
  }
}

// ---- the deterministic composition adjoint with two voxels of one column per lane (planes
// 2 zp and 2 zp + 1 of one chain; grid z = planes / 2 x chains), merged along D as well
__global__ void k_compose_bwd_dz(const __grid_constant__ ComposeBwdTab t, Dims n, FxArgs fx) {
  const int nzp = (n.n0 + 1) / 2;
  const int zp = blockIdx.z % nzp, ci = blockIdx.z / nzp;
  const ComposeBwdDesc c = t.d[ci];
  const Tile2 tl = tile2();
  const int x = tl.x, y = tl.y;
  const bool inxy = x < n.n2 && y < n.n1;
  const int V = (int)vox(n);
  const FxQ qout = fx_quantum(fx.gmax, fx.off_out);
  float4 a[2], G[2], P[2];
  int v[2];
  bool vin[2];
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    const int z = 2 * zp + dz;
    vin[dz] = inxy && z < n.n0;
    v[dz] = vin[dz] ? (z * n.n1 + y) * n.n2 + x : 0;
    a[dz] = vin[dz] ? c.Uprev[v[dz]] : make_float4(0.f, 0.f, 0.f, 0.f);
    G[dz] = vin[dz] ? c.G[v[dz]] : make_float4(0.f, 0.f, 0.f, 0.f);
    P[dz] = vin[dz] ? c.Gprev[v[dz]] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  auto emit = [&](int o, float4 q) { red4_fx(c.gacc, V, o, q, qout); };
  KeepZ1 kp;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    Corners k{};
    if (vin[dz]) {
      const Samp4 s = sample4_grad(c.u, n, 2 * zp + dz + a[dz].x, y + a[dz].y, x + a[dz].z, &k);
      const float4 g = G[dz];
      float4 p = P[dz];
      p.x += g.x + f4dot3(s.d0, g);
      p.y += g.y + f4dot3(s.d1, g);
      p.z += g.z + f4dot3(s.d2, g);
      c.Gprev[v[dz]] = p;
      fx_guard(g, qout, fx.oflow);
    }
    float4 val[2][2][2];
    int offs[2][2][2];
    bool placed;
    merge_2d(k, G[dz], vin[dz], tl.lx, tl.ly, float4{}, -1, val, offs, placed);
    if (dz == 0)
      dz_first(val, offs, kp, emit);
    else
      dz_second(val, offs, kp, emit);
  }
}

// ---- Appendix Gaussian Smoothing along one axis: circular convolution of every field with
// the taps (inverse DFT of the Gaussian response, symmetric: taps[d] = taps[m - d]) over
// the offsets lo..hi (either the whole circle or the taps above FP32 resolution)
__global__ void k_smooth_axis(const float4* __restrict__ in, float4* __restrict__ out, Dims n, int axis,
                              const float* __restrict__ taps, int lo, int hi) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int V = (int)vox(n);
  if (v >= V) return;
  const size_t off = (size_t)blockIdx.y * V;
  int z, y, x;
  unflat(n, v, z, y, x);
  const int p = axis == 0 ? z : (axis == 1 ? y : x);
  const int m = axis == 0 ? n.n0 : (axis == 1 ? n.n1 : n.n2);
  const int stride = axis == 0 ? n.n1 * n.n2 : (axis == 1 ? n.n2 : 1);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int d = lo; d <= hi; ++d) {
    int q = p - d;
    if (q < 0) q += m;
    if (q >= m) q -= m;
    const float w = __ldg(taps + (d < 0 ? d + m : d));
    const float4 a = __ldg(in + off + v + (q - p) * stride);
    acc.x = fmaf(w, a.x, acc.x);
    acc.y = fmaf(w, a.y, acc.y);
    acc.z = fmaf(w, a.z, acc.z);
  }
  out[off + v] = acc;
}

__global__ void k_add(const __grid_constant__ AddTab t, int V) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const AddDesc a = t.d[blockIdx.y];
  a.dst[v] = f4add(a.dst[v], a.src[v]);
}

// The CTA's sums of three per-thread values, written to out[0..2] by thread 0: float-float
// sums within each warp, then the warp sums in double.
__device__ __forceinline__ void block_sum3(float a, float b, float c, double* out) {
  __shared__ float sh[3][2][kThreads / 32];
  const FF s[3] = {warp_sum_ff(FF{a, 0.f}), warp_sum_ff(FF{b, 0.f}), warp_sum_ff(FF{c, 0.f})};
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
    for (int k = 0; k < 3; ++k) {
      sh[k][0][w] = s[k].hi;
      sh[k][1][w] = s[k].lo;
    }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) {
      double r = 0.0;
      for (int i = 0; i < kThreads / 32; ++i) r += (double)sh[k][0][i] + (double)sh[k][1][i];
      out[k] = r;
    }
}

// ---- Eq. reg_ss / the L2 term / Eq. reg_ts (means over the flow grid) and the
// total gradient dL/dphi = (G0+ - G0-) / 2^K + dL_reg/dphi.
// With fx.ain (deterministic mode) G0 is completed with its fixed-point sums, which are cleared.
// CLEAR: G0 read through G0clr (the same buffer) and cleared after the read (see
// k_squaring_bwd's Gclr)
template <bool CLEAR>
__global__ void k_reg_grad(const float4* __restrict__ th, const float4* __restrict__ G0,
                           float4* __restrict__ grad, double* __restrict__ part, Dims n, RegArgs a, FxArgs fx,
                           float4* G0clr) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int V = (int)vox(n);
  const int f = blockIdx.y, F = a.n_fields;
  float lss = 0.f, ll2 = 0.f, lts = 0.f;
  if (v < V) {
    const float4* T = th + (size_t)f * V;
    int z, y, x;
    unflat(n, v, z, y, x);
    const float4 c = T[v];
    float4 gp = make_float4(0.f, 0.f, 0.f, 0.f), gm = gp;
    if (CLEAR) {
      gp = G0clr[(size_t)f * V + v];
      gm = G0clr[(size_t)(F + f) * V + v];
      G0clr[(size_t)f * V + v] = make_float4(0.f, 0.f, 0.f, 0.f);
      G0clr[(size_t)(F + f) * V + v] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else if (G0) {
      gp = G0[(size_t)f * V + v];
      gm = G0[(size_t)(F + f) * V + v];
    }
    if (fx.ain) {
      gp = f4add(gp, load_fx(fx.ain + (size_t)2 * f * V, V, v));
      gm = f4add(gm, load_fx(fx.ain + (size_t)2 * (F + f) * V, V, v));
    }
    float4 g = f4scale(f4sub(gp, gm), a.inv2K);
    const int pos[3] = {z, y, x}, ext[3] = {n.n0, n.n1, n.n2};
    const int stride[3] = {n.n1 * n.n2, n.n2, 1};
    const float kss = 2.f * a.alpha_ss / (float)F;
    for (int ax = 0; ax < 3; ++ax) {
      if (ext[ax] < 2) continue;
      const float invM = (float)ext[ax] / ((float)(ext[ax] - 1) * (float)V);
      if (pos[ax] + 1 < ext[ax]) {
        const float4 d = f4sub(T[v + stride[ax]], c);
        lss += f4dot3(d, d) * invM;
        g = f4sub(g, f4scale(d, kss * invM));
      }
      if (pos[ax] > 0) g = f4add(g, f4scale(f4sub(c, T[v - stride[ax]]), kss * invM));
    }
    const float invV = 1.f / (float)V;
    ll2 = f4dot3(c, c) * invV;
    g = f4add(g, f4scale(c, 2.f * a.alpha_l2 * invV / (float)F));
    if (a.n_sessions >= 3) {
      const float kts = 2.f * a.alpha_ts * invV / (float)(a.n_sessions - 2);
      if (f + 1 < F) {  // term of session f+1: phi_f / dt_f - phi_{f+1} / dt_{f+1}
        const float4 r = f4sub(f4scale(c, a.inv_dt[f]), f4scale(th[(size_t)(f + 1) * V + v], a.inv_dt[f + 1]));
        lts = f4dot3(r, r) * invV;
        g = f4add(g, f4scale(r, kts * a.inv_dt[f]));
      }
      if (f >= 1) {  // term of session f: phi_{f-1} / dt_{f-1} - phi_f / dt_f
        const float4 r = f4sub(f4scale(th[(size_t)(f - 1) * V + v], a.inv_dt[f - 1]), f4scale(c, a.inv_dt[f]));
        g = f4sub(g, f4scale(r, kts * a.inv_dt[f]));
      }
    }
    grad[(size_t)f * V + v] = g;
    if (fx.ain) {
      clear_fx(fx.ain + (size_t)2 * f * V, V, v);
      clear_fx(fx.ain + (size_t)2 * (F + f) * V, V, v);
    }
  }
  const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
  block_sum3(lss, ll2, lts, part + 3 * b);
}

// ---- Adam (PyTorch update rule) or SGD with the per-step schedule
// sched[3*s] = lr_s, sched[3*s+1] = 1/(1-beta1^s), sched[3*s+2] = 1/(1-beta2^s)
__global__ void k_adam(float4* __restrict__ th, float4* __restrict__ m, float4* __restrict__ v,
                       const float4* __restrict__ g, size_t count, const float* __restrict__ sched,
                       const int* __restrict__ step, int sgd, float b1, float b2, float eps) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int s = *step;
  const float lr = sched[3 * s], ib1 = sched[3 * s + 1], ib2 = sched[3 * s + 2];
  const float4 gg = g[i];
  float4 t = th[i];
  if (sgd) {
    t = f4sub(t, f4scale(gg, lr));
  } else {
    float4 mm = m[i], vv = v[i];
    const float ga[3] = {gg.x, gg.y, gg.z};
    float ma[3] = {mm.x, mm.y, mm.z}, va[3] = {vv.x, vv.y, vv.z}, ta[3] = {t.x, t.y, t.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ma[c] = b1 * ma[c] + (1.f - b1) * ga[c];
      va[c] = b2 * va[c] + (1.f - b2) * ga[c] * ga[c];
      ta[c] -= lr * (ma[c] * ib1) / (sqrtf(va[c] * ib2) + eps);
    }
    m[i] = make_float4(ma[0], ma[1], ma[2], 0.f);
    v[i] = make_float4(va[0], va[1], va[2], 0.f);
    t = make_float4(ta[0], ta[1], ta[2], 0.f);
  }
  th[i] = t;
}

__global__ void k_f4_to_planar(const float4* __restrict__ in, float* __restrict__ out, size_t V) {
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const size_t f = blockIdx.y;
  const float4 a = in[f * V + v];
  out[(3 * f + 0) * V + v] = a.x;
  out[(3 * f + 1) * V + v] = a.y;
  out[(3 * f + 2) * V + v] = a.z;
}

__global__ void k_planar_to_f4(const float* __restrict__ in, float4* __restrict__ out, size_t V) {
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const size_t f = blockIdx.y;
  out[f * V + v] = make_float4(in[(3 * f + 0) * V + v], in[(3 * f + 1) * V + v], in[(3 * f + 2) * V + v], 0.f);
}
}  // namespace

void launch_prolong(const float4* coarse, Dims nc, float4* fine, Dims nf, int n_fields, cudaStream_t s) {
  k_prolong<<<dim3(blocks_for(vox(nf)), n_fields), kThreads, 0, s>>>(coarse, nc, fine, nf);
}
void launch_exp_init(const float4* theta, float4* u0, int n_fields, Dims n, float scale, cudaStream_t s,
                     unsigned* zero) {
  k_exp_init<<<dim3(blocks_for(vox(n)), 2 * n_fields), kThreads, 0, s>>>(theta, u0, n_fields, (int)vox(n), scale,
                                                                          zero);
}
// fields (or chains) per thread of the flow-grid gather kernels: 1 or 2 (the launch
// configuration; the results do not depend on it)
unsigned groups(int count, int nf) { return (unsigned)((count + nf - 1) / nf); }

void launch_squaring(const float4* u, float4* un, int n_fields2, Dims n, cudaStream_t s, int nf) {
  const dim3 g(blocks_for(vox(n)), groups(n_fields2, nf));
  if (nf == 1)
    k_squaring<1><<<g, kThreads, 0, s>>>(u, un, n, n_fields2);
  else
    k_squaring<2><<<g, kThreads, 0, s>>>(u, un, n, n_fields2);
}
void launch_squaring_first(const float4* theta, float4* u0, float4* u1, int n_fields, Dims n, float scale,
                           cudaStream_t s, int nf, unsigned* zero) {
  const dim3 g(blocks_for(vox(n)), groups(2 * n_fields, nf));
  if (nf == 1)
    k_squaring_first<1><<<g, kThreads, 0, s>>>(theta, u0, u1, n, 2 * n_fields, n_fields, scale, zero);
  else
    k_squaring_first<2><<<g, kThreads, 0, s>>>(theta, u0, u1, n, 2 * n_fields, n_fields, scale, zero);
}
// grid of the 2-D layout: W tiles, H tiles, D planes x groups of fields
dim3 grid2(Dims n, int count, int nf) {
  return dim3((n.n2 + kT2 - 1) / kT2, (n.n1 + kT2 - 1) / kT2, (unsigned)n.n0 * groups(count, nf));
}
template <int NF>
void squaring_bwd_nf(const float4* u, const float4* Gin, float4* Gout, int n_fields2, Dims n, const FxArgs* fx,
                     const PairGradTab& pg, float4* Gclr, cudaStream_t s) {
  if (fx)
    k_squaring_bwd<true, NF><<<grid2(n, n_fields2, NF), kThreads, 0, s>>>(u, Gin, Gout, n, n_fields2, *fx, pg,
                                                                          nullptr);
  else if (Gclr)
    k_squaring_bwd<false, NF, true><<<dim3(blocks_for(vox(n)), groups(n_fields2, NF)), kThreads, 0, s>>>(
        u, Gin, Gout, n, n_fields2, FxArgs{}, pg, Gclr);
  else
    k_squaring_bwd<false, NF><<<dim3(blocks_for(vox(n)), groups(n_fields2, NF)), kThreads, 0, s>>>(
        u, Gin, Gout, n, n_fields2, FxArgs{}, pg, nullptr);
}
// the 2-D layout puts planes x field groups on grid z (at most 65535): one field per thread
// only while that fits (a 2048-plane flow grid takes 31 groups of two fields at most)
int fx_nf(const FxArgs* fx, Dims n, int count, int nf) {
  return (fx && nf == 1 && (size_t)n.n0 * count > 65535) ? 2 : nf;
}
// grid of the deterministic two-plane layout: W tiles, H tiles, plane pairs x fields or chains
dim3 grid_dz(Dims n, int count) {
  return dim3((n.n2 + kT2 - 1) / kT2, (n.n1 + kT2 - 1) / kT2, (unsigned)((n.n0 + 1) / 2) * count);
}
bool dz_fits(Dims n, int count) { return (size_t)((n.n0 + 1) / 2) * count <= 65535; }

void launch_squaring_bwd(const float4* u, const float4* Gin, float4* Gout, int n_fields2, Dims n, const FxArgs* fx,
                         cudaStream_t s, int nf, const PairGradTab* pg, bool clear_in) {
  PairGradTab t{};
  if (pg && n_fields2 <= kMaxDescPerLaunch) t = *pg;
  if (fx && dz_fits(n, n_fields2)) {
    k_squaring_bwd_dz<<<grid_dz(n, n_fields2), kThreads, 0, s>>>(u, Gin, n, *fx, t);
    return;
  }
  nf = fx_nf(fx, n, n_fields2, nf);
  float4* clr = !fx && clear_in ? const_cast<float4*>(Gin) : nullptr;
  if (nf == 1)
    squaring_bwd_nf<1>(u, Gin, Gout, n_fields2, n, fx, t, clr, s);
  else
    squaring_bwd_nf<2>(u, Gin, Gout, n_fields2, n, fx, t, clr, s);
}
void launch_compose(const ComposeDesc* d, int n_chains, Dims n, cudaStream_t s, int nf) {
  for (int c0 = 0; c0 < n_chains; c0 += kMaxDescPerLaunch) {
    const int cnt = std::min(kMaxDescPerLaunch, n_chains - c0);
    ComposeTab t;
    for (int c = 0; c < cnt; ++c) t.d[c] = d[c0 + c];
    const dim3 g(blocks_for(vox(n)), groups(cnt, nf));
    if (nf == 1)
      k_compose<1><<<g, kThreads, 0, s>>>(t, n, cnt);
    else
      k_compose<2><<<g, kThreads, 0, s>>>(t, n, cnt);
  }
}
template <int NF>
void compose_bwd_nf(const ComposeBwdTab& t, int n_chains, Dims n, const FxArgs* fx, cudaStream_t s) {
  if (fx)
    k_compose_bwd<true, NF><<<grid2(n, n_chains, NF), kThreads, 0, s>>>(t, n, n_chains, *fx);
  else
    k_compose_bwd<false, NF><<<dim3(blocks_for(vox(n)), groups(n_chains, NF)), kThreads, 0, s>>>(t, n, n_chains,
                                                                                               FxArgs{});
}
void launch_compose_bwd(const ComposeBwdDesc* d, int n_chains, Dims n, const FxArgs* fx, cudaStream_t s, int nf) {
  for (int c0 = 0; c0 < n_chains; c0 += kMaxDescPerLaunch) {
    const int cnt = std::min(kMaxDescPerLaunch, n_chains - c0);
    ComposeBwdTab t;
    for (int c = 0; c < cnt; ++c) t.d[c] = d[c0 + c];
    if (fx && dz_fits(n, cnt))
      k_compose_bwd_dz<<<grid_dz(n, cnt), kThreads, 0, s>>>(t, n, *fx);
    else if (fx_nf(fx, n, cnt, nf) == 1)
      compose_bwd_nf<1>(t, cnt, n, fx, s);
    else
      compose_bwd_nf<2>(t, cnt, n, fx, s);
  }
}
void launch_add(const AddDesc* d, int n, Dims dims, cudaStream_t s) {
  for (int c0 = 0; c0 < n; c0 += kMaxDescPerLaunch) {
    const int cnt = std::min(kMaxDescPerLaunch, n - c0);
    AddTab t;
    for (int c = 0; c < cnt; ++c) t.d[c] = d[c0 + c];
    k_add<<<dim3(blocks_for(vox(dims)), cnt), kThreads, 0, s>>>(t, (int)vox(dims));
  }
}
int reg_blocks(Dims n) { return (int)blocks_for(vox(n)); }
void launch_reg_grad(const float4* theta, const float4* G0, float4* grad, double* partials, Dims n,
                     const RegArgs& a, const FxArgs* fx, cudaStream_t s, bool clear_g0) {
  const dim3 g(blocks_for(vox(n)), a.n_fields);
  if (clear_g0 && G0)
    k_reg_grad<true><<<g, kThreads, 0, s>>>(theta, G0, grad, partials, n, a, fx ? *fx : FxArgs{},
                                             const_cast<float4*>(G0));
  else
    k_reg_grad<false><<<g, kThreads, 0, s>>>(theta, G0, grad, partials, n, a, fx ? *fx : FxArgs{}, nullptr);
}
void launch_smooth(const float4* in, float4* out, float4* tmp_a, float4* tmp_b, int n_fields, Dims n,
                   const SmoothAxis axes[3], cudaStream_t s) {
  const dim3 g(blocks_for(vox(n)), n_fields);
  k_smooth_axis<<<g, kThreads, 0, s>>>(in, tmp_a, n, 0, axes[0].taps, axes[0].lo, axes[0].hi);
  k_smooth_axis<<<g, kThreads, 0, s>>>(tmp_a, tmp_b, n, 1, axes[1].taps, axes[1].lo, axes[1].hi);
  k_smooth_axis<<<g, kThreads, 0, s>>>(tmp_b, out, n, 2, axes[2].taps, axes[2].lo, axes[2].hi);
}
void launch_adam(float4* theta, float4* m, float4* v, const float4* grad, size_t count, const float* sched,
                 const int* step, int sgd, float beta1, float beta2, float eps, cudaStream_t s) {
  k_adam<<<blocks_for(count), kThreads, 0, s>>>(theta, m, v, grad, count, sched, step, sgd, beta1, beta2, eps);
}
void launch_f4_to_planar(const float4* in, float* out, int n_fields, size_t V, cudaStream_t s) {
  k_f4_to_planar<<<dim3(blocks_for(V), n_fields), kThreads, 0, s>>>(in, out, V);
}
void launch_planar_to_f4(const float* in, float4* out, int n_fields, size_t V, cudaStream_t s) {
  k_planar_to_f4<<<dim3(blocks_for(V), n_fields), kThreads, 0, s>>>(in, out, V);
}

}  // namespace muster
