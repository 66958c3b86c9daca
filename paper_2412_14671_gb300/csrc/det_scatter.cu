// det_scatter.cu -- deterministic transpose of trilinear sampling (the "scatter"
// half of the squaring and composition adjoints) without floating-point atomics.
//
// For each scatter group g (one field) every source voxel x has a sample point
// q(x) = x + pos_g(x) and a value val_g(x); the adjoint adds w_e(q) val_g(x) to
// the 8 corners of q's cell. Here the sources are bucketed by cell with a
// counting sort (integer counts, exclusive scan, fill, then each bucket sorted
// by source index), and every destination node gathers from the 8 cells that
// have it as a corner, in a fixed order. The sum for each node is therefore
// formed in the same order on every run: bit-reproducible.
#include "kernels.h"

namespace muster {

namespace {
constexpr int kThreads = 256;
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__host__ __device__ inline unsigned blocks_for(size_t V) { return (unsigned)((V + kThreads - 1) / kThreads); }

__global__ void k_det_count(const ScatterGroup* __restrict__ gr, Dims n, int* __restrict__ cell,
                            int* __restrict__ count) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int V = (int)vox(n);
  if (x >= V) return;
  const size_t base = (size_t)blockIdx.y * V;
  int z, y, xx;
  unflat(n, x, z, y, xx);
  const float4 p = gr[blockIdx.y].pos[x];
  const Corners k = corners_of(n, z + p.x, y + p.y, xx + p.z);
  cell[base + x] = k.o000;
  atomicAdd(count + base + k.o000, 1);
}

__global__ void k_det_fill(const int* __restrict__ cell, const int* __restrict__ offset, int* __restrict__ cursor,
                           int* __restrict__ list, int V) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= V) return;
  const size_t base = (size_t)blockIdx.y * V;
  const size_t c = base + cell[base + x];
  list[offset[c] + atomicAdd(cursor + c, 1)] = x;
}

// each bucket sorted by source index (buckets are small: about one source per cell)
__global__ void k_det_sort(const int* __restrict__ offset, int* __restrict__ list, size_t ncells) {
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const int a = offset[c], b = offset[c + 1];
  for (int i = a + 1; i < b; ++i) {
    const int key = list[i];
    int j = i - 1;
    while (j >= a && list[j] > key) {
      list[j + 1] = list[j];
      --j;
    }
    list[j + 1] = key;
  }
}

__global__ void k_det_gather(const ScatterGroup* __restrict__ gr, Dims n, const int* __restrict__ offset,
                             const int* __restrict__ list) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  const int V = (int)vox(n);
  if (y >= V) return;
  const ScatterGroup g = gr[blockIdx.y];
  const size_t base = (size_t)blockIdx.y * V;
  int z0, y0, x0;
  unflat(n, y, z0, y0, x0);
  float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
  for (int e0 = 0; e0 < 2; ++e0) {
    const int cz = z0 - e0;
    if (cz < 0) continue;
#pragma unroll
    for (int e1 = 0; e1 < 2; ++e1) {
      const int cy = y0 - e1;
      if (cy < 0) continue;
#pragma unroll
      for (int e2 = 0; e2 < 2; ++e2) {
        const int cx = x0 - e2;
        if (cx < 0) continue;
        const size_t c = base + ((size_t)cz * n.n1 + cy) * n.n2 + cx;
        const int a = offset[c], b = offset[c + 1];
        for (int s = a; s < b; ++s) {
          const int src = list[s];
          int sz, sy, sx;
          unflat(n, src, sz, sy, sx);
          const float4 p = g.pos[src];
          const Corners k = corners_of(n, sz + p.x, sy + p.y, sx + p.z);
          const float w = (e0 ? k.t0 : 1.f - k.t0) * (e1 ? k.t1 : 1.f - k.t1) * (e2 ? k.t2 : 1.f - k.t2);
          const float4 v = g.val[src];
          ax = fmaf(w, v.x, ax);
          ay = fmaf(w, v.y, ay);
          az = fmaf(w, v.z, az);
        }
      }
    }
  }
  float4 d = g.dst[y];
  d.x += ax;
  d.y += ay;
  d.z += az;
  g.dst[y] = d;
}

// ---- exclusive scan of int32 (fixed order, three phases)
__device__ __forceinline__ int warp_incl(int v) {
  const int l = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (l >= o) v += t;
  }
  return v;
}

__global__ void k_scan_tiles(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ tile_sum, size_t n) {
  __shared__ int ws[kScanThreads / 32];
  const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  int v[kScanItems], s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += v[i];
  }
  const int incl = warp_incl(s);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 31) ws[w] = incl;
  __syncthreads();
  if (w == 0) {
    int t = l < kScanThreads / 32 ? ws[l] : 0;
    t = warp_incl(t);
    if (l < kScanThreads / 32) ws[l] = t;
  }
  __syncthreads();
  int run = incl - s + (w > 0 ? ws[w - 1] : 0);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == kScanThreads - 1) tile_sum[blockIdx.x] = run;
}

__global__ void k_scan_add(int* __restrict__ out, const int* __restrict__ tile_off, size_t n) {
  const size_t i = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  const int add = tile_off[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (i + k < n) out[i + k] += add;
}

__global__ void k_set_total(int* __restrict__ out, size_t n, const int* __restrict__ in) {
  // out[n] = out[n-1] + in[n-1]
  out[n] = out[n - 1] + in[n - 1];
}
}  // namespace

size_t scan_scratch_ints(size_t n) {
  const size_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles <= 1) return 2;
  return 2 * tiles + 2 + scan_scratch_ints(tiles);
}

// exclusive scan of in[0, n) into out[0, n], out[n] = total; scratch from scan_scratch_ints(n)
void launch_scan(const int* in, int* out, size_t n, int* scratch, cudaStream_t s) {
  const size_t tiles = (n + kScanTile - 1) / kScanTile;
  int* sums = scratch;
  int* sums_scan = scratch + tiles + 1;
  k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, sums, n);
  if (tiles > 1) {
    launch_scan(sums, sums_scan, tiles, sums_scan + tiles + 1, s);
    k_scan_add<<<(unsigned)tiles, kScanThreads, 0, s>>>(out, sums_scan, n);
  }
  k_set_total<<<1, 1, 0, s>>>(out, n, in);
}

void det_scatter(const ScatterGroup* groups, int n_groups, Dims n, const DetScratch& w, cudaStream_t s) {
  if (n_groups <= 0) return;
  const size_t V = vox(n), total = V * n_groups;
  cudaMemsetAsync(w.count, 0, sizeof(int) * total, s);
  k_det_count<<<dim3(blocks_for(V), n_groups), kThreads, 0, s>>>(groups, n, w.cell, w.count);
  launch_scan(w.count, w.offset, total, w.scan, s);
  cudaMemsetAsync(w.count, 0, sizeof(int) * total, s);
  k_det_fill<<<dim3(blocks_for(V), n_groups), kThreads, 0, s>>>(w.cell, w.offset, w.count, w.list, (int)V);
  k_det_sort<<<blocks_for(total), kThreads, 0, s>>>(w.offset, w.list, total);
  k_det_gather<<<dim3(blocks_for(V), n_groups), kThreads, 0, s>>>(groups, n, w.offset, w.list);
}

}  // namespace muster
