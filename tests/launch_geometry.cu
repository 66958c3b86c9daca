// Host-only check of the launch geometry of the image-grid kernels (no device needed; the SM
// count falls back to GB300's 152 without one). The engine sizes the per-CTA partial-sum
// buffers and the pair batch from the geometry at a batch of one pair, and launches with its
// real batch, so for every shape, window and batch:
//   - the D chunks of the window-sum kernels cover the depth exactly once (tz >= 1,
//     nzc * tz >= D > (nzc - 1) * tz);
//   - a larger batch never needs more chunks or more CTAs per pair than a batch of one;
//   - the same holds for the D chunks and CTAs per pair of the warp adjoint on the flow grid.
// Prints the number of cases checked and exits non-zero on the first violation.
#include <cstdio>

#include "kernels.h"

using namespace muster;

static int fail(const char* what, Dims n, int w, int b) {
  std::printf("FAIL %s at D=%d H=%d W=%d window=%d batch=%d\n", what, n.n0, n.n1, n.n2, w, b);
  return 1;
}

int main() {
  const int sizes[] = {1, 2, 3, 5, 8, 17, 20, 24, 40, 48, 64, 80, 96, 128, 160, 192, 224, 256, 511, 1024, 4096};
  const int windows[] = {3, 5, 7, 9, 11};
  const int batches[] = {1, 2, 3, 7, 30, 90, 132, 240, 992};
  long checked = 0;
  for (int D : sizes)
    for (int H : sizes)
      for (int W : sizes) {
        const Dims n{D, H, W};
        const Dims nf{(D + 1) / 2, (H + 1) / 2, (W + 1) / 2};
        const int z1 = warp_bwd_zchunks(nf, 1), c1 = warp_bwd_ctas_per_pair(nf, 1);
        for (int w : windows) {
          const SimGeom g1 = sim_geom(n, w, 1);
          for (int b : batches) {
            const SimGeom g = sim_geom(n, w, b);
            if (g.tz < 1 || (long)g.nzc * g.tz < D || (long)(g.nzc - 1) * g.tz >= D) return fail("chunk cover", n, w, b);
            if (g.nzc > g1.nzc || g.ctas > g1.ctas) return fail("sim chunks above batch 1", n, w, b);
            const int zb = warp_bwd_zchunks(nf, b), cb = warp_bwd_ctas_per_pair(nf, b);
            if (zb < 1 || zb > nf.n0 || zb > z1 || cb > c1 || cb < 1) return fail("warp adjoint chunks", n, w, b);
            ++checked;
          }
        }
      }
  std::printf("GEOMETRY-OK %ld\n", checked);
  return 0;
}
