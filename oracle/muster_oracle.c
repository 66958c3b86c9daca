/*
 * muster_oracle.c -- FP64 CPU oracle of MUSTER's per-iteration registration loop
 * (Grodem et al., "MUSTER: Longitudinal Deformable Registration by Composition
 * of Consecutive Deformations", arXiv 2412.14671).
 *
 * TEST INFRASTRUCTURE. This file is the slow, literal restatement of the method
 * that the CUDA library is checked against. Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark load it. It shares no code, header,
 * table or helper with the CUDA library.
 *
 * Each function follows the paper's definition in the paper's order. Where the
 * paper is silent or garbled, the reading taken is stated next to the code:
 *   - sampling S[g](q): index coordinates with voxel centres at integers, each
 *     coordinate clamped to [0, n-1] (clamp-to-edge), cell = floor of the clamped
 *     coordinate, upper node min(i0+1, n-1), trilinear weights; the derivative
 *     with respect to q uses that cell and is zero on a clamped side;
 *   - Alg. 1 runs exactly N_iter squarings in the displacement form given in
 *     its comment, u <- u + u o (x + u), starting from u = sign*phi/2^K;
 *   - compositions accumulate outward from the fixed session (Eq. cum_deformation
 *     with the intermediate session adjacent to the moving one);
 *   - velocities live on a grid f times coarser than the image (Sec.
 *     Implementation Details) and are integrated and composed there; the pair
 *     displacement is then upsampled with voxel-centre alignment
 *     q = (p + 1/2)/f - 1/2 and scaled by f;
 *   - similarity windows are the valid w^3 windows (all voxels inside the image);
 *     LNCC_R = 1 - S_FW/sqrt(S_FF*S_WW + eps), SiLNCC_R = (S_WW - S_FW^2/(S_FF + eps))/|R|
 *     with centred window sums (Eq. LNCC, the SiLNCC equation); the fixed image
 *     is the regressor;
 *   - regularisers are means over the flow grid in flow-voxel units; L_ts takes
 *     the rate difference phi_{i-1}/(t_i - t_{i-1}) - phi_i/(t_{i+1} - t_i);
 *   - Adam with the PyTorch update rule; warm-up over ceil(0.2 T) steps then
 *     cosine decay; optimiser state reset at each level.
 *
 * Parity pinned: see the header of oracle/__init__.py for the pin of each function.
 */
#include "muster_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI_D 3.14159265358979323846

static size_t nvox(const int n[3]) { return (size_t)n[0] * (size_t)n[1] * (size_t)n[2]; }
static size_t at(const int n[3], int z, int y, int x) {
  return ((size_t)z * (size_t)n[1] + (size_t)y) * (size_t)n[2] + (size_t)x;
}
static double* zalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

/* ---------------------------------------------------------------------------
 * Sampling operator (trilinear interpolation; Sec. Background, Eq. cum_deformation).
 * ------------------------------------------------------------------------- */
typedef struct {
  int i0, i1;
  double t;      /* fractional position inside the cell */
  double inside; /* 1 if q was inside [0, n-1], 0 if it was clamped */
} axis_cell;

static axis_cell cell_of(double q, int n) {
  axis_cell c;
  c.inside = 1.0;
  if (q < 0.0) {
    q = 0.0;
    c.inside = 0.0;
  }
  if (q > (double)(n - 1)) {
    q = (double)(n - 1);
    c.inside = 0.0;
  }
  double f = floor(q);
  c.i0 = (int)f;
  c.i1 = c.i0 + 1 < n ? c.i0 + 1 : n - 1;
  c.t = q - f;
  return c;
}

double or_sample(const double* g, const int n[3], const double q[3], double grad[3]) {
  axis_cell c[3];
  for (int a = 0; a < 3; ++a) c[a] = cell_of(q[a], n[a]);
  double v = 0.0, d0 = 0.0, d1 = 0.0, d2 = 0.0;
  for (int e0 = 0; e0 < 2; ++e0)
    for (int e1 = 0; e1 < 2; ++e1)
      for (int e2 = 0; e2 < 2; ++e2) {
        double val = g[at(n, e0 ? c[0].i1 : c[0].i0, e1 ? c[1].i1 : c[1].i0,
                          e2 ? c[2].i1 : c[2].i0)];
        double w0 = e0 ? c[0].t : 1.0 - c[0].t;
        double w1 = e1 ? c[1].t : 1.0 - c[1].t;
        double w2 = e2 ? c[2].t : 1.0 - c[2].t;
        v += w0 * w1 * w2 * val;
        d0 += (e0 ? 1.0 : -1.0) * w1 * w2 * val;
        d1 += w0 * (e1 ? 1.0 : -1.0) * w2 * val;
        d2 += w0 * w1 * (e2 ? 1.0 : -1.0) * val;
      }
  if (grad) {
    grad[0] = d0 * c[0].inside;
    grad[1] = d1 * c[1].inside;
    grad[2] = d2 * c[2].inside;
  }
  return v;
}

/* transpose of sampling with respect to the sampled values: acc[corner] += weight * value */
static void scatter(double* acc, const int n[3], const double q[3], double value) {
  axis_cell c[3];
  for (int a = 0; a < 3; ++a) c[a] = cell_of(q[a], n[a]);
  for (int e0 = 0; e0 < 2; ++e0)
    for (int e1 = 0; e1 < 2; ++e1)
      for (int e2 = 0; e2 < 2; ++e2) {
        double w0 = e0 ? c[0].t : 1.0 - c[0].t;
        double w1 = e1 ? c[1].t : 1.0 - c[1].t;
        double w2 = e2 ? c[2].t : 1.0 - c[2].t;
        acc[at(n, e0 ? c[0].i1 : c[0].i0, e1 ? c[1].i1 : c[1].i0, e2 ? c[2].i1 : c[2].i0)] +=
            w0 * w1 * w2 * value;
      }
}

/* S[u](x + U(x)) for a vector field u; J (nullable) = d/dq, J[c][a] */
static void sample_vec(const double* u, const int n[3], const double q[3], double out[3],
                       double J[3][3]) {
  size_t V = nvox(n);
  for (int c = 0; c < 3; ++c) out[c] = or_sample(u + c * V, n, q, J ? J[c] : NULL);
}

/* ---------------------------------------------------------------------------
 * Alg. 1: Exp(phi) by scaling and squaring, displacement form.
 * ------------------------------------------------------------------------- */
void or_exp(const double* phi, const int n[3], int K, double sign, double* u_out,
            double* inter) {
  size_t V = nvox(n);
  double* u = zalloc(3 * V);
  double* un = zalloc(3 * V);
  double scale = ldexp(sign, -K); /* sign / 2^K */
  for (size_t i = 0; i < 3 * V; ++i) u[i] = scale * phi[i];
  if (inter) memcpy(inter, u, 3 * V * sizeof(double));
  for (int s = 0; s < K; ++s) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < n[0]; ++z)
      for (int y = 0; y < n[1]; ++y)
        for (int x = 0; x < n[2]; ++x) {
          size_t i = at(n, z, y, x);
          double q[3] = {z + u[i], y + u[V + i], x + u[2 * V + i]};
          double s3[3];
          sample_vec(u, n, q, s3, NULL);
          for (int c = 0; c < 3; ++c) un[c * V + i] = u[c * V + i] + s3[c];
        }
    double* tmp = u;
    u = un;
    un = tmp;
    if (inter) memcpy(inter + (size_t)(s + 1) * 3 * V, u, 3 * V * sizeof(double));
  }
  memcpy(u_out, u, 3 * V * sizeof(double));
  free(u);
  free(un);
}

/* Reverse of the K squarings: u_{s+1}(x) = u_s(x) + S[u_s](x + u_s(x)) gives
   g_s(x) = g_{s+1}(x) + J^T g_{s+1}(x)   (through the sample point)
   g_s(y) += sum_x w(y; x + u_s(x)) g_{s+1}(x)   (through the sampled values). */
void or_exp_adjoint(const double* phi, const int n[3], int K, double sign, const double* g_u,
                    double* g_phi) {
  size_t V = nvox(n);
  double* inter = zalloc((size_t)(K + 1) * 3 * V);
  double* u = zalloc(3 * V);
  or_exp(phi, n, K, sign, u, inter);
  double* G = zalloc(3 * V);
  double* Gp = zalloc(3 * V);
  memcpy(G, g_u, 3 * V * sizeof(double));
  for (int s = K - 1; s >= 0; --s) {
    const double* us = inter + (size_t)s * 3 * V;
    memcpy(Gp, G, 3 * V * sizeof(double));
    for (int z = 0; z < n[0]; ++z)
      for (int y = 0; y < n[1]; ++y)
        for (int x = 0; x < n[2]; ++x) {
          size_t i = at(n, z, y, x);
          double q[3] = {z + us[i], y + us[V + i], x + us[2 * V + i]};
          double val[3], J[3][3];
          sample_vec(us, n, q, val, J);
          for (int a = 0; a < 3; ++a) {
            double acc = 0.0;
            for (int c = 0; c < 3; ++c) acc += J[c][a] * G[c * V + i];
            Gp[a * V + i] += acc;
          }
          for (int c = 0; c < 3; ++c) scatter(Gp + c * V, n, q, G[c * V + i]);
        }
    double* tmp = G;
    G = Gp;
    Gp = tmp;
  }
  double scale = ldexp(sign, -K);
  for (size_t i = 0; i < 3 * V; ++i) g_phi[i] = scale * G[i];
  free(inter);
  free(u);
  free(G);
  free(Gp);
}

/* ---------------------------------------------------------------------------
 * Eq. cum_deformation: Phi_ki = Phi_ji + (Phi_kj - Omega) o Phi_ji, with the
 * intermediate session j next to k, accumulated outward from the fixed session i.
 * ------------------------------------------------------------------------- */
static double* pair_ptr(double* U, int N, int k, int i, size_t V) {
  return U + ((size_t)k * N + i) * 3 * V;
}

/* Unew(x) = Uprev(x) + S[u](x + Uprev(x)) */
static void compose_step(const double* Uprev, const double* u, const int n[3], double* Unew) {
  size_t V = nvox(n);
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < n[0]; ++z)
    for (int y = 0; y < n[1]; ++y)
      for (int x = 0; x < n[2]; ++x) {
        size_t i = at(n, z, y, x);
        double q[3] = {z + Uprev[i], y + Uprev[V + i], x + Uprev[2 * V + i]};
        double s3[3];
        sample_vec(u, n, q, s3, NULL);
        for (int c = 0; c < 3; ++c) Unew[c * V + i] = Uprev[c * V + i] + s3[c];
      }
}

void or_compose(const double* up, const double* um, int N, const int n[3], double* U) {
  size_t V = nvox(n);
  memset(U, 0, (size_t)N * N * 3 * V * sizeof(double));
  for (int i = 0; i < N; ++i) {
    /* sessions after i: Phi_{i+1,i} = Exp(phi_i); then through k-1 */
    if (i + 1 < N) memcpy(pair_ptr(U, N, i + 1, i, V), up + (size_t)i * 3 * V, 3 * V * sizeof(double));
    for (int k = i + 2; k < N; ++k)
      compose_step(pair_ptr(U, N, k - 1, i, V), up + (size_t)(k - 1) * 3 * V, n,
                   pair_ptr(U, N, k, i, V));
    /* sessions before i: Phi_{i-1,i} = Exp(-phi_{i-1}); then through k+1 */
    if (i - 1 >= 0)
      memcpy(pair_ptr(U, N, i - 1, i, V), um + (size_t)(i - 1) * 3 * V, 3 * V * sizeof(double));
    for (int k = i - 2; k >= 0; --k)
      compose_step(pair_ptr(U, N, k + 1, i, V), um + (size_t)k * 3 * V, n,
                   pair_ptr(U, N, k, i, V));
  }
}

/* reverse of one compose_step: Gprev += G + J^T G ; g_field += scatter(G) */
static void compose_step_adjoint(const double* Uprev, const double* u, const int n[3],
                                 const double* G, double* Gprev, double* g_field) {
  size_t V = nvox(n);
  for (int z = 0; z < n[0]; ++z)
    for (int y = 0; y < n[1]; ++y)
      for (int x = 0; x < n[2]; ++x) {
        size_t i = at(n, z, y, x);
        double q[3] = {z + Uprev[i], y + Uprev[V + i], x + Uprev[2 * V + i]};
        double val[3], J[3][3];
        sample_vec(u, n, q, val, J);
        for (int a = 0; a < 3; ++a) {
          double acc = G[a * V + i];
          for (int c = 0; c < 3; ++c) acc += J[c][a] * G[c * V + i];
          Gprev[a * V + i] += acc;
        }
        for (int c = 0; c < 3; ++c) scatter(g_field + c * V, n, q, G[c * V + i]);
      }
}

void or_compose_adjoint(const double* up, const double* um, int N, const int n[3],
                        const double* gU, double* g_up, double* g_um) {
  size_t V = nvox(n);
  size_t tot = (size_t)N * N * 3 * V;
  double* U = zalloc(tot);
  double* G = zalloc(tot);
  or_compose(up, um, N, n, U);
  memcpy(G, gU, tot * sizeof(double));
  memset(g_up, 0, (size_t)(N - 1) * 3 * V * sizeof(double));
  memset(g_um, 0, (size_t)(N - 1) * 3 * V * sizeof(double));
  for (int i = 0; i < N; ++i) {
    for (int k = N - 1; k >= i + 2; --k)
      compose_step_adjoint(pair_ptr(U, N, k - 1, i, V), up + (size_t)(k - 1) * 3 * V, n,
                           pair_ptr(G, N, k, i, V), pair_ptr(G, N, k - 1, i, V),
                           g_up + (size_t)(k - 1) * 3 * V);
    if (i + 1 < N) {
      const double* Gd = pair_ptr(G, N, i + 1, i, V);
      double* dst = g_up + (size_t)i * 3 * V;
      for (size_t e = 0; e < 3 * V; ++e) dst[e] += Gd[e];
    }
    for (int k = 0; k <= i - 2; ++k)
      compose_step_adjoint(pair_ptr(U, N, k + 1, i, V), um + (size_t)k * 3 * V, n,
                           pair_ptr(G, N, k, i, V), pair_ptr(G, N, k + 1, i, V),
                           g_um + (size_t)k * 3 * V);
    if (i - 1 >= 0) {
      const double* Gd = pair_ptr(G, N, i - 1, i, V);
      double* dst = g_um + (size_t)(i - 1) * 3 * V;
      for (size_t e = 0; e < 3 * V; ++e) dst[e] += Gd[e];
    }
  }
  free(U);
  free(G);
}

/* ---------------------------------------------------------------------------
 * Flow grid -> image grid (Sec. Implementation Details: flows at a coarser grid).
 * ------------------------------------------------------------------------- */
static double centre_map(int p, int f) { return ((double)p + 0.5) / (double)f - 0.5; }

void or_upsample(const double* U, const int nf[3], const int ni[3], int f, double* Ut) {
  size_t Vf = nvox(nf), Vi = nvox(ni);
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < ni[0]; ++z)
    for (int y = 0; y < ni[1]; ++y)
      for (int x = 0; x < ni[2]; ++x) {
        double q[3] = {centre_map(z, f), centre_map(y, f), centre_map(x, f)};
        size_t i = at(ni, z, y, x);
        for (int c = 0; c < 3; ++c) Ut[c * Vi + i] = (double)f * or_sample(U + c * Vf, nf, q, NULL);
      }
}

void or_upsample_adjoint(const double* gUt, const int nf[3], const int ni[3], int f,
                         double* gU) {
  size_t Vf = nvox(nf), Vi = nvox(ni);
  memset(gU, 0, 3 * Vf * sizeof(double));
  for (int z = 0; z < ni[0]; ++z)
    for (int y = 0; y < ni[1]; ++y)
      for (int x = 0; x < ni[2]; ++x) {
        double q[3] = {centre_map(z, f), centre_map(y, f), centre_map(x, f)};
        size_t i = at(ni, z, y, x);
        for (int c = 0; c < 3; ++c) scatter(gU + c * Vf, nf, q, (double)f * gUt[c * Vi + i]);
      }
}

/* I_j o Phi_ji^i by trilinear interpolation (Sec. Background) */
void or_warp(const double* I, const int ni[3], const double* Ut, double* W) {
  size_t Vi = nvox(ni);
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < ni[0]; ++z)
    for (int y = 0; y < ni[1]; ++y)
      for (int x = 0; x < ni[2]; ++x) {
        size_t i = at(ni, z, y, x);
        double q[3] = {z + Ut[i], y + Ut[Vi + i], x + Ut[2 * Vi + i]};
        W[i] = or_sample(I, ni, q, NULL);
      }
}

void or_warp_adjoint(const double* I, const int ni[3], const double* Ut, const double* gW,
                     double* gUt) {
  size_t Vi = nvox(ni);
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < ni[0]; ++z)
    for (int y = 0; y < ni[1]; ++y)
      for (int x = 0; x < ni[2]; ++x) {
        size_t i = at(ni, z, y, x);
        double q[3] = {z + Ut[i], y + Ut[Vi + i], x + Ut[2 * Vi + i]};
        double d[3];
        or_sample(I, ni, q, d);
        for (int c = 0; c < 3; ++c) gUt[c * Vi + i] = gW[i] * d[c];
      }
}

/* ---------------------------------------------------------------------------
 * Eq. LNCC, Eq. sum_lncc, the SiLNCC equation and Eq. sim_loss.
 * ------------------------------------------------------------------------- */
static int window_grid(const int n[3], int w, int m[3]) {
  int ok = 1;
  for (int a = 0; a < 3; ++a) {
    m[a] = n[a] - w + 1;
    if (m[a] < 1) ok = 0;
  }
  return ok;
}

void or_window_stats(const double* F, const double* W, const int n[3], int w, double* muF,
                     double* muW, double* Sff, double* Sww, double* Sfw) {
  int m[3];
  if (!window_grid(n, w, m)) return;
  int r = w / 2;
  double nw = (double)w * w * w;
#pragma omp parallel for collapse(2) schedule(static)
  for (int cz = 0; cz < m[0]; ++cz)
    for (int cy = 0; cy < m[1]; ++cy)
      for (int cx = 0; cx < m[2]; ++cx) {
        int z0 = cz, y0 = cy, x0 = cx; /* window = [c, c + w) in voxel indices, centre c + r */
        (void)r;
        double sf = 0.0, sw = 0.0;
        for (int dz = 0; dz < w; ++dz)
          for (int dy = 0; dy < w; ++dy)
            for (int dx = 0; dx < w; ++dx) {
              size_t i = at(n, z0 + dz, y0 + dy, x0 + dx);
              sf += F[i];
              sw += W[i];
            }
        double mf = sf / nw, mw = sw / nw;
        double ff = 0.0, ww = 0.0, fw = 0.0;
        for (int dz = 0; dz < w; ++dz)
          for (int dy = 0; dy < w; ++dy)
            for (int dx = 0; dx < w; ++dx) {
              size_t i = at(n, z0 + dz, y0 + dy, x0 + dx);
              double a = F[i] - mf, b = W[i] - mw;
              ff += a * a;
              ww += b * b;
              fw += a * b;
            }
        size_t o = at(m, cz, cy, cx);
        if (muF) muF[o] = mf;
        if (muW) muW[o] = mw;
        if (Sff) Sff[o] = ff;
        if (Sww) Sww[o] = ww;
        if (Sfw) Sfw[o] = fw;
      }
}

double or_similarity(const double* F, const double* W, const int n[3], int w, int kind,
                     double eps, double* dW) {
  int m[3];
  size_t V = nvox(n);
  if (!window_grid(n, w, m)) {
    if (dW) memset(dW, 0, V * sizeof(double));
    return 0.0;
  }
  size_t NR = nvox(m);
  double nw = (double)w * w * w;
  double *muF = zalloc(NR), *muW = zalloc(NR), *Sff = zalloc(NR), *Sww = zalloc(NR),
         *Sfw = zalloc(NR);
  double *c1 = zalloc(NR), *c2 = zalloc(NR);
  or_window_stats(F, W, n, w, muF, muW, Sff, Sww, Sfw);
  double total = 0.0;
  for (size_t R = 0; R < NR; ++R) {
    if (kind == OR_SILNCC) {
      double beta = Sfw[R] / (Sff[R] + eps);
      total += (Sww[R] - Sfw[R] * Sfw[R] / (Sff[R] + eps)) / nw;
      /* d SiLNCC_R / d W(p) = (2/|R|) (Wbar(p) - beta Fbar(p)) */
      c1[R] = 2.0 / nw;
      c2[R] = 2.0 / nw * beta;
    } else {
      double Q = Sff[R] * Sww[R] + eps;
      total += 1.0 - Sfw[R] / sqrt(Q);
      /* d LNCC_R / d W(p) = S_FW S_FF Wbar(p) / Q^{3/2} - Fbar(p) / sqrt(Q) */
      c1[R] = Sfw[R] * Sff[R] / (Q * sqrt(Q));
      c2[R] = 1.0 / sqrt(Q);
    }
  }
  if (dW) {
    int r = w / 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < n[0]; ++z)
      for (int y = 0; y < n[1]; ++y)
        for (int x = 0; x < n[2]; ++x) {
          /* windows [c, c+w) containing p: c in [p - w + 1, p], inside the centre grid */
          int p[3] = {z, y, x}, lo[3], hi[3];
          for (int a = 0; a < 3; ++a) {
            lo[a] = p[a] - w + 1 > 0 ? p[a] - w + 1 : 0;
            hi[a] = p[a] < m[a] - 1 ? p[a] : m[a] - 1;
          }
          (void)r;
          size_t i = at(n, z, y, x);
          double acc = 0.0;
          for (int cz = lo[0]; cz <= hi[0]; ++cz)
            for (int cy = lo[1]; cy <= hi[1]; ++cy)
              for (int cx = lo[2]; cx <= hi[2]; ++cx) {
                size_t R = at(m, cz, cy, cx);
                acc += c1[R] * (W[i] - muW[R]) - c2[R] * (F[i] - muF[R]);
              }
          dW[i] = acc / (double)NR;
        }
  }
  free(muF);
  free(muW);
  free(Sff);
  free(Sww);
  free(Sfw);
  free(c1);
  free(c2);
  return total / (double)NR;
}

/* ---------------------------------------------------------------------------
 * Eq. reg_ss, the L2 loss, Eq. reg_ts and Eq. reg_sum.
 * ------------------------------------------------------------------------- */
void or_regulariser(const double* phi, int N, const int n[3], const double* t, double a_ss,
                    double a_l2, double a_ts, double L[3], double* grad) {
  size_t V = nvox(n);
  int F = N - 1;
  L[0] = L[1] = L[2] = 0.0;
  if (grad) memset(grad, 0, (size_t)F * 3 * V * sizeof(double));
  if (F < 1) return;
  /* L_ss: mean over valid forward differences along each axis */
  for (int mf = 0; mf < F; ++mf)
    for (int c = 0; c < 3; ++c) {
      const double* p = phi + ((size_t)mf * 3 + c) * V;
      double* g = grad ? grad + ((size_t)mf * 3 + c) * V : NULL;
      for (int a = 0; a < 3; ++a) {
        if (n[a] < 2) continue;
        double M = (double)V / n[a] * (n[a] - 1);
        double acc = 0.0;
        for (int z = 0; z < n[0]; ++z)
          for (int y = 0; y < n[1]; ++y)
            for (int x = 0; x < n[2]; ++x) {
              int pp[3] = {z, y, x};
              if (pp[a] + 1 >= n[a]) continue;
              int qq[3] = {z, y, x};
              qq[a] += 1;
              size_t i0 = at(n, z, y, x), i1 = at(n, qq[0], qq[1], qq[2]);
              double d = p[i1] - p[i0];
              acc += d * d;
              if (g) {
                double s = a_ss * 2.0 * d / M / (double)F;
                g[i1] += s;
                g[i0] -= s;
              }
            }
        L[0] += acc / M / (double)F;
      }
    }
  /* L_L2 */
  for (int mf = 0; mf < F; ++mf)
    for (size_t e = 0; e < 3 * V; ++e) {
      double v = phi[(size_t)mf * 3 * V + e];
      L[1] += v * v / (double)V / (double)F;
      if (grad) grad[(size_t)mf * 3 * V + e] += a_l2 * 2.0 * v / (double)V / (double)F;
    }
  /* L_ts: sessions i = 1..N-2 (0-based) have a flow on both sides */
  if (N >= 3) {
    for (int i = 1; i <= N - 2; ++i) {
      double dtm = t[i] - t[i - 1], dtp = t[i + 1] - t[i];
      const double* a = phi + (size_t)(i - 1) * 3 * V;
      const double* b = phi + (size_t)i * 3 * V;
      for (size_t e = 0; e < 3 * V; ++e) {
        double r = a[e] / dtm - b[e] / dtp;
        L[2] += r * r / (double)V / (double)(N - 2);
        if (grad) {
          double s = a_ts * 2.0 * r / (double)V / (double)(N - 2);
          grad[(size_t)(i - 1) * 3 * V + e] += s / dtm;
          grad[(size_t)i * 3 * V + e] -= s / dtp;
        }
      }
    }
  }
}

/* ---------------------------------------------------------------------------
 * Multi-resolution pyramid (Sec. Implementation Details).
 * ------------------------------------------------------------------------- */
void or_downsample2(const double* in, const int n[3], double* out) {
  int m[3] = {(n[0] + 1) / 2, (n[1] + 1) / 2, (n[2] + 1) / 2};
  for (int z = 0; z < m[0]; ++z)
    for (int y = 0; y < m[1]; ++y)
      for (int x = 0; x < m[2]; ++x) {
        double s = 0.0;
        for (int e0 = 0; e0 < 2; ++e0)
          for (int e1 = 0; e1 < 2; ++e1)
            for (int e2 = 0; e2 < 2; ++e2) {
              int zz = 2 * z + e0, yy = 2 * y + e1, xx = 2 * x + e2;
              if (zz > n[0] - 1) zz = n[0] - 1;
              if (yy > n[1] - 1) yy = n[1] - 1;
              if (xx > n[2] - 1) xx = n[2] - 1;
              s += in[at(n, zz, yy, xx)];
            }
        out[at(m, z, y, x)] = s / 8.0;
      }
}

void or_prolong(const double* v, const int nc[3], const int nf[3], double* out) {
  size_t Vc = nvox(nc), Vf = nvox(nf);
  for (int z = 0; z < nf[0]; ++z)
    for (int y = 0; y < nf[1]; ++y)
      for (int x = 0; x < nf[2]; ++x) {
        double q[3] = {centre_map(z, 2), centre_map(y, 2), centre_map(x, 2)};
        for (int c = 0; c < 3; ++c)
          out[c * Vf + at(nf, z, y, x)] = 2.0 * or_sample(v + c * Vc, nc, q, NULL);
      }
}

void or_level_dims(const int n[3], int n_levels, int level, int flow_factor, int ni[3],
                   int nf[3]) {
  for (int a = 0; a < 3; ++a) {
    int s = n[a];
    for (int l = n_levels - 1; l > level; --l) s = (s + 1) / 2;
    ni[a] = s;
    nf[a] = (s + flow_factor - 1) / flow_factor;
  }
}

/* ---------------------------------------------------------------------------
 * Total loss (Sec. MUSTER overview) and its gradient, in the paper's order:
 * Exp of +-phi, composition, warp of every ordered pair, similarity, regulariser.
 * ------------------------------------------------------------------------- */
/* ------------------------------------------------------------------------------------------
 * Appendix Gaussian Smoothing: exp(-1/2 (f/omega)^2) on the DFT, f in cycles per mm */
static const double kPi = 3.14159265358979323846;

static double dft_freq(int j, int n, double h) { /* numpy.fft.fftfreq(n, d=h)[j] */
  return (double)(j < (n + 1) / 2 ? j : j - n) / ((double)n * h);
}

void or_smooth(const double* in, const int n[3], const double h[3], double omega, double* out) {
  const size_t V = nvox(n);
  double* a = zalloc(V);
  double* b = zalloc(V);
  memcpy(a, in, V * sizeof(double));
  for (int ax = 0; ax < 3; ++ax) {
    const int m = n[ax];
    /* taps of the circular convolution: inverse DFT of the (real, even) response */
    double* tap = zalloc((size_t)m);
    for (int d = 0; d < m; ++d) {
      double acc = 0.0;
      for (int j = 0; j < m; ++j) {
        const double f = dft_freq(j, m, h[ax]);
        acc += exp(-0.5 * (f / omega) * (f / omega)) * cos(2.0 * kPi * (double)j * (double)d / (double)m);
      }
      tap[d] = acc / (double)m;
    }
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < n[0]; ++z)
      for (int y = 0; y < n[1]; ++y)
        for (int x = 0; x < n[2]; ++x) {
          int p[3] = {z, y, x};
          double acc = 0.0;
          for (int d = 0; d < m; ++d) {
            int q[3] = {z, y, x};
            q[ax] = ((p[ax] - d) % m + m) % m;
            acc += tap[d] * a[at(n, q[0], q[1], q[2])];
          }
          b[at(n, z, y, x)] = acc;
        }
    free(tap);
    double* t = a;
    a = b;
    b = t;
  }
  memcpy(out, a, V * sizeof(double));
  free(a);
  free(b);
}

static double loss_grad_phi(const double* imgs, int N, const int ni[3], const double* phi,
                            const int nf[3], const or_params* p, const double* t, const double* rho,
                            double tscale, double split[4], double* grad, double* grad_rho);

/* ------------------------------------------------------------------------------------------
 * Sec. Rigid Registration: R = R_0(a0) R_1(a1) R_2(a2), R_a rotating the plane of the two
 * other axes (a+1, a+2 mod 3) by a */
static void axis_rotation(int a, double ang, double M[9], double dM[9]) {
  const double c = cos(ang), s = sin(ang);
  for (int k = 0; k < 9; ++k) M[k] = dM[k] = 0.0;
  const int u = (a + 1) % 3, w = (a + 2) % 3;
  M[3 * a + a] = 1.0;
  M[3 * u + u] = c;
  M[3 * u + w] = -s;
  M[3 * w + u] = s;
  M[3 * w + w] = c;
  dM[3 * u + u] = -s;
  dM[3 * u + w] = -c;
  dM[3 * w + u] = c;
  dM[3 * w + w] = -s;
}
static void mat3_mul(const double A[9], const double B[9], double C[9]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}
void or_rotation(const double a[3], double R[9], double dR[27]) {
  double M[3][9], dM[3][9], T[9];
  for (int k = 0; k < 3; ++k) axis_rotation(k, a[k], M[k], dM[k]);
  mat3_mul(M[0], M[1], T);
  mat3_mul(T, M[2], R);
  if (!dR) return;
  for (int k = 0; k < 3; ++k) {
    const double* A0 = k == 0 ? dM[0] : M[0];
    const double* A1 = k == 1 ? dM[1] : M[1];
    const double* A2 = k == 2 ? dM[2] : M[2];
    mat3_mul(A0, A1, T);
    mat3_mul(T, A2, dR + 9 * k);
  }
}

double or_loss_grad(const double* imgs, int N, const int ni[3], const double* theta,
                    const int nf[3], const or_params* p, const double* t, double split[4],
                    double* grad) {
  return or_loss_grad_rigid(imgs, N, ni, theta, nf, p, t, NULL, 1.0, split, grad, NULL);
}

double or_loss_grad_rigid(const double* imgs, int N, const int ni[3], const double* theta,
                          const int nf[3], const or_params* p, const double* t, const double* rho,
                          double tscale, double split[4], double* grad, double* grad_rho) {
  if (!(p->smooth_omega > 0.0))
    return loss_grad_phi(imgs, N, ni, theta, nf, p, t, rho, tscale, split, grad, grad_rho);
  /* phi = S(theta) per component; dL/dtheta = S(dL/dphi) (S is symmetric) */
  const size_t Vf = nvox(nf), n = (size_t)(N - 1) * 3;
  const double h[3] = {p->spacing[0] * p->flow_factor, p->spacing[1] * p->flow_factor,
                       p->spacing[2] * p->flow_factor};
  double* phi = zalloc(n * Vf);
  for (size_t c = 0; c < n; ++c) or_smooth(theta + c * Vf, nf, h, p->smooth_omega, phi + c * Vf);
  double* gphi = grad ? zalloc(n * Vf) : NULL;
  const double total = loss_grad_phi(imgs, N, ni, phi, nf, p, t, rho, tscale, split, gphi, grad_rho);
  if (grad)
    for (size_t c = 0; c < n; ++c) or_smooth(gphi + c * Vf, nf, h, p->smooth_omega, grad + c * Vf);
  free(phi);
  free(gphi);
  return total;
}

static double loss_grad_phi(const double* imgs, int N, const int ni[3], const double* phi,
                            const int nf[3], const or_params* p, const double* t, const double* rho,
                            double tscale, double split[4], double* grad, double* grad_rho) {
  size_t Vi = nvox(ni), Vf = nvox(nf);
  int F = N - 1, f = p->flow_factor;
  double* up = zalloc((size_t)F * 3 * Vf);
  double* um = zalloc((size_t)F * 3 * Vf);
  for (int m = 0; m < F; ++m) {
    or_exp(phi + (size_t)m * 3 * Vf, nf, p->K, +1.0, up + (size_t)m * 3 * Vf, NULL);
    or_exp(phi + (size_t)m * 3 * Vf, nf, p->K, -1.0, um + (size_t)m * 3 * Vf, NULL);
  }
  double* U = zalloc((size_t)N * N * 3 * Vf);
  or_compose(up, um, N, nf, U);
  double* gU = grad ? zalloc((size_t)N * N * 3 * Vf) : NULL;
  double* Ut = zalloc(3 * Vi);
  double* W = zalloc(Vi);
  double* dW = (grad || grad_rho) ? zalloc(Vi) : NULL;
  double* gUt = (grad || grad_rho) ? zalloc(3 * Vi) : NULL;
  double sim = 0.0;
  const double cen[3] = {0.5 * (ni[0] - 1), 0.5 * (ni[1] - 1), 0.5 * (ni[2] - 1)};
  double* Ur = rho ? zalloc(3 * Vi) : NULL; /* deformation plus the rigid part of grid i */
  if (grad_rho)
    for (size_t e = 0; e < (size_t)(N - 1) * 6; ++e) grad_rho[e] = 0.0;
  for (int i = 0; i < N; ++i) {
    double R[9], dR[27], GA[9] = {0}, gb[3] = {0};
    const int rigid_i = rho && i >= 1;
    if (rigid_i) or_rotation(rho + (size_t)(i - 1) * 6, R, dR);
    for (int k = 0; k < N; ++k) {
      if (k == i) continue;
      or_upsample(pair_ptr(U, N, k, i, Vf), nf, ni, f, Ut);
      const double* Uq = Ut;
      if (rigid_i) {
        /* Sec. Rigid Registration: Phi_total = Phi + (Phi_lin - identity) on grid i */
        const double* tr = rho + (size_t)(i - 1) * 6 + 3;
        for (int z = 0; z < ni[0]; ++z)
          for (int y = 0; y < ni[1]; ++y)
            for (int x = 0; x < ni[2]; ++x) {
              const size_t e = at(ni, z, y, x);
              const double d[3] = {z - cen[0], y - cen[1], x - cen[2]}, pp[3] = {z, y, x};
              for (int r = 0; r < 3; ++r)
                Ur[r * Vi + e] = Ut[r * Vi + e] + R[3 * r] * d[0] + R[3 * r + 1] * d[1] + R[3 * r + 2] * d[2] +
                                 cen[r] + tr[r] / tscale - pp[r];
            }
        Uq = Ur;
      }
      or_warp(imgs + (size_t)k * Vi, ni, Uq, W);
      sim += or_similarity(imgs + (size_t)i * Vi, W, ni, p->window, p->sim_kind, p->sim_eps, dW);
      if (grad || grad_rho) {
        double* g = gUt;
        or_warp_adjoint(imgs + (size_t)k * Vi, ni, Uq, dW, g);
        if (grad) or_upsample_adjoint(g, nf, ni, f, pair_ptr(gU, N, k, i, Vf));
        if (rigid_i && grad_rho)
          for (int z = 0; z < ni[0]; ++z)
            for (int y = 0; y < ni[1]; ++y)
              for (int x = 0; x < ni[2]; ++x) {
                const size_t e = at(ni, z, y, x);
                const double pp[3] = {z, y, x};
                for (int r = 0; r < 3; ++r) {
                  gb[r] += g[r * Vi + e];
                  for (int c = 0; c < 3; ++c) GA[3 * r + c] += g[r * Vi + e] * pp[c];
                }
              }
      }
    }
    if (rigid_i && grad_rho) {
      /* dL/dR = sum g (p - c)^T; angles through dR; translations in finest voxels */
      double* gr = grad_rho + (size_t)(i - 1) * 6;
      for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) acc += (GA[3 * r + c] - gb[r] * cen[c]) * dR[9 * a + 3 * r + c];
        gr[a] = acc;
        gr[3 + a] = gb[a] / tscale;
      }
    }
  }
  free(Ur);
  double L[3];
  or_regulariser(phi, N, nf, t, p->alpha_ss, p->alpha_l2, p->alpha_ts, L, grad);
  double total = sim + p->alpha_ss * L[0] + p->alpha_l2 * L[1] + p->alpha_ts * L[2];
  if (split) {
    split[0] = sim;
    split[1] = L[0];
    split[2] = L[1];
    split[3] = L[2];
  }
  if (grad) {
    double* g_up = zalloc((size_t)F * 3 * Vf);
    double* g_um = zalloc((size_t)F * 3 * Vf);
    double* tmp = zalloc(3 * Vf);
    or_compose_adjoint(up, um, N, nf, gU, g_up, g_um);
    for (int m = 0; m < F; ++m) {
      double* gm = grad + (size_t)m * 3 * Vf;
      or_exp_adjoint(phi + (size_t)m * 3 * Vf, nf, p->K, +1.0, g_up + (size_t)m * 3 * Vf, tmp);
      for (size_t e = 0; e < 3 * Vf; ++e) gm[e] += tmp[e];
      or_exp_adjoint(phi + (size_t)m * 3 * Vf, nf, p->K, -1.0, g_um + (size_t)m * 3 * Vf, tmp);
      for (size_t e = 0; e < 3 * Vf; ++e) gm[e] += tmp[e];
    }
    free(g_up);
    free(g_um);
    free(tmp);
  }
  free(up);
  free(um);
  free(U);
  free(gU);
  free(Ut);
  free(W);
  free(dW);
  free(gUt);
  return total;
}

/* ---------------------------------------------------------------------------
 * Sec. Implementation Details: Adam, linear warm-up over the first 20% of the
 * iterations, then cosine decay.
 * ------------------------------------------------------------------------- */
double or_lr(int step, int T, double lr, double warmup_frac) {
  int Wu = (int)ceil(warmup_frac * (double)T);
  if (Wu < 1) Wu = 1;
  if (step <= Wu) return lr * (double)step / (double)Wu;
  return lr * 0.5 * (1.0 + cos(PI_D * (double)(step - Wu) / (double)(T - Wu)));
}

void or_adam_step(double* theta, double* m, double* v, const double* g, size_t n, int step,
                  double lr_t, double b1, double b2, double eps) {
  double bc1 = 1.0 - pow(b1, step), bc2 = 1.0 - pow(b2, step);
  for (size_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    double mh = m[i] / bc1, vh = v[i] / bc2;
    theta[i] -= lr_t * mh / (sqrt(vh) + eps);
  }
}

double or_run(const double* imgs, int N, const int n[3], const or_params* p, const double* t,
              double* theta_out, double* loss_hist) {
  return or_run_rigid(imgs, N, n, p, t, theta_out, loss_hist, NULL);
}

double or_run_rigid(const double* imgs, int N, const int n[3], const or_params* p, const double* t,
                    double* theta_out, double* loss_hist, double* rho_out) {
  int L = p->n_levels, F = N - 1;
  size_t V = nvox(n);
  /* pyramid, finest level first in memory order of construction */
  double** pyr = (double**)calloc((size_t)L, sizeof(double*));
  int(*dims)[3] = calloc((size_t)L, sizeof(*dims));
  pyr[L - 1] = zalloc((size_t)N * V);
  memcpy(pyr[L - 1], imgs, (size_t)N * V * sizeof(double));
  memcpy(dims[L - 1], n, sizeof(int) * 3);
  for (int l = L - 2; l >= 0; --l) {
    for (int a = 0; a < 3; ++a) dims[l][a] = (dims[l + 1][a] + 1) / 2;
    size_t Vl = nvox(dims[l]), Vu = nvox(dims[l + 1]);
    pyr[l] = zalloc((size_t)N * Vl);
    for (int s = 0; s < N; ++s) or_downsample2(pyr[l + 1] + s * Vu, dims[l + 1], pyr[l] + s * Vl);
  }
  double* theta = NULL;
  int nf_prev[3] = {0, 0, 0};
  /* rigid parameters of sessions 1..N-1 (kept across levels; Adam state reset per level) */
  const int rigid = p->rigid != 0;
  double* rho = zalloc((size_t)F * 6);
  double* grho = zalloc((size_t)F * 6);
  const double rmax = 0.5 * (double)(n[0] > n[1] ? (n[0] > n[2] ? n[0] : n[2]) : (n[1] > n[2] ? n[1] : n[2]));
  double loss = 0.0;
  size_t hist = 0;
  for (int l = 0; l < L; ++l) {
    int ni[3], nf[3];
    or_level_dims(n, L, l, p->flow_factor, ni, nf);
    size_t Vf = nvox(nf);
    double* th = zalloc((size_t)F * 3 * Vf);
    if (theta) {
      size_t Vp = nvox(nf_prev);
      for (int m = 0; m < F; ++m)
        or_prolong(theta + (size_t)m * 3 * Vp, nf_prev, nf, th + (size_t)m * 3 * Vf);
      free(theta);
    }
    theta = th;
    memcpy(nf_prev, nf, sizeof(nf));
    /* level l images are 2^(L-1-l) times coarser than the finest */
    or_params pl = *p;
    for (int a = 0; a < 3; ++a) pl.spacing[a] = p->spacing[a] * (double)(1 << (L - 1 - l));
    double* m1 = zalloc((size_t)F * 3 * Vf);
    double* m2 = zalloc((size_t)F * 3 * Vf);
    double* g = zalloc((size_t)F * 3 * Vf);
    double* rm1 = zalloc((size_t)F * 6);
    double* rm2 = zalloc((size_t)F * 6);
    const double tscale = (double)(1 << (L - 1 - l));
    int T = p->steps[l];
    for (int s = 1; s <= T; ++s) {
      loss = or_loss_grad_rigid(pyr[l], N, ni, theta, nf, &pl, t, rigid ? rho : NULL, tscale, NULL, g,
                                rigid ? grho : NULL);
      if (loss_hist) loss_hist[hist++] = loss;
      double lr_t = or_lr(s, T, p->lr, p->warmup_frac);
      if (p->optimizer == OR_ADAM)
        or_adam_step(theta, m1, m2, g, (size_t)F * 3 * Vf, s, lr_t, p->beta1, p->beta2, p->adam_eps);
      else
        for (size_t e = 0; e < (size_t)F * 3 * Vf; ++e) theta[e] -= lr_t * g[e];
      if (rigid) {
        /* the rigid parameters follow the same schedule, scaled to rigid_lr (translations,
           voxels) and rigid_lr / rmax (angles, radians) */
        const double f = lr_t / p->lr;
        const double bc1 = 1.0 - pow(p->beta1, s), bc2 = 1.0 - pow(p->beta2, s);
        for (int e = 0; e < F * 6; ++e) {
          const double lr_e = f * p->rigid_lr / ((e % 6) < 3 ? rmax : 1.0);
          if (p->optimizer == OR_ADAM) {
            rm1[e] = p->beta1 * rm1[e] + (1.0 - p->beta1) * grho[e];
            rm2[e] = p->beta2 * rm2[e] + (1.0 - p->beta2) * grho[e] * grho[e];
            rho[e] -= lr_e * (rm1[e] / bc1) / (sqrt(rm2[e] / bc2) + p->adam_eps);
          } else {
            rho[e] -= lr_e * grho[e];
          }
        }
      }
    }
    free(rm1);
    free(rm2);
    free(m1);
    free(m2);
    free(g);
  }
  if (theta_out && theta) {
    int ni[3], nf[3];
    or_level_dims(n, L, L - 1, p->flow_factor, ni, nf);
    memcpy(theta_out, theta, (size_t)F * 3 * nvox(nf) * sizeof(double));
  }
  if (rho_out) memcpy(rho_out, rho, (size_t)F * 6 * sizeof(double));
  free(rho);
  free(grho);
  free(theta);
  for (int l = 0; l < L; ++l) free(pyr[l]);
  free(pyr);
  free(dims);
  return loss;
}

/* ------------------------------------------------------------------------------------------
 * Jacobian determinant maps (Sec. Sensitivity to clinical outcomes; Fig. 1c) */
static double diff_along(const double* f, const int n[3], int z, int y, int x, int axis) {
  int p[3] = {z, y, x};
  const int m = n[axis];
  if (m == 1) return 0.0;
  int lo[3] = {z, y, x}, hi[3] = {z, y, x};
  double h;
  if (p[axis] == 0) {
    hi[axis] = 1;
    h = 1.0;
  } else if (p[axis] == m - 1) {
    lo[axis] = m - 2;
    h = 1.0;
  } else {
    lo[axis] = p[axis] - 1;
    hi[axis] = p[axis] + 1;
    h = 2.0;
  }
  return (f[at(n, hi[0], hi[1], hi[2])] - f[at(n, lo[0], lo[1], lo[2])]) / h;
}

void or_jacobian_det(const double* u, const int n[3], double* J) {
  const size_t V = nvox(n);
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < n[0]; ++z)
    for (int y = 0; y < n[1]; ++y)
      for (int x = 0; x < n[2]; ++x) {
        double M[3][3]; /* M[c][a] = delta_ca + d u_c / d x_a */
        for (int c = 0; c < 3; ++c)
          for (int a = 0; a < 3; ++a) M[c][a] = (c == a ? 1.0 : 0.0) + diff_along(u + (size_t)c * V, n, z, y, x, a);
        J[at(n, z, y, x)] = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                            M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                            M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
      }
}

/* ------------------------------------------------------------------------------------------
 * Sec. Evaluation Metrics: Eu, PCC and the regression slope B */
void or_deformation_metrics(const double* ut, const double* ue, const unsigned char* roi, const int n[3],
                            double out[16]) {
  const size_t V = nvox(n);
  double cnt = 0.0, eu = 0.0, mt[3] = {0, 0, 0}, me[3] = {0, 0, 0};
  for (size_t v = 0; v < V; ++v) {
    if (roi && !roi[v]) continue;
    double d2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double a = ut[(size_t)c * V + v], b = ue[(size_t)c * V + v];
      d2 += (a - b) * (a - b);
      mt[c] += a;
      me[c] += b;
    }
    eu += sqrt(d2);
    cnt += 1.0;
  }
  for (int i = 0; i < 16; ++i) out[i] = 0.0;
  out[15] = cnt;
  if (cnt == 0.0) return;
  for (int c = 0; c < 3; ++c) {
    mt[c] /= cnt;
    me[c] /= cnt;
  }
  /* centred second moments: Ctt = sum (ut-mt)(ut-mt)^T, Cet = sum (ue-me)(ut-mt)^T */
  double Ctt[3][3] = {{0}}, Cet[3][3] = {{0}}, see = 0.0;
  for (size_t v = 0; v < V; ++v) {
    if (roi && !roi[v]) continue;
    double a[3], b[3];
    for (int c = 0; c < 3; ++c) {
      a[c] = ut[(size_t)c * V + v] - mt[c];
      b[c] = ue[(size_t)c * V + v] - me[c];
    }
    for (int r = 0; r < 3; ++r) {
      see += b[r] * b[r];
      for (int c = 0; c < 3; ++c) {
        Ctt[r][c] += a[r] * a[c];
        Cet[r][c] += b[r] * a[c];
      }
    }
  }
  const double stt = Ctt[0][0] + Ctt[1][1] + Ctt[2][2], ste = Cet[0][0] + Cet[1][1] + Cet[2][2];
  out[0] = eu / cnt;
  out[1] = ste / (sqrt(stt) * sqrt(see));
  /* A = Cet Ctt^-1 (normal equations of the fit with intercept), b = me - A mt */
  double inv[3][3];
  const double det = Ctt[0][0] * (Ctt[1][1] * Ctt[2][2] - Ctt[1][2] * Ctt[2][1]) -
                     Ctt[0][1] * (Ctt[1][0] * Ctt[2][2] - Ctt[1][2] * Ctt[2][0]) +
                     Ctt[0][2] * (Ctt[1][0] * Ctt[2][1] - Ctt[1][1] * Ctt[2][0]);
  inv[0][0] = (Ctt[1][1] * Ctt[2][2] - Ctt[1][2] * Ctt[2][1]) / det;
  inv[0][1] = (Ctt[0][2] * Ctt[2][1] - Ctt[0][1] * Ctt[2][2]) / det;
  inv[0][2] = (Ctt[0][1] * Ctt[1][2] - Ctt[0][2] * Ctt[1][1]) / det;
  inv[1][0] = (Ctt[1][2] * Ctt[2][0] - Ctt[1][0] * Ctt[2][2]) / det;
  inv[1][1] = (Ctt[0][0] * Ctt[2][2] - Ctt[0][2] * Ctt[2][0]) / det;
  inv[1][2] = (Ctt[0][2] * Ctt[1][0] - Ctt[0][0] * Ctt[1][2]) / det;
  inv[2][0] = (Ctt[1][0] * Ctt[2][1] - Ctt[1][1] * Ctt[2][0]) / det;
  inv[2][1] = (Ctt[0][1] * Ctt[2][0] - Ctt[0][0] * Ctt[2][1]) / det;
  inv[2][2] = (Ctt[0][0] * Ctt[1][1] - Ctt[0][1] * Ctt[1][0]) / det;
  double A[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) A[r][c] = Cet[r][0] * inv[0][c] + Cet[r][1] * inv[1][c] + Cet[r][2] * inv[2][c];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) out[3 + 3 * r + c] = A[r][c];
    out[12 + r] = me[r] - (A[r][0] * mt[0] + A[r][1] * mt[1] + A[r][2] * mt[2]);
  }
  out[2] = (A[0][0] + A[1][1] + A[2][2]) / 3.0;
}
