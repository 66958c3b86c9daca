// rigid_kernels.cu -- rigid registration in parallel with the deformable one (Sec. Rigid
// Registration). Session i >= 1 has Euler angles a (radians) and a translation t (voxels of
// the finest level); every pair pulled onto grid i samples at p + U(p) + A_i p + b_i with
// A_i = R_i - I, b_i = (I - R_i) c + t_i / tscale, R = R_0(a0) R_1(a1) R_2(a2) (R_k rotating
// the plane of the two other axes), c the centre of the level's image grid and tscale the
// finest voxels per voxel of the level. The warp adjoint leaves per-CTA sums of dL/dq and
// dL/dq p^T; here they are reduced in a fixed order per session and chained to the angles
// and the translation, and the six parameters take an Adam (or plain) step on the velocity
// schedule scaled to rigid_lr.
#include "kernels.h"

namespace muster {

namespace {

__device__ void axis_rot(int k, double ang, double M[9], double dM[9]) {
  const double c = cos(ang), s = sin(ang);
  for (int e = 0; e < 9; ++e) M[e] = dM[e] = 0.0;
  const int u = (k + 1) % 3, w = (k + 2) % 3;
  M[3 * k + k] = 1.0;
  M[3 * u + u] = c;
  M[3 * u + w] = -s;
  M[3 * w + u] = s;
  M[3 * w + w] = c;
  dM[3 * u + u] = -s;
  dM[3 * u + w] = -c;
  dM[3 * w + u] = c;
  dM[3 * w + w] = -s;
}
__device__ void mul3(const double A[9], const double B[9], double C[9]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}
// R and, when dR is given, dR/da_k for k = 0, 1, 2
__device__ void rotation(const float a[3], double R[9], double* dR) {
  double M[3][9], dM[3][9], T[9];
  for (int k = 0; k < 3; ++k) axis_rot(k, (double)a[k], M[k], dM[k]);
  mul3(M[0], M[1], T);
  mul3(T, M[2], R);
  if (!dR) return;
  for (int k = 0; k < 3; ++k) {
    mul3(k == 0 ? dM[0] : M[0], k == 1 ? dM[1] : M[1], T);
    mul3(T, k == 2 ? dM[2] : M[2], dR + 9 * k);
  }
}
// table row of session i: A = R - I (row-major), b = (I - R) c + t / tscale
__device__ void table_row(const float* rho, int i, const RigidArgs& a, float* row) {
  if (i == 0) {
    for (int e = 0; e < 12; ++e) row[e] = 0.f;
    return;
  }
  const float* r = rho + 6 * (i - 1);
  double R[9];
  rotation(r, R, nullptr);
  const double c[3] = {a.c0, a.c1, a.c2};
  for (int q = 0; q < 3; ++q) {
    for (int s = 0; s < 3; ++s) row[3 * q + s] = (float)(R[3 * q + s] - (q == s ? 1.0 : 0.0));
    const double Rc = R[3 * q] * c[0] + R[3 * q + 1] * c[1] + R[3 * q + 2] * c[2];
    row[9 + q] = (float)(c[q] - Rc + (double)r[3 + q] / a.tscale);
  }
}

__global__ void k_rigid_table(const float* __restrict__ rho, float* __restrict__ tab, RigidArgs a) {
  const int i = threadIdx.x;
  if (i < a.N) table_row(rho, i, a, tab + 12 * i);
}

// one thread per session i >= 1: pairs (k -> i) are i*(N-1) + r, r = 0..N-2
__global__ void k_rigid_grad(const float* __restrict__ rpart, const float* __restrict__ rho,
                             float* __restrict__ grad, RigidArgs a) {
  const int i = threadIdx.x + 1;
  if (i >= a.N) return;
  double S[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int r = 0; r < a.N - 1; ++r) {
    const float* p = rpart + ((size_t)(i * (a.N - 1) + r) * a.per_pair) * 12;
    for (int c = 0; c < a.per_pair; ++c)
      for (int e = 0; e < 12; ++e) S[e] += (double)p[(size_t)c * 12 + e];
  }
  double R[9], dR[27];
  rotation(rho + 6 * (i - 1), R, dR);
  const double c[3] = {a.c0, a.c1, a.c2};
  float* g = grad + 6 * (i - 1);
  for (int k = 0; k < 3; ++k) {
    double acc = 0.0;  // sum over (q, s) of (sum g_q p_s - sum g_q c_s) dR_k[q][s]
    for (int q = 0; q < 3; ++q)
      for (int s = 0; s < 3; ++s) acc += (S[3 + 3 * q + s] - S[q] * c[s]) * dR[9 * k + 3 * q + s];
    g[k] = (float)acc;
    g[3 + k] = (float)(S[k] / a.tscale);
  }
}

// the optimiser step of the rigid parameters, then the table of the new parameters
__global__ void k_rigid_step(float* __restrict__ rho, float* __restrict__ m, float* __restrict__ v,
                             const float* __restrict__ grad, const float* __restrict__ sched,
                             const int* __restrict__ step, float* __restrict__ tab, RigidArgs a) {
  const int e = threadIdx.x, n = 6 * (a.N - 1);
  if (e < n) {
    const int s = *step;
    const float lr_t = sched[3 * s], ib1 = sched[3 * s + 1], ib2 = sched[3 * s + 2];
    const float lr = lr_t / a.lr_base * a.rigid_lr / ((e % 6) < 3 ? a.rmax : 1.f);
    const float gg = grad[e];
    if (a.sgd) {
      rho[e] -= lr * gg;
    } else {
      const float mm = a.b1 * m[e] + (1.f - a.b1) * gg;
      const float vv = a.b2 * v[e] + (1.f - a.b2) * gg * gg;
      m[e] = mm;
      v[e] = vv;
      rho[e] -= lr * (mm * ib1) / (sqrtf(vv * ib2) + a.eps);
    }
  }
  __syncthreads();
  if (e < a.N) table_row(rho, e, a, tab + 12 * e);
}

// u (planar (3, D, H, W), image voxels) += A_i p + b_i of table row `row`
__global__ void k_add_rigid(float* __restrict__ u, Dims n, const float* __restrict__ row) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= n.n2) return;
  const size_t V = vox(n), o = ((size_t)z * n.n1 + y) * n.n2 + x;
  const float p[3] = {(float)z, (float)y, (float)x};
  for (int q = 0; q < 3; ++q) u[q * V + o] += row[3 * q] * p[0] + row[3 * q + 1] * p[1] + row[3 * q + 2] * p[2] + row[9 + q];
}
}  // namespace

void launch_rigid_table(const float* rho, float* tab, const RigidArgs& a, cudaStream_t s) {
  k_rigid_table<<<1, 32, 0, s>>>(rho, tab, a);
}
void launch_rigid_grad(const float* rpart, const float* rho, float* grad, const RigidArgs& a, cudaStream_t s) {
  k_rigid_grad<<<1, 32, 0, s>>>(rpart, rho, grad, a);
}
void launch_rigid_step(float* rho, float* m, float* v, const float* grad, const float* sched, const int* step,
                       float* tab, const RigidArgs& a, cudaStream_t s) {
  k_rigid_step<<<1, 192, 0, s>>>(rho, m, v, grad, sched, step, tab, a);
}
void launch_add_rigid(float* u, Dims n, const float* row, cudaStream_t s) {
  k_add_rigid<<<dim3((n.n2 + 127) / 128, n.n1, n.n0), 128, 0, s>>>(u, n, row);
}

}  // namespace muster
