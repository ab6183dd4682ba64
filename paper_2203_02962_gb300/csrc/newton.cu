// Newton's method of Algorithm 1 for a nonlinear scalar conductivity on the trilinear hexahedron
// (2 x 2 x 2 Gauss points): per-quadrature-point flux and tangent (Sec. 3, nonlinear system; Sec. 3.1,
// Eq. lin_system), the tangent apply K_t x = D^T W A D x for the linear solves, and the gradient norm
// of the Newton test (Sec. 6).  FP64 throughout.
//
// The tangent varies from quadrature point to quadrature point, so the element is evaluated at its
// eight Gauss points (not in the modal form of the linear kernels, which needs a material constant
// per voxel).  One thread per voxel writes its eight nodal contributions; a second kernel gathers,
// for each node, the contributions of the eight voxels around it (fixed order, no atomics).
//
// Law, per phase p: q(g) = k_p s^((n_p - 1) / 2) g, s = 1 + |g|^2 / g0^2, with tangent
// A(g) = k_p s^((n_p - 1) / 2) (I + (n_p - 1) g g^T / (g0^2 s)).
#include "fehom_internal.cuh"

#include <algorithm>

namespace fehom {
namespace {

constexpr int NLT = 128;

__device__ __forceinline__ int wrapn(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ double nl_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (l == 0) sh[0] = t;
  }
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

// Gradient of the trilinear field u[corner], corner = a + 2 b + 4 c, at the Gauss point q of the
// same numbering (xi_q = (2 qa - 1) / sqrt 3, ...): du/dx = (1 / (4 h_x)) sum_c s_a (1 + s_b eta)(1 + s_c zeta) u_c.
__device__ __forceinline__ void qp_gradient(const double (&u)[8], int q, const double (&ih)[3], double (&g)[3]) {
  const double r3 = 0.57735026918962576451;
  const double xq[3] = {(q & 1) ? r3 : -r3, (q & 2) ? r3 : -r3, (q & 4) ? r3 : -r3};
  g[0] = g[1] = g[2] = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const double s0 = (c & 1) ? 1.0 : -1.0, s1 = (c & 2) ? 1.0 : -1.0, s2 = (c & 4) ? 1.0 : -1.0;
    const double f0 = 1.0 + s0 * xq[0], f1 = 1.0 + s1 * xq[1], f2 = 1.0 + s2 * xq[2];
    g[0] = fma(s0 * f1 * f2, u[c], g[0]);
    g[1] = fma(s1 * f0 * f2, u[c], g[1]);
    g[2] = fma(s2 * f0 * f1, u[c], g[2]);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) g[i] *= 0.25 * ih[i];
}

// f[c] += w grad N_c(q) . t  (the transposed gradient at Gauss point q)
__device__ __forceinline__ void qp_scatter(const double (&t)[3], int q, const double (&ih)[3], double w, double (&f)[8]) {
  const double r3 = 0.57735026918962576451;
  const double xq[3] = {(q & 1) ? r3 : -r3, (q & 2) ? r3 : -r3, (q & 4) ? r3 : -r3};
  const double t0 = 0.25 * ih[0] * w * t[0], t1 = 0.25 * ih[1] * w * t[1], t2 = 0.25 * ih[2] * w * t[2];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const double s0 = (c & 1) ? 1.0 : -1.0, s1 = (c & 2) ? 1.0 : -1.0, s2 = (c & 4) ? 1.0 : -1.0;
    const double f0 = 1.0 + s0 * xq[0], f1 = 1.0 + s1 * xq[1], f2 = 1.0 + s2 * xq[2];
    f[c] += s0 * f1 * f2 * t0 + s1 * f0 * f2 * t1 + s2 * f0 * f1 * t2;
  }
}

// MODE 0: flux and tangent at u (gradient e + D u): element residual contributions, tangents stored
//         per Gauss point (xx, yy, zz, yz, xz, xy), block partials of sum w q (3) and sum w A (6).
// MODE 1: tangent apply to x: element contributions of D^T W A D x.
// MODE 2: block partials of sum w |D x|^2.
template <int MODE>
__global__ void __launch_bounds__(NLT) nl_element_kernel(NlArgs a) {
  __shared__ double sh[32];
  const Dims d = a.d;
  const long long N = d.N;
  const long long v = blockIdx.x * (long long)NLT + threadIdx.x;
  const bool on = v < N;
  const int i = on ? (int)(v % d.nx) : 0, j = on ? (int)((v / d.nx) % d.ny) : 0;
  const int k = on ? (int)(v / ((long long)d.nx * d.ny)) : 0;
  const double ih[3] = {1.0 / a.h[0], 1.0 / a.h[1], 1.0 / a.h[2]};
  const double w = a.vvox / 8.0;
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (on) {
    double u[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const long long node = ((long long)wrapn(k + ((c >> 2) & 1), d.nz) * d.ny + wrapn(j + ((c >> 1) & 1), d.ny)) * d.nx +
                             wrapn(i + (c & 1), d.nx);
      u[c] = a.x[node];
    }
    double f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int ph = a.ids ? a.ids[v] : 0;
    const double kp = a.kp[ph], np = a.np[ph];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      double g[3];
      qp_gradient(u, q, ih, g);
      if (MODE == 0) {
        g[0] += a.e[0];
        g[1] += a.e[1];
        g[2] += a.e[2];
        const double s = 1.0 + (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) / (a.g0 * a.g0);
        const double fs = kp * pow(s, 0.5 * (np - 1.0));
        const double cc = (np - 1.0) / (a.g0 * a.g0 * s);
        const double t[3] = {fs * g[0], fs * g[1], fs * g[2]};
        double A[6] = {fs * (1.0 + cc * g[0] * g[0]), fs * (1.0 + cc * g[1] * g[1]), fs * (1.0 + cc * g[2] * g[2]),
                       fs * cc * g[1] * g[2], fs * cc * g[0] * g[2], fs * cc * g[0] * g[1]};
        double* T = a.T + (v * 8 + q) * 6;
#pragma unroll
        for (int r = 0; r < 6; ++r) T[r] = A[r];
        qp_scatter(t, q, ih, w, f);
#pragma unroll
        for (int r = 0; r < 3; ++r) acc[r] += w * t[r];
#pragma unroll
        for (int r = 0; r < 6; ++r) acc[3 + r] += w * A[r];
      } else if (MODE == 1) {
        const double* T = a.T + (v * 8 + q) * 6;
        const double t[3] = {T[0] * g[0] + T[5] * g[1] + T[4] * g[2], T[5] * g[0] + T[1] * g[1] + T[3] * g[2],
                             T[4] * g[0] + T[3] * g[1] + T[2] * g[2]};
        qp_scatter(t, q, ih, w, f);
      } else {
        acc[0] += w * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
      }
    }
    if (MODE != 2) {
#pragma unroll
      for (int c = 0; c < 8; ++c) a.E[v * 8 + c] = f[c];
    }
  }
  if (MODE != 1) {
    const int nacc = MODE == 0 ? 9 : 1;
    for (int r = 0; r < nacc; ++r) {
      const double t = nl_block_sum(acc[r], sh);
      if (threadIdx.x == 0) a.partial[(long long)blockIdx.x * nacc + r] = t;
    }
  }
}

// y[node] = s * sum over the 8 voxels around the node of their contribution to it; with dot != 0 also
// block partials of sum y x.
__global__ void __launch_bounds__(NLT) nl_gather_kernel(NlArgs a, double s, int dot) {
  __shared__ double sh[32];
  const Dims d = a.d;
  const long long node = blockIdx.x * (long long)NLT + threadIdx.x;
  double acc = 0.0;
  if (node < d.N) {
    const int i = (int)(node % d.nx), j = (int)((node / d.nx) % d.ny), k = (int)(node / ((long long)d.nx * d.ny));
    double y = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      // the voxel whose corner c is this node
      const long long vox = ((long long)wrapn(k - ((c >> 2) & 1), d.nz) * d.ny + wrapn(j - ((c >> 1) & 1), d.ny)) * d.nx +
                            wrapn(i - (c & 1), d.nx);
      y += a.E[vox * 8 + c];
    }
    y *= s;
    a.y[node] = y;
    if (dot) acc = y * a.x[node];
  }
  if (dot) {
    const double t = nl_block_sum(acc, sh);
    if (threadIdx.x == 0) a.partial[blockIdx.x] = t;
  }
}

// y = alpha x + beta y; optional block partials of sum y z
__global__ void nl_axpby_kernel(long long n, double alpha, const double* x, double beta, double* y, const double* z,
                                double* partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)NLT + threadIdx.x; t < n; t += (long long)gridDim.x * NLT) {
    const double v = fma(alpha, x[t], beta * y[t]);
    y[t] = v;
    if (z) acc = fma(v, z[t], acc);
  }
  if (partial) {
    const double s = nl_block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

__global__ void nl_dot_kernel(long long n, const double* x, const double* y, double* partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)NLT + threadIdx.x; t < n; t += (long long)gridDim.x * NLT)
    acc = fma(x[t], y[t], acc);
  const double s = nl_block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

}  // namespace

int nl_blocks(long long n) { return (int)std::max<long long>(1, (n + NLT - 1) / NLT); }
int nl_vec_blocks() { return 2 * 152; }

cudaError_t launch_nl_element(const NlArgs& a, int mode, cudaStream_t s) {
  const int b = nl_blocks(a.d.N);
  if (mode == 0) nl_element_kernel<0><<<b, NLT, 0, s>>>(a);
  else if (mode == 1) nl_element_kernel<1><<<b, NLT, 0, s>>>(a);
  else nl_element_kernel<2><<<b, NLT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_nl_gather(const NlArgs& a, double scale, int dot, cudaStream_t s) {
  nl_gather_kernel<<<nl_blocks(a.d.N), NLT, 0, s>>>(a, scale, dot);
  return cudaGetLastError();
}

cudaError_t launch_nl_axpby(long long n, double alpha, const double* x, double beta, double* y, const double* z,
                            double* partial, cudaStream_t s) {
  nl_axpby_kernel<<<nl_vec_blocks(), NLT, 0, s>>>(n, alpha, x, beta, y, z, partial);
  return cudaGetLastError();
}

cudaError_t launch_nl_dot(long long n, const double* x, const double* y, double* partial, cudaStream_t s) {
  nl_dot_kernel<<<nl_vec_blocks(), NLT, 0, s>>>(n, x, y, partial);
  return cudaGetLastError();
}

}  // namespace fehom
