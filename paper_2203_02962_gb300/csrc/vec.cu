// Small vector kernels of the solve driver: precision casts of the iterative-refinement loop and
// mean removal.  All reductions are FP64 with a fixed order.
#include "fehom_internal.cuh"

#include <algorithm>
#include <cstdint>

namespace fehom {
namespace {

constexpr int VT = 256;

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>(8 * 152, (n + VT - 1) / VT)); }

__global__ void cast_d2f_kernel(const double* __restrict__ x, float* __restrict__ y, double s, long long n) {
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT)
    y[i] = (float)(s * x[i]);
}

__global__ void add_f2d_kernel(const float* __restrict__ x, double* __restrict__ y, double s, long long n) {
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT)
    y[i] = fma(s, (double)x[i], y[i]);
}

// the same four elements at a time (16-byte accesses; both arrays 16-byte aligned); the last n mod 4
// elements by the first threads of block 0
__global__ void cast_d2f4_kernel(const double* __restrict__ x, float* __restrict__ y, double s, long long n) {
  const long long n4 = n / 4;
  const double2* x2 = reinterpret_cast<const double2*>(x);
  float4* y4 = reinterpret_cast<float4*>(y);
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n4; i += (long long)gridDim.x * VT) {
    const double2 a = x2[2 * i], b = x2[2 * i + 1];
    y4[i] = make_float4((float)(s * a.x), (float)(s * a.y), (float)(s * b.x), (float)(s * b.y));
  }
  if (blockIdx.x == 0 && threadIdx.x < n - 4 * n4) y[4 * n4 + threadIdx.x] = (float)(s * x[4 * n4 + threadIdx.x]);
}

__global__ void add_f2d4_kernel(const float* __restrict__ x, double* __restrict__ y, double s, long long n) {
  const long long n4 = n / 4;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  double2* y2 = reinterpret_cast<double2*>(y);
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n4; i += (long long)gridDim.x * VT) {
    const float4 v = x4[i];
    const double2 a = y2[2 * i], b = y2[2 * i + 1];
    y2[2 * i] = make_double2(fma(s, (double)v.x, a.x), fma(s, (double)v.y, a.y));
    y2[2 * i + 1] = make_double2(fma(s, (double)v.z, b.x), fma(s, (double)v.w, b.y));
  }
  if (blockIdx.x == 0 && threadIdx.x < n - 4 * n4) {
    const long long j = 4 * n4 + threadIdx.x;
    y[j] = fma(s, (double)x[j], y[j]);
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

__device__ double block_sum(double v) {
  __shared__ double sh[32];
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

// mean removal per (component, load): CTA partial sums, then every CTA re-adds the partials of its
// (component, load) in index order (the same sum in every CTA) and subtracts the mean from its slice
constexpr int SM_BLOCKS = 2 * 152;

__global__ void mean_partial_kernel(const double* __restrict__ x, long long N, long long load_stride, double* partial) {
  const double* p = x + (long long)blockIdx.z * load_stride + (long long)blockIdx.y * N;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < N; i += (long long)gridDim.x * VT) acc += p[i];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) partial[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
}

__global__ void mean_subtract_kernel(double* __restrict__ x, long long N, long long load_stride,
                                     const double* __restrict__ partial) {
  const double* pp = partial + ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += VT) acc += pp[b];
  const double mean = block_sum(acc) / (double)N;
  double* p = x + (long long)blockIdx.z * load_stride + (long long)blockIdx.y * N;
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < N; i += (long long)gridDim.x * VT) p[i] -= mean;
}

// Galerkin scaling of a warm start: CTA partial sums of x.kx and x.b per load, then every CTA re-adds
// the partials of its load in index order, forms gamma and scales its slice
__global__ void dot2_partial_kernel(const double* __restrict__ x, const double* __restrict__ kx,
                                    const double* __restrict__ b, long long n, double* partial) {
  const long long off = (long long)blockIdx.y * n;
  double s1 = 0.0, s2 = 0.0;
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT) {
    s1 = fma(x[off + i], kx[off + i], s1);
    s2 = fma(x[off + i], b[off + i], s2);
  }
  const double t1 = block_sum(s1);
  const double t2 = block_sum(s2);
  if (threadIdx.x == 0) {
    partial[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 2] = t1;
    partial[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 2 + 1] = t2;
  }
}

__global__ void galerkin_scale_kernel(double* __restrict__ x, long long n, const double* __restrict__ partial) {
  const double* pp = partial + (long long)blockIdx.y * gridDim.x * 2;
  double a1 = 0.0, a2 = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += VT) {
    a1 += pp[2 * k];
    a2 += pp[2 * k + 1];
  }
  const double xkx = block_sum(a1), xb = block_sum(a2);
  const double gamma = (xkx > 0.0 && isfinite(xb / xkx)) ? xb / xkx : 0.0;
  double* p = x + (long long)blockIdx.y * n;
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT) p[i] *= gamma;
}

// Energy-form effective tensor: for loads i, j < L <= 6, the dots x_i . r_j over n entries, in one
// pass that reads each x_i and r_j once.  partial[blk * L * L + i * L + j]; then out[i * L + j] sums
// the G partials in block order.
constexpr int kPairMax = 6;
__global__ void pair_dots_kernel(const double* __restrict__ x, const double* __restrict__ r, int L, long long n,
                                 double* partial) {
  double acc[kPairMax * kPairMax];
#pragma unroll
  for (int q = 0; q < kPairMax * kPairMax; ++q) acc[q] = 0.0;
  for (long long k = blockIdx.x * (long long)VT + threadIdx.x; k < n; k += (long long)gridDim.x * VT) {
    double xv[kPairMax], rv[kPairMax];
#pragma unroll
    for (int i = 0; i < kPairMax; ++i) {
      xv[i] = i < L ? x[(long long)i * n + k] : 0.0;
      rv[i] = i < L ? r[(long long)i * n + k] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < kPairMax; ++i)
#pragma unroll
      for (int j = 0; j < kPairMax; ++j)
        if (i < L && j < L) acc[i * kPairMax + j] = fma(xv[i], rv[j], acc[i * kPairMax + j]);
  }
#pragma unroll
  for (int i = 0; i < kPairMax; ++i)
#pragma unroll
    for (int j = 0; j < kPairMax; ++j)
      if (i < L && j < L) {  // uniform: every thread reaches the block sum's barriers
        const double t = block_sum(acc[i * kPairMax + j]);
        if (threadIdx.x == 0) partial[(long long)blockIdx.x * L * L + i * L + j] = t;
      }
}

__global__ void pair_dots_final_kernel(const double* __restrict__ partial, int L, int G, double* out) {
  const int q = threadIdx.x;  // (i, j) flattened, L L entries
  if (q >= L * L) return;
  double s = 0.0;
  for (int g = 0; g < G; ++g) s += partial[(long long)g * L * L + q];
  out[q] = s;
}

__global__ void impulse_scatter_kernel(const double* __restrict__ py, Dims pd, Dims full, int c, double* out) {
  const int nb = full.dim == 3 ? 27 : 9;
  const int t = threadIdx.x;
  if (t >= c * c * nb) return;
  const int o = t % nb, pair = t / nb, al = pair % c, be = pair / c;
  const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = full.dim == 3 ? o / 9 - 1 : 0;
  auto wrapi = [](int i, int n) { return ((i % n) + n) % n; };
  const long long ps = ((long long)wrapi(dz, pd.nz) * pd.ny + wrapi(dy, pd.ny)) * pd.nx + wrapi(dx, pd.nx);
  const long long fs = ((long long)wrapi(dz, full.nz) * full.ny + wrapi(dy, full.ny)) * full.nx + wrapi(dx, full.nx);
  out[((long long)be * c + al) * full.N + fs] = py[((long long)be * c + al) * pd.N + ps];
}

}  // namespace

cudaError_t launch_impulse_scatter(const double* py, const Dims& pd, const Dims& full, int c, double* out,
                                   cudaStream_t s) {
  impulse_scatter_kernel<<<1, 256, 0, s>>>(py, pd, full, c, out);
  return cudaGetLastError();
}

cudaError_t launch_cast_d2f(const double* x, float* y, double scale, long long n, cudaStream_t s) {
  if (aligned16(x) && aligned16(y)) cast_d2f4_kernel<<<grid_for((n + 3) / 4), VT, 0, s>>>(x, y, scale, n);
  else cast_d2f_kernel<<<grid_for(n), VT, 0, s>>>(x, y, scale, n);
  return cudaGetLastError();
}

cudaError_t launch_add_f2d(const float* x, double* y, double scale, long long n, cudaStream_t s) {
  if (aligned16(x) && aligned16(y)) add_f2d4_kernel<<<grid_for((n + 3) / 4), VT, 0, s>>>(x, y, scale, n);
  else add_f2d_kernel<<<grid_for(n), VT, 0, s>>>(x, y, scale, n);
  return cudaGetLastError();
}

cudaError_t launch_pair_dots(const double* x, const double* r, int L, long long n, double* partial, double* out,
                             cudaStream_t s) {
  if (L < 1 || L > kPairMax) return cudaErrorInvalidValue;
  pair_dots_kernel<<<SM_BLOCKS, VT, 0, s>>>(x, r, L, n, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  pair_dots_final_kernel<<<1, 128, 0, s>>>(partial, L, SM_BLOCKS, out);
  return cudaGetLastError();
}

cudaError_t launch_galerkin_scale(double* x, const double* kx, const double* b, int n_loads, long long n,
                                  double* partial, cudaStream_t s) {
  const dim3 grid(SM_BLOCKS, n_loads);
  dot2_partial_kernel<<<grid, VT, 0, s>>>(x, kx, b, n, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  galerkin_scale_kernel<<<grid, VT, 0, s>>>(x, n, partial);
  return cudaGetLastError();
}

cudaError_t launch_sub_mean(double* x, int c, long long N, int n_loads, long long load_stride, double* partial,
                            cudaStream_t s) {
  const dim3 grid(SM_BLOCKS, c, n_loads);
  mean_partial_kernel<<<grid, VT, 0, s>>>(x, N, load_stride, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  mean_subtract_kernel<<<grid, VT, 0, s>>>(x, N, load_stride, partial);
  return cudaGetLastError();
}

}  // namespace fehom
