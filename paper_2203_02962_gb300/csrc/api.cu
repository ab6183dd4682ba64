// Host runtime of libfehom.so: the C ABI declared in include/fehom.h.
//
// fehom_setup        validates the grid and materials, uploads the phase ids, forms the reference
//                    material (volume mean C_mean of Sec. 6.2 unless given) and the gradient-space
//                    material tables used by the stiffness kernel.
// fehom_precond_build Algorithm 2 (Sec. 5.2) on the device + the block (pseudo-)inverse (Sec. 5.3).
// fehom_solve        PCG of Sec. 4.1 (symmetric form) for a batch of loads, each iteration one
//                    stiffness launch and the FFT passes, with alpha, beta and the stopping test kept
//                    in device memory; iterations replayed from a captured CUDA graph.  The mixed
//                    precision variant wraps an FP32 PCG in FP64 iterative refinement.
#include "fehom_internal.cuh"
#include "../../include/fehom.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

using namespace fehom;

struct fehom_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  fehom_options opt{};
  Dims d{};
  int physics = 0, m = 0, D = 0;  // D: gradient-space size c * dim
  double h[3] = {1, 1, 1};
  double vol = 1.0;
  int n_phases = 0;
  std::vector<double> moduli;     // [phase][m*m]
  std::vector<double> cref;       // [m*m]
  std::vector<double> frac;       // volume fractions
  std::vector<double> c_eff_energy;  // energy-form C_eff of the last solve with m loads (empty: none)
  bool iso = false;               // isotropic phases on a cubic grid (fast stiffness path)
  bool iso_ref = false;
  // device
  uint8_t* ids = nullptr;
  double* mats64 = nullptr; float* mats32 = nullptr;   // [phase][D*D]
  double* iso64 = nullptr; float* iso32 = nullptr;     // [phase][kIsoStride]
  float* isodf = nullptr;                               // [phase][16]: the iso constants as (hi, lo) float pairs
  double* rmats64 = nullptr; double* riso64 = nullptr;  // reference material (one phase)
  double2* tw64[3] = {nullptr, nullptr, nullptr};
  float2* tw32[3] = {nullptr, nullptr, nullptr};
  double* sym64 = nullptr; float* sym32 = nullptr;
  bool built = false;
  // work buffers (grown on demand)
  int cap64 = 0, cap32 = 0;
  double *x64 = nullptr, *r64 = nullptr, *p64 = nullptr, *ap64 = nullptr, *b64 = nullptr;
  double2* spec64 = nullptr;
  float *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *ap32 = nullptr;
  float2* spec32 = nullptr;
  PcgState* st = nullptr;
  RedScratch red{};
  double* tau = nullptr;       // [load][phase][D]
  float* taudf = nullptr;      // [load][phase][D][2]: tau as (hi, lo) float pairs (double-float right-hand side)
  double* partial = nullptr;   // general reduction scratch
  size_t partial_cap = 0;
  // captured iteration graphs
  cudaGraphExec_t graph_exec = nullptr;
  long long graph_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int graph_launches = 0;      // kernels per graph replay
  // launch accounting and optional per-kernel event timing
  long long launches = 0;
  bool counting = true;        // false while a graph is being captured
  bool events_made = false;
  cudaEvent_t ev[8][FEHOM_K_COUNT][2];
  struct FftPlan {
    int pairs = 0, tc_y = 0, tc_last = 0;
    int xy = 0;        // 1: fused x-y passes
    int last_reg = 0;  // 1: register-split last-axis pass
    int tuned_loads = 0;
    double ms[3] = {0, 0, 0};
  } plan[2];                   // [0] FP64 kernels, [1] FP32 kernels
  struct StencilPlan {
    int rows = 0;         // hex8 PCG apply: node rows per tile (0 = the precision's default)
    int staging = 0;      // FP32 node-plane staging: 0 cp.async copies, 3 tensor-memory-accelerator boxes
    int tuned_loads = 0;
    double ms[4] = {0, 0, 0, 0};  // timed candidates: 8 / 16 rows with cp.async, 8 / 16 rows with TMA
  } stencil[2];               // [0] FP64 kernels, [1] FP32 kernels
  PcgState* tune_st = nullptr;  // running states for the stencil tuner's PCG-apply launches
  double kms[2][FEHOM_K_COUNT] = {{0}};
  int hist_count[kMaxLoads] = {0};  // PCG coefficients recorded per load by the last PCG run
  long long kcnt[2][FEHOM_K_COUNT] = {{0}};
  std::string err;
};

namespace {

thread_local std::string g_setup_error;  // message of the last failed fehom_setup on this thread

constexpr int kRedBlocks = 1 << 16;
constexpr int kChunk = 8;  // PCG iterations per graph replay / convergence poll (<= 8: event slots)

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);              \
      return e_ == cudaErrorMemoryAllocation ? FEHOM_E_OOM : FEHOM_E_CUDA;        \
    }                                                                             \
  } while (0)

#define FAIL(code, msg)      \
  do {                       \
    ctx->err = (msg);        \
    return (code);           \
  } while (0)

#define TRY(x)                          \
  do {                                  \
    fehom_status s_ = (x);              \
    if (s_ != FEHOM_OK) return s_;      \
  } while (0)

bool size_ok(long long n) {
  if (n < 2 || n > 1024) return false;
  while (n % 2 == 0) n /= 2;
  return n == 1 || n == 3;
}

template <typename P> void dfree(P*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// symmetric positive definite check (Cholesky) of an m x m row-major matrix
bool spd(const double* A, int m) {
  std::vector<double> L(m * m, 0.0);
  double mx = 0;
  for (int i = 0; i < m * m; ++i) {
    if (!std::isfinite(A[i])) return false;
    mx = std::max(mx, std::fabs(A[i]));
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j)
      if (std::fabs(A[i * m + j] - A[j * m + i]) > 1e-12 * mx) return false;
  for (int j = 0; j < m; ++j) {
    double s = A[j * m + j];
    for (int k = 0; k < j; ++k) s -= L[j * m + k] * L[j * m + k];
    if (!(s > 1e-14 * mx)) return false;
    L[j * m + j] = std::sqrt(s);
    for (int i = j + 1; i < m; ++i) {
      double t = A[i * m + j];
      for (int k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
      L[i * m + j] = t / L[j * m + j];
    }
  }
  return true;
}

// P: flux vector (m) <- gradient vector (D, index comp * dim + deriv for elasticity, deriv for scalar)
std::vector<double> grad_to_flux(int dim, int physics) {
  if (physics == FEHOM_SCALAR) {
    std::vector<double> P(dim * dim, 0.0);
    for (int i = 0; i < dim; ++i) P[i * dim + i] = 1.0;
    return P;
  }
  const int m = dim * (dim + 1) / 2, D = dim * dim;
  std::vector<double> P(m * D, 0.0);
  for (int a = 0; a < dim; ++a) P[a * D + a * dim + a] = 1.0;
  const double r2 = 1.0 / std::sqrt(2.0);
  const int pairs3[3][2] = {{1, 2}, {0, 2}, {0, 1}};
  const int pairs2[1][2] = {{0, 1}};
  const int np = dim == 3 ? 3 : 1;
  for (int s = 0; s < np; ++s) {
    const int a = dim == 3 ? pairs3[s][0] : pairs2[s][0];
    const int b = dim == 3 ? pairs3[s][1] : pairs2[s][1];
    const int I = dim + s;
    P[I * D + a * dim + b] = r2;
    P[I * D + b * dim + a] = r2;
  }
  return P;
}

// element weight and per-direction gradient scale of the stiffness kernel's gradient coordinates
void kernel_scales(const fehom_ctx* ctx, double* w, double s[3]) {
  for (int i = 0; i < 3; ++i) {
    if (ctx->d.elem == HEX8_3D) s[i] = 1.0 / (4.0 * ctx->h[i]);        // d/dx = (2/h) d/dxi, modal sums carry 8
    else if (ctx->d.elem == Q1_2D) s[i] = 1.0 / (2.0 * ctx->h[i]);     // (2/h) / 4
    else s[i] = 1.0 / ctx->h[i];                                       // raw differences of P1
  }
  *w = (ctx->d.elem == P1TRI2_2D) ? 0.5 * ctx->vol : (ctx->d.elem == P1TRI4_2D ? 0.25 * ctx->vol : ctx->vol);
}

// Chat = w S P^T C P S  (D x D) for one material C (m x m)
void grad_material(const fehom_ctx* ctx, const double* C, double* out) {
  const int dim = ctx->d.dim, m = ctx->m, D = ctx->D;
  const std::vector<double> P = grad_to_flux(dim, ctx->physics);
  double w, s[3];
  kernel_scales(ctx, &w, s);
  std::vector<double> sc(D);
  for (int k = 0; k < D; ++k) sc[k] = s[k % dim];
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      double acc = 0.0;
      for (int I = 0; I < m; ++I)
        for (int J = 0; J < m; ++J) acc += P[I * D + a] * C[I * m + J] * P[J * D + b];
      out[a * D + b] = w * sc[a] * sc[b] * acc;
    }
}

// tau = w S P^T C e (D)
void grad_prestress(const fehom_ctx* ctx, const double* C, const double* e, double* out) {
  const int dim = ctx->d.dim, m = ctx->m, D = ctx->D;
  const std::vector<double> P = grad_to_flux(dim, ctx->physics);
  double w, s[3];
  kernel_scales(ctx, &w, s);
  for (int a = 0; a < D; ++a) {
    double acc = 0.0;
    for (int I = 0; I < m; ++I)
      for (int J = 0; J < m; ++J) acc += P[I * D + a] * C[I * m + J] * e[J];
    out[a] = w * s[a % dim] * acc;
  }
}

// isotropic elastic Mandel matrix C = lam J + 2 mu I ?
bool iso_elastic(const double* C, int dim, double* lam, double* mu) {
  const int m = dim * (dim + 1) / 2;
  double mx = 0;
  for (int i = 0; i < m * m; ++i) mx = std::max(mx, std::fabs(C[i]));
  const double l = C[0 * m + 1], mu2 = C[(m - 1) * m + (m - 1)];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double v = 0;
      if (i < dim && j < dim) v = l;
      if (i == j) v += mu2;
      if (std::fabs(C[i * m + j] - v) > 1e-13 * mx) return false;
    }
  *lam = l;
  *mu = 0.5 * mu2;
  return true;
}

// scalar conductivity C = k I (3 x 3) ?
bool iso_scalar(const double* C, double* k) {
  double mx = 0;
  for (int i = 0; i < 9; ++i) mx = std::max(mx, std::fabs(C[i]));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (std::fabs(C[i * 3 + j] - (i == j ? C[0] : 0.0)) > 1e-13 * mx) return false;
  *k = C[0];
  return true;
}

// the isotropic fast-path entry (kIsoStride values, gradient coordinates) of material C for hex8 on cubic
// voxels, or false when C is not isotropic
bool iso_material(const fehom_ctx* ctx, const double* C, double* out) {
  double w, sc[3];
  kernel_scales(ctx, &w, sc);
  const double f = w * sc[0] * sc[0];
  if (ctx->physics == FEHOM_ELASTIC) {
    double lam, mu;
    if (!iso_elastic(C, 3, &lam, &mu)) return false;
    iso_entry(f * lam, f * mu, out);
    return true;
  }
  double k;
  if (!iso_scalar(C, &k)) return false;
  iso_entry_scalar(f * k, out);
  return true;
}

// symmetric Jacobi eigen-decomposition (small n), for the k = 0 pseudo-inverse
void jacobi_eig(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& ev) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off < 1e-300) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
        const double c = 1 / std::sqrt(t * t + 1), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  ev.resize(n);
  for (int i = 0; i < n; ++i) ev[i] = A[i * n + i];
}

void fill_dims_args(fehom_ctx* ctx, FftArgs& f, bool fp32, int n_loads) {
  f.d = ctx->d;
  f.n_loads = n_loads;
  f.load_stride_f = (long long)ctx->d.c * ctx->d.N;
  f.load_stride_s = (long long)ctx->d.c * ctx->d.Nh;
  if (fp32) {
    f.tw = Twiddles{ctx->tw32[0], ctx->tw32[1], ctx->tw32[2]};
    f.sym = ctx->sym32;
  } else {
    f.tw = Twiddles{ctx->tw64[0], ctx->tw64[1], ctx->tw64[2]};
    f.sym = ctx->sym64;
  }
  f.st = nullptr;
  f.red = ctx->red;
  f.init = 0;
  f.mode = FX_PLAIN;
  f.f0 = nullptr;
  f.f1 = nullptr;
  f.f2 = nullptr;
  f.spec = fp32 ? (void*)ctx->spec32 : (void*)ctx->spec64;
  const auto& pl = ctx->plan[fp32 ? 1 : 0];
  f.pairs = pl.pairs;
  f.tc_y = pl.tc_y;
  f.tc_last = pl.tc_last;
  f.herm = ctx->d.elem == P1TRI4_2D ? 1 : 0;
  f.xy = (ctx->opt.fft_xy == 1 || (ctx->opt.fft_xy < 0 && pl.xy)) && fft_xy_supported(ctx->d, fp32) ? 1 : 0;
  f.last_reg =
      (ctx->opt.fft_xy == 1 || (ctx->opt.fft_xy < 0 && pl.last_reg)) && fft_last_rs_supported(ctx->d, fp32) ? 1 : 0;
}

// Removes the constant null mode from every load's field: the mean of each component, or for the
// two-node stencil the common mean of all nodes of both types (its only null mode).
cudaError_t sub_mean_fields(fehom_ctx* ctx, double* x, int n_loads, cudaStream_t s) {
  const long long cN = (long long)ctx->d.c * ctx->d.N;
  if (ctx->d.elem == P1TRI4_2D) return launch_sub_mean(x, 1, cN, n_loads, cN, ctx->partial, s);
  return launch_sub_mean(x, ctx->d.c, ctx->d.N, n_loads, cN, ctx->partial, s);
}

StencilArgs stencil_args(fehom_ctx* ctx, bool fp32, int n_loads) {
  StencilArgs a{};
  a.d = ctx->d;
  a.ids = ctx->ids;
  a.mats = fp32 ? (const void*)ctx->mats32 : (const void*)ctx->mats64;
  a.iso = ctx->iso ? (fp32 ? (const void*)ctx->iso32 : (const void*)ctx->iso64) : nullptr;
  a.tau = nullptr;
  a.n_phases = ctx->n_phases;
  a.n_loads = n_loads;
  a.load_stride = (long long)ctx->d.c * ctx->d.N;
  a.y_scale = 1.0;
  a.st = nullptr;
  a.red = ctx->red;
  a.tile_rows = ctx->stencil[fp32 ? 1 : 0].rows;
  a.staging = ctx->stencil[fp32 ? 1 : 0].staging;
  return a;
}

fehom_status grow64(fehom_ctx* ctx, int n) {
  if (n <= ctx->cap64) return FEHOM_OK;
  dfree(ctx->x64); dfree(ctx->r64); dfree(ctx->p64); dfree(ctx->ap64); dfree(ctx->b64); dfree(ctx->spec64);
  ctx->graph_key[0] = 0;
  const size_t f = (size_t)n * ctx->d.c * ctx->d.N, sp = (size_t)n * ctx->d.c * ctx->d.Nh;
  CK(cudaMalloc(&ctx->x64, f * sizeof(double)));
  CK(cudaMalloc(&ctx->r64, f * sizeof(double)));
  CK(cudaMalloc(&ctx->p64, f * sizeof(double)));
  CK(cudaMalloc(&ctx->ap64, f * sizeof(double)));
  CK(cudaMalloc(&ctx->b64, f * sizeof(double)));
  CK(cudaMalloc(&ctx->spec64, sp * sizeof(double2)));
  ctx->cap64 = n;
  return FEHOM_OK;
}

fehom_status grow32(fehom_ctx* ctx, int n) {
  if (n <= ctx->cap32) return FEHOM_OK;
  dfree(ctx->x32); dfree(ctx->r32); dfree(ctx->p32); dfree(ctx->ap32); dfree(ctx->spec32);
  ctx->graph_key[0] = 0;
  const size_t f = (size_t)n * ctx->d.c * ctx->d.N, sp = (size_t)n * ctx->d.c * ctx->d.Nh;
  CK(cudaMalloc(&ctx->x32, f * sizeof(float)));
  CK(cudaMalloc(&ctx->r32, f * sizeof(float)));
  CK(cudaMalloc(&ctx->p32, f * sizeof(float)));
  CK(cudaMalloc(&ctx->ap32, f * sizeof(float)));
  CK(cudaMalloc(&ctx->spec32, sp * sizeof(float2)));
  ctx->cap32 = n;
  return FEHOM_OK;
}

fehom_status ensure_partial(fehom_ctx* ctx, size_t n) {
  if (n <= ctx->partial_cap) return FEHOM_OK;
  dfree(ctx->partial);
  CK(cudaMalloc(&ctx->partial, n * sizeof(double)));
  ctx->partial_cap = n;
  return FEHOM_OK;
}

inline void count_launch(fehom_ctx* ctx, int n = 1) {
  if (ctx->counting) ctx->launches += n;
}

// event record that also works inside stream capture (becomes a timing node of the graph)
inline cudaError_t record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t err = cudaStreamIsCapturing(s, &cs);
  if (err != cudaSuccess) return err;
  if (cs == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  return cudaEventRecord(e, s);
}

// ------------------------------------------------------------------------------------------------
// preconditioner passes
// ------------------------------------------------------------------------------------------------
template <typename T>
cudaError_t fft_forward(fehom_ctx* ctx, FftArgs f, cudaStream_t s) {
  cudaError_t e = launch_fft_x_fwd<T>(f, s);
  if (e != cudaSuccess) return e;
  if (ctx->d.dim == 3 && (e = launch_fft_y<T>(f, 0, s)) != cudaSuccess) return e;
  return cudaSuccess;
}

// ev: optional [FEHOM_K_COUNT][2] events recorded around each pass (PCG profiling)
template <typename T>
cudaError_t precond_passes(fehom_ctx* ctx, FftArgs f, int fwd_mode, int inv_mode, void* fwd_field,
                           const void* fwd_ap, void* inv_f0, void* inv_f2, cudaStream_t s,
                           cudaEvent_t (*ev)[2] = nullptr) {
  cudaError_t e;
  auto timed = [&](int k, auto&& launch) -> cudaError_t {
    cudaError_t r;
    if (ev && (r = record(ev[k][0], s)) != cudaSuccess) return r;
    if ((r = launch()) != cudaSuccess) return r;
    count_launch(ctx);
    if (ev && (r = record(ev[k][1], s)) != cudaSuccess) return r;
    return cudaSuccess;
  };
  f.mode = fwd_mode;
  f.f0 = fwd_field;
  f.f1 = fwd_ap;
  if (f.xy) {  // fused x-y passes: their times are reported under the x classes
    if ((e = timed(FEHOM_K_FFT_X_FWD, [&] { return launch_fft_xy<T>(f, 0, s); })) != cudaSuccess) return e;
    if ((e = timed(FEHOM_K_FFT_LAST, [&] { return launch_fft_last_solve<T>(f, s); })) != cudaSuccess) return e;
    f.mode = inv_mode;
    f.f0 = inv_f0;
    f.f2 = inv_f2;
    return timed(FEHOM_K_FFT_X_INV, [&] { return launch_fft_xy<T>(f, 1, s); });
  }
  if ((e = timed(FEHOM_K_FFT_X_FWD, [&] { return launch_fft_x_fwd<T>(f, s); })) != cudaSuccess) return e;
  if (ctx->d.dim == 3 && (e = timed(FEHOM_K_FFT_Y_FWD, [&] { return launch_fft_y<T>(f, 0, s); })) != cudaSuccess) return e;
  if ((e = timed(FEHOM_K_FFT_LAST, [&] { return launch_fft_last_solve<T>(f, s); })) != cudaSuccess) return e;
  if (ctx->d.dim == 3 && (e = timed(FEHOM_K_FFT_Y_INV, [&] { return launch_fft_y<T>(f, 1, s); })) != cudaSuccess) return e;
  f.mode = inv_mode;
  f.f0 = inv_f0;
  f.f2 = inv_f2;
  return timed(FEHOM_K_FFT_X_INV, [&] { return launch_fft_x_inv<T>(f, s); });
}

// one PCG iteration for every active load
template <typename T>
cudaError_t pcg_iteration(fehom_ctx* ctx, int n_loads, T* x, T* r, T* p, T* ap, cudaStream_t s,
                          cudaEvent_t (*ev)[2] = nullptr) {
  const bool fp32 = sizeof(T) == 4;
  StencilArgs a = stencil_args(ctx, fp32, n_loads);
  a.x = p;
  a.y = ap;
  a.st = ctx->st;
  cudaError_t e;
  if (ev && (e = record(ev[FEHOM_K_STIFFNESS][0], s)) != cudaSuccess) return e;
  if ((e = launch_stiffness<T>(a, s)) != cudaSuccess) return e;
  count_launch(ctx);
  if (ev && (e = record(ev[FEHOM_K_STIFFNESS][1], s)) != cudaSuccess) return e;
  FftArgs f;
  fill_dims_args(ctx, f, fp32, n_loads);
  f.st = ctx->st;
  return precond_passes<T>(ctx, f, FX_PCG, FX_PCG, r, ap, x, p, s, ev);
}

fehom_status make_events(fehom_ctx* ctx) {
  if (ctx->events_made) return FEHOM_OK;
  for (int i = 0; i < kChunk; ++i)
    for (int k = 0; k < FEHOM_K_COUNT; ++k)
      for (int j = 0; j < 2; ++j) CK(cudaEventCreate(&ctx->ev[i][k][j]));
  ctx->events_made = true;
  return FEHOM_OK;
}

// accumulate the event times of the first `n_iter` iterations of the last chunk
fehom_status harvest_events(fehom_ctx* ctx, int prec, int n_iter) {
  const int nk = FEHOM_K_COUNT;
  for (int i = 0; i < std::min(n_iter, kChunk); ++i)
    for (int k = 0; k < nk; ++k) {
      const bool no_y = ctx->d.dim == 2 || (ctx->opt.fft_xy == 1 || (ctx->opt.fft_xy < 0 && ctx->plan[prec].xy)) &&
                                                fft_xy_supported(ctx->d, prec == 1);
      if (no_y && (k == FEHOM_K_FFT_Y_FWD || k == FEHOM_K_FFT_Y_INV)) continue;
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, ctx->ev[i][k][0], ctx->ev[i][k][1]));
      ctx->kms[prec][k] += ms;
      ctx->kcnt[prec][k] += 1;
    }
  return FEHOM_OK;
}

// Tuned launch plans shared by every context of the process.  A plan depends only on the device, the
// grid, the field blocks, the batch size, the precision and the options that restrict it, so a
// context of the same shape (a new cell of a series, a solver rebuilt per request) takes the first
// context's choice instead of timing the candidates again.
struct PlanKey {
  int v[12];
  bool operator<(const PlanKey& o) const { return std::lexicographical_compare(v, v + 12, o.v, o.v + 12); }
};
std::mutex g_plan_mu;
std::map<PlanKey, fehom_ctx::FftPlan> g_fft_plans;
std::map<PlanKey, fehom_ctx::StencilPlan> g_stencil_plans;

PlanKey plan_key(const fehom_ctx* ctx, int kind, int prec, int n_loads) {
  return PlanKey{{kind, prec, ctx->device, ctx->d.elem, ctx->d.dim, ctx->d.nx, ctx->d.ny, ctx->d.nz, ctx->d.c,
                  n_loads, kind == 0 ? ctx->opt.fft_xy : 0, kind == 1 ? (ctx->iso ? 1 : 0) : 0}};
}

// Launch-plan tuner of the FFT passes: each candidate is timed with CUDA events on the context's
// stream over the solve's own buffers (zeroed first), for the batch size of the solve.
template <typename T>
fehom_status autotune_fft(fehom_ctx* ctx, int n_loads) {
  const int prec = sizeof(T) == 4 ? 1 : 0;
  auto& pl = ctx->plan[prec];
  if (!ctx->opt.autotune || pl.tuned_loads == n_loads) return FEHOM_OK;
  // register-split passes forced on every axis: the generic passes are not used, nothing to time
  if (prec == 1 && ctx->opt.fft_xy == 1 && fft_xy_supported(ctx->d, true) && fft_last_rs_supported(ctx->d, true)) {
    pl.tuned_loads = n_loads;
    return FEHOM_OK;
  }
  const PlanKey key = plan_key(ctx, 0, prec, n_loads);
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    const auto it = g_fft_plans.find(key);
    if (it != g_fft_plans.end()) {
      pl = it->second;
      ctx->graph_key[0] = 0;  // captured iterations used the previous plan
      return FEHOM_OK;
    }
  }
  cudaStream_t s = ctx->stream;
  T* fin = prec ? (T*)ctx->r32 : (T*)ctx->r64;
  T* fout = prec ? (T*)ctx->ap32 : (T*)ctx->ap64;
  void* spec = prec ? (void*)ctx->spec32 : (void*)ctx->spec64;
  const size_t fb = sizeof(T) * (size_t)n_loads * ctx->d.c * ctx->d.N;
  const size_t sb = 2 * sizeof(T) * (size_t)n_loads * ctx->d.c * ctx->d.Nh;
  CK(cudaMemsetAsync(fin, 0, fb, s));
  CK(cudaMemsetAsync(spec, 0, sb, s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  FftArgs base;
  fill_dims_args(ctx, base, prec == 1, n_loads);
  base.st = nullptr;
  base.mode = FX_PLAIN;
  base.xy = 0;
  base.last_reg = 0;
  auto timeit = [&](auto&& body) -> double {
    if (body() != cudaSuccess) {
      cudaGetLastError();
      return -1.0;
    }
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r) body();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / 3.0;
  };
  auto pick = [&](const int* cand, int nc, auto&& body, int* best, double* best_ms) {
    *best = 0;
    *best_ms = 1e30;
    for (int i = 0; i < nc; ++i) {
      const double ms = timeit([&] { return body(cand[i]); });
      if (ms > 0 && ms < *best_ms) {
        *best_ms = ms;
        *best = cand[i];
      }
    }
  };
  const int pairs[3] = {16, 8, 4};
  const int tcs[4] = {16, 8, 4, 2};
  int bp, by = 0, bl;
  double mp, my = 0, ml;
  pick(pairs, 3, [&](int P) {
    FftArgs f = base;
    f.pairs = P;
    f.f0 = fin;
    cudaError_t e = launch_fft_x_fwd<T>(f, s);
    if (e != cudaSuccess) return e;
    f.f0 = fout;
    return launch_fft_x_inv<T>(f, s);
  }, &bp, &mp);
  if (ctx->d.dim == 3)
    pick(tcs, 4, [&](int TC) {
      FftArgs f = base;
      f.tc_y = TC;
      cudaError_t e = launch_fft_y<T>(f, 0, s);
      if (e != cudaSuccess) return e;
      return launch_fft_y<T>(f, 1, s);
    }, &by, &my);
  pick(tcs, 4, [&](int TC) {
    FftArgs f = base;
    f.tc_last = TC;
    return launch_fft_last_solve<T>(f, s);
  }, &bl, &ml);
  // fused x-y passes against the best separate x and y passes
  int xy = 0;
  if (ctx->opt.fft_xy < 0 && fft_xy_supported(ctx->d, prec == 1)) {
    const double mxy = timeit([&] {
      FftArgs f = base;
      f.f0 = fin;
      cudaError_t e = launch_fft_xy<T>(f, 0, s);
      if (e != cudaSuccess) return e;
      f.f0 = fout;
      return launch_fft_xy<T>(f, 1, s);
    });
    if (mxy > 0 && mxy < mp + my) {
      xy = 1;
      mp = mxy;
      my = 0;
    }
  }
  int last_reg = 0;
  if (ctx->opt.fft_xy < 0 && fft_last_rs_supported(ctx->d, prec == 1)) {
    const double mreg = timeit([&] {
      FftArgs f = base;
      f.last_reg = 1;
      return launch_fft_last_solve<T>(f, s);
    });
    if (mreg > 0 && mreg < ml) {
      last_reg = 1;
      ml = mreg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  pl.pairs = bp;
  pl.tc_y = by;
  pl.tc_last = bl;
  pl.xy = ctx->opt.fft_xy == 1 ? (fft_xy_supported(ctx->d, prec == 1) ? 1 : 0) : xy;
  pl.last_reg = ctx->opt.fft_xy == 1 ? (fft_last_rs_supported(ctx->d, prec == 1) ? 1 : 0) : last_reg;
  pl.ms[0] = mp;
  pl.ms[1] = my;
  pl.ms[2] = ml;
  pl.tuned_loads = n_loads;
  ctx->graph_key[0] = 0;  // captured iterations used the previous plan
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_fft_plans[key] = pl;
  }
  return FEHOM_OK;
}

// Stencil tuner: times the hex8 PCG stiffness apply with 8- and 16-row tiles (both precisions), and for
// the FP32 kernels on full x tiles with both node-plane stagings (cp.async copies by every thread, or one
// tensor-memory-accelerator box per plane), on the solve's buffers for the batch size of the solve, and
// keeps the fastest; option stencil_rows (8 or 16) fixes the height (cp.async staging).  The launches
// use running scratch states, not the solve's.
template <typename T>
fehom_status autotune_stencil(fehom_ctx* ctx, int n_loads) {
  const int prec = sizeof(T) == 4 ? 1 : 0;
  auto& sp = ctx->stencil[prec];
  if (ctx->d.elem != HEX8_3D) return FEHOM_OK;
  if (ctx->opt.stencil_rows == 8 || ctx->opt.stencil_rows == 16) {
    if (sp.rows != ctx->opt.stencil_rows || sp.staging != 0) ctx->graph_key[0] = 0;
    sp.rows = ctx->opt.stencil_rows;
    sp.staging = 0;
    sp.tuned_loads = n_loads;
    return FEHOM_OK;
  }
  if (!ctx->opt.autotune || sp.tuned_loads == n_loads) return FEHOM_OK;
  const PlanKey key = plan_key(ctx, 1, prec, n_loads);
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    const auto it = g_stencil_plans.find(key);
    if (it != g_stencil_plans.end()) {
      if (sp.rows != it->second.rows || sp.staging != it->second.staging) ctx->graph_key[0] = 0;
      sp = it->second;
      return FEHOM_OK;
    }
  }
  cudaStream_t s = ctx->stream;
  if (!ctx->tune_st) CK(cudaMalloc(&ctx->tune_st, sizeof(PcgState) * kMaxLoads));
  std::vector<PcgState> hs(n_loads);
  for (auto& st : hs) {
    std::memset(&st, 0, sizeof(st));
    st.state = ST_RUN;
    st.rz = 1.0;
  }
  T* pin = prec ? (T*)ctx->p32 : (T*)ctx->p64;
  T* pout = prec ? (T*)ctx->ap32 : (T*)ctx->ap64;
  // every component field of every load takes two values (a step halfway through its planes), so
  // <p, K p> > 0 and the running states stay running (a zero or constant p would end them by
  // breakdown and the timed launches would be empty)
  const size_t row = sizeof(T) * (size_t)ctx->d.N, half = sizeof(T) * (size_t)(ctx->d.N / 2);
  const size_t rows = (size_t)n_loads * ctx->d.c;
  CK(cudaMemset2DAsync(pin, row, 0x3F, half, rows, s));
  CK(cudaMemset2DAsync(reinterpret_cast<char*>(pin) + half, row, 0x40, row - half, rows, s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e30;
  int rows_best = 0, staging_best = 0;
  for (int ci = 0; ci < 4; ++ci) {
    const int rows = (ci & 1) ? 16 : 8, staging = ci < 2 ? 0 : 3;
    sp.ms[ci] = 0.0;
    if (staging == 3 && prec == 0) continue;  // the FP64 kernels stage nothing
    StencilArgs a = stencil_args(ctx, prec == 1, n_loads);
    a.x = pin;
    a.y = pout;
    a.st = ctx->tune_st;
    a.red.hist = nullptr;
    a.tile_rows = rows;
    a.staging = staging;
    CK(cudaMemcpyAsync(ctx->tune_st, hs.data(), sizeof(PcgState) * n_loads, cudaMemcpyHostToDevice, s));
    double ms = -1.0;
    if (launch_stiffness<T>(a, s) == cudaSuccess) {
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3; ++r) launch_stiffness<T>(a, s);
      cudaEventRecord(e1, s);
      float t = 0.f;
      if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = t / 3.0;
    }
    cudaGetLastError();
    count_launch(ctx, 4);
    sp.ms[ci] = ms;
    if (ms > 0 && ms < best) {
      best = ms;
      rows_best = rows;
      staging_best = staging;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rows_best == 0) FAIL(FEHOM_E_CUDA, "stencil tuner: no candidate ran");
  sp.rows = rows_best;
  sp.staging = staging_best;
  sp.tuned_loads = n_loads;
  ctx->graph_key[0] = 0;  // captured iterations used the previous tile
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_stencil_plans[key] = sp;
  }
  return FEHOM_OK;
}

template <typename T>
fehom_status run_iterations(fehom_ctx* ctx, int n_loads, T* x, T* r, T* p, T* ap, int max_iter,
                            std::vector<PcgState>& hs) {
  cudaStream_t s = ctx->stream;
  const auto& spl = ctx->stencil[sizeof(T) == 4 ? 1 : 0];
  const long long key[8] = {(ctx->opt.profile ? 2 : 1) + 4 * spl.rows + 1024 * spl.staging, (long long)n_loads, (long long)(size_t)x, (long long)(size_t)r, (long long)(size_t)p,
                            (long long)(size_t)ap, (long long)sizeof(T), (long long)(size_t)ctx->st};
  const bool prof = ctx->opt.profile != 0;
  if (prof) TRY(make_events(ctx));
  const int prec = sizeof(T) == 4 ? 1 : 0;
  bool use_graph = ctx->opt.use_graph != 0;
  if (use_graph && std::memcmp(key, ctx->graph_key, sizeof(key)) != 0) {
    if (ctx->graph_exec) {
      cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
    }
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    const long long before = ctx->launches;
    for (int i = 0; i < kChunk && e == cudaSuccess; ++i)
      e = pcg_iteration<T>(ctx, n_loads, x, r, p, ap, s, prof ? ctx->ev[i] : nullptr);
    ctx->graph_launches = (int)(ctx->launches - before);
    ctx->launches = before;  // captured kernels are counted when the graph is replayed
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    CK(e);
    CK(e2);
    CK(cudaGraphInstantiate(&ctx->graph_exec, g, 0));
    cudaGraphDestroy(g);
    std::memcpy(ctx->graph_key, key, sizeof(key));
  }
  hs.resize(n_loads);
  std::vector<PcgState> prev(n_loads);
  CK(cudaMemcpyAsync(prev.data(), ctx->st, sizeof(PcgState) * n_loads, cudaMemcpyDeviceToHost, s));
  for (int done = 0; done < max_iter + kChunk;) {
    if (use_graph) {
      CK(cudaGraphLaunch(ctx->graph_exec, s));
      ctx->launches += ctx->graph_launches;
    } else {
      for (int i = 0; i < kChunk; ++i) CK(pcg_iteration<T>(ctx, n_loads, x, r, p, ap, s, prof ? ctx->ev[i] : nullptr));
    }
    done += kChunk;
    CK(cudaMemcpyAsync(hs.data(), ctx->st, sizeof(PcgState) * n_loads, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (prof) {
      int worked = 0;
      for (int l = 0; l < n_loads; ++l) worked = std::max(worked, hs[l].iter - prev[l].iter);
      TRY(harvest_events(ctx, prec, worked));
      prev = hs;
    }
    bool all = true;
    for (int l = 0; l < n_loads; ++l)
      if (hs[l].state == ST_RUN || hs[l].state == ST_CONV || hs[l].state == ST_FIN_MAX) all = false;
    if (all) break;
  }
  for (int l = 0; l < n_loads; ++l) ctx->hist_count[l] = std::min(hs[l].iter, kHist);
  return FEHOM_OK;
}

// initial preconditioner apply of PCG: z0 = K_ref^+ r0, p0 = z0, rz0, bnorm2
template <typename T>
fehom_status pcg_init(fehom_ctx* ctx, int n_loads, T* r, T* p) {
  FftArgs f;
  fill_dims_args(ctx, f, sizeof(T) == 4, n_loads);
  f.st = ctx->st;
  f.init = 1;
  CK(precond_passes<T>(ctx, f, FX_PLAIN, FX_PCG_INIT, r, nullptr, nullptr, p, ctx->stream));
  return FEHOM_OK;
}

fehom_status set_states(fehom_ctx* ctx, int n_loads, double tol_rel, int max_iter, double bnorm2) {
  std::vector<PcgState> hs(n_loads);
  for (auto& s : hs) {
    std::memset(&s, 0, sizeof(s));
    s.bnorm2 = bnorm2;
    s.tol2_rel = tol_rel * tol_rel;
    s.state = ST_RUN;
    s.max_iter = max_iter;
  }
  CK(cudaMemcpyAsync(ctx->st, hs.data(), sizeof(PcgState) * n_loads, cudaMemcpyHostToDevice, ctx->stream));
  return FEHOM_OK;
}

// per-phase prestress tau_l = w S P^T C_p e_l of every load, uploaded for the stiffness kernel
fehom_status upload_tau(fehom_ctx* ctx, int n_loads, const double* loads) {
  const int P = ctx->n_phases, D = ctx->D;
  std::vector<double> tau((size_t)n_loads * P * D);
  for (int l = 0; l < n_loads; ++l)
    for (int ph = 0; ph < P; ++ph)
      grad_prestress(ctx, &ctx->moduli[(size_t)ph * ctx->m * ctx->m], loads + (size_t)l * ctx->m,
                     &tau[((size_t)l * P + ph) * D]);
  dfree(ctx->tau);
  CK(cudaMalloc(&ctx->tau, tau.size() * sizeof(double)));
  CK(cudaMemcpyAsync(ctx->tau, tau.data(), tau.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  std::vector<float> tdf(2 * tau.size());
  for (size_t i = 0; i < tau.size(); ++i) {
    tdf[2 * i] = (float)tau[i];
    tdf[2 * i + 1] = (float)(tau[i] - (double)tdf[2 * i]);
  }
  dfree(ctx->taudf);
  CK(cudaMalloc(&ctx->taudf, tdf.size() * sizeof(float)));
  CK(cudaMemcpyAsync(ctx->taudf, tdf.data(), tdf.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  return FEHOM_OK;
}

// y = -D^T W C (e_l + D x_l) for every load (x == NULL: the right-hand side b = -D^T W C e), in FP64,
// with the fused statistics: y2[l] = ||y_l||^2 and flux[l] = <sigma>_l (Sec. 2 average with the
// quadrature of Eq. global_sum), recovered from the summed monomial-1 duals as P S^-1 sum T / |Y|.
// Needs upload_tau for the same loads first.
// Volume-averaged flux / stress of every load from the sums T (n_loads x D) of the monomial-1 duals
// over all elements (sum T = |Y| S P^T <sigma>).
void sums_to_flux(const fehom_ctx* ctx, int n_loads, const std::vector<double>& T, std::vector<double>* flux) {
  const int dim = ctx->d.dim, m = ctx->m, D = ctx->D;
  const std::vector<double> P = grad_to_flux(dim, ctx->physics);
  double w, sc[3];
  kernel_scales(ctx, &w, sc);
  double cell = 1.0;
  const int n3[3] = {ctx->d.nx, ctx->d.ny, ctx->d.nz};
  for (int i = 0; i < dim; ++i) cell *= ctx->h[i] * n3[i];
  flux->assign((size_t)n_loads * m, 0.0);
  for (int l = 0; l < n_loads; ++l)
    for (int I = 0; I < m; ++I) {
      double v = 0.0;
      for (int q = 0; q < D; ++q) v += P[I * D + q] * T[(size_t)l * D + q] / sc[q % dim];
      (*flux)[(size_t)l * m + I] = v / cell;
    }
}

// Per-load sums of the stiffness statistics partials [load][cta][1 + D]: y2 = sum y^2, T = dual sums.
fehom_status reduce_stats(fehom_ctx* ctx, int n_loads, int ctas, std::vector<double>* y2, std::vector<double>* T) {
  const int D = ctx->D, W = 1 + D;
  std::vector<double> hp((size_t)n_loads * ctas * W);
  CK(cudaMemcpyAsync(hp.data(), ctx->partial, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (y2) y2->assign(n_loads, 0.0);
  if (T) T->assign((size_t)n_loads * D, 0.0);
  for (int l = 0; l < n_loads; ++l)
    for (int b = 0; b < ctas; ++b) {  // fixed order
      const double* pb = &hp[((size_t)l * ctas + b) * W];
      if (y2) (*y2)[l] += pb[0];
      if (T)
        for (int i = 0; i < D; ++i) (*T)[(size_t)l * D + i] += pb[1 + i];
    }
  return FEHOM_OK;
}

fehom_status residual_stats(fehom_ctx* ctx, int n_loads, const double* x, double* y, std::vector<double>* y2,
                            std::vector<double>* flux, std::vector<double>* tsum = nullptr) {
  StencilArgs a = stencil_args(ctx, false, n_loads);
  a.x = x;
  a.y = y;
  a.tau = ctx->tau;
  a.y_scale = -1.0;
  const int ctas = stiffness_ctas(ctx->d, n_loads);
  const int W = 1 + ctx->D;
  TRY(ensure_partial(ctx, (size_t)n_loads * ctas * W));
  a.stats = ctx->partial;
  int got = 0;
  CK(launch_stiffness<double>(a, ctx->stream, &got));
  count_launch(ctx);
  if (got != ctas) FAIL(FEHOM_E_CUDA, "stiffness statistics: CTA count mismatch");
  std::vector<double> T;
  TRY(reduce_stats(ctx, n_loads, ctas, y2, &T));
  if (flux) sums_to_flux(ctx, n_loads, T, flux);
  if (tsum) *tsum = T;
  return FEHOM_OK;
}

// Refinement residual in double-float arithmetic: r_out = r_in - K d for FP32 corrections d
// (hex8 elasticity, isotropic phases, cubic voxels), with ||r_out||^2 and the dual sums of d.
bool residual_df_supported(const fehom_ctx* ctx) {
  return ctx->isodf != nullptr && ctx->d.elem == HEX8_3D && ctx->d.c == 3;
}

fehom_status residual_update_df(fehom_ctx* ctx, int n_loads, const float* d, const double* r_in, double* r_out,
                                std::vector<double>* y2, std::vector<double>* dT) {
  StencilArgs a = stencil_args(ctx, true, n_loads);
  a.x = d;
  a.y = r_out;
  a.iso = ctx->isodf;
  const int ctas = residual_df_ctas(ctx->d, n_loads);
  TRY(ensure_partial(ctx, (size_t)n_loads * ctas * (1 + ctx->D)));
  a.stats = ctx->partial;
  int got = 0;
  CK(launch_residual_df(a, r_in, nullptr, ctx->stream, &got));
  count_launch(ctx);
  if (got != ctas) FAIL(FEHOM_E_CUDA, "double-float residual: CTA count mismatch");
  return reduce_stats(ctx, n_loads, ctas, y2, dT);
}

// Right-hand side b = -D^T W C e of every load in double-float arithmetic (after upload_tau), with
// ||b||^2 and the prestress sums (the dual sums at zero fluctuation).
fehom_status rhs_df(fehom_ctx* ctx, int n_loads, double* b, std::vector<double>* y2, std::vector<double>* T) {
  StencilArgs a = stencil_args(ctx, true, n_loads);
  a.x = nullptr;
  a.y = b;
  const int ctas = residual_df_ctas(ctx->d, n_loads);
  TRY(ensure_partial(ctx, (size_t)n_loads * ctas * (1 + ctx->D)));
  a.stats = ctx->partial;
  int got = 0;
  CK(launch_residual_df(a, nullptr, ctx->taudf, ctx->stream, &got));
  count_launch(ctx);
  if (got != ctas) FAIL(FEHOM_E_CUDA, "double-float right-hand side: CTA count mismatch");
  return reduce_stats(ctx, n_loads, ctas, y2, T);
}

// --------------------------------------------------------------------------------------------------
// Allocation-free volume average (fehom_mean_flux_noalloc).  Its scratch is this fixed device array:
// every GPU that loads the library holds it until the process exits.  Layout per call: the per-CTA
// partial sums [ctas][1 + D], then the reduced sums [1 + D], then the per-phase prestress [P][D].
// --------------------------------------------------------------------------------------------------
constexpr int kNoallocDoubles = 8192;  // 64 KiB
constexpr int kMaxDevices = 64;
__device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[kMaxDevices] = {};

// gradient -> flux map P (m x D, row-major) into a caller-provided array (no heap use)
void flux_map_into(int dim, int physics, double* P) {
  const int m = physics == FEHOM_SCALAR ? dim : dim * (dim + 1) / 2;
  const int D = physics == FEHOM_SCALAR ? dim : dim * dim;
  for (int i = 0; i < m * D; ++i) P[i] = 0.0;
  if (physics == FEHOM_SCALAR) {
    for (int i = 0; i < dim; ++i) P[i * D + i] = 1.0;
    return;
  }
  for (int a = 0; a < dim; ++a) P[a * D + a * dim + a] = 1.0;
  const double r2 = 1.0 / std::sqrt(2.0);
  const int pairs[3][2] = {{1, 2}, {0, 2}, {0, 1}};
  for (int k = 0; k < (dim == 3 ? 3 : 1); ++k) {
    const int a = dim == 3 ? pairs[k][0] : 0, b = dim == 3 ? pairs[k][1] : 1;
    P[(dim + k) * D + a * dim + b] = r2;
    P[(dim + k) * D + b * dim + a] = r2;
  }
}

// sums the per-CTA partials column by column in CTA order (the order the host uses elsewhere)
__global__ void noalloc_sum_kernel(double* scratch, int ctas, int W) {
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < ctas; ++b) acc += scratch[(long long)b * W + i];
    scratch[(long long)ctas * W + i] = acc;
  }
}

// device address of the scratch array on the context's device, looked up once per device with that
// device current (the host-side symbol is only a stand-in and must never reach a kernel)
fehom_status noalloc_scratch(fehom_ctx* ctx, double** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  const int dev = ctx->device;
  if (dev < 0 || dev >= kMaxDevices) FAIL(FEHOM_E_INVALID, "device index out of range for the fixed scratch table");
  if (!g_noalloc_addr[dev]) {
    int prev = 0;
    CK(cudaGetDevice(&prev));
    if (prev != dev) CK(cudaSetDevice(dev));
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev != dev) cudaSetDevice(prev);
    CK(e);
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return FEHOM_OK;
}

}  // namespace

// ==================================================================================================
// C ABI
// ==================================================================================================
extern "C" {

void fehom_default_options(fehom_options* opt) {
  if (!opt) return;
  opt->precision = FEHOM_FP64;
  opt->max_iter = 10000;
  opt->inner_tol = 1e-3;
  opt->stream = nullptr;
  opt->use_graph = 1;
  opt->profile = 0;
  opt->autotune = 1;
  opt->x0_scaling = 1;
  opt->fft_xy = -1;
  opt->residual_df = 1;
  opt->stencil_rows = 0;
}

const char* fehom_last_error(const fehom_ctx* ctx) { return ctx ? ctx->err.c_str() : g_setup_error.c_str(); }

fehom_status fehom_kernel_times(const fehom_ctx* ctx, int precision, double* ms, int64_t* count) {
  if (!ctx || !ms || !count) return FEHOM_E_INVALID;
  const int p = precision == FEHOM_MIXED ? 1 : 0;
  for (int k = 0; k < FEHOM_K_COUNT; ++k) {
    ms[k] = ctx->kms[p][k];
    count[k] = ctx->kcnt[p][k];
  }
  return FEHOM_OK;
}

fehom_status fehom_pcg_coefficients(fehom_ctx* ctx, int load, int capacity, double* alpha, double* beta, int* count) {
  if (!ctx || !alpha || !beta || !count || load < 0 || load >= kMaxLoads || capacity < 0) return FEHOM_E_INVALID;
  const int n = std::min(capacity, ctx->hist_count[load]);
  *count = n;
  if (n == 0) return FEHOM_OK;
  CK(cudaMemcpyAsync(alpha, ctx->red.hist + (size_t)load * 2 * kHist, sizeof(double) * n, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaMemcpyAsync(beta, ctx->red.hist + ((size_t)load * 2 + 1) * kHist, sizeof(double) * n,
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FEHOM_OK;
}

fehom_status fehom_eig_bounds(fehom_ctx* ctx, double* lo_values, int64_t* lo_counts, int* n_lo, double* hi_values,
                              int64_t* hi_counts, int* n_hi) {
  if (!ctx || !lo_values || !lo_counts || !n_lo || !hi_values || !hi_counts || !n_hi) return FEHOM_E_INVALID;
  if (ctx->d.elem == P1TRI4_2D) FAIL(FEHOM_E_INVALID, "fehom_eig_bounds: not available for the two-node stencil");
  const int m = ctx->m, P = ctx->n_phases;
  // extreme generalized eigenvalues of (C_p, C_ref): eigenvalues of L^-1 C_p L^-T with C_ref = L L^T
  std::vector<double> L((size_t)m * m, 0.0);
  const double* R = ctx->cref.data();
  for (int j = 0; j < m; ++j) {
    double sj = R[j * m + j];
    for (int k = 0; k < j; ++k) sj -= L[j * m + k] * L[j * m + k];
    L[j * m + j] = std::sqrt(sj);
    for (int i = j + 1; i < m; ++i) {
      double t = R[i * m + j];
      for (int k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
      L[i * m + j] = t / L[j * m + j];
    }
  }
  auto lsolve = [&](std::vector<double>& B) {  // B <- L^-1 B (column by column)
    for (int col = 0; col < m; ++col)
      for (int i = 0; i < m; ++i) {
        double t = B[i * m + col];
        for (int k = 0; k < i; ++k) t -= L[i * m + k] * B[k * m + col];
        B[i * m + col] = t / L[i * m + i];
      }
  };
  std::vector<double> lo(P), hi(P);
  for (int p = 0; p < P; ++p) {
    std::vector<double> A(ctx->moduli.begin() + (size_t)p * m * m, ctx->moduli.begin() + (size_t)(p + 1) * m * m);
    lsolve(A);                                    // L^-1 C
    std::vector<double> At((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) At[i * m + j] = A[j * m + i];
    lsolve(At);                                   // L^-1 (L^-1 C)^T = L^-1 C L^-T (symmetric)
    std::vector<double> V, ev;
    jacobi_eig(m, At, V, ev);
    lo[p] = *std::min_element(ev.begin(), ev.end());
    hi[p] = *std::max_element(ev.begin(), ev.end());
  }
  double* dv = nullptr;
  unsigned long long* dh = nullptr;
  CK(cudaMalloc(&dv, sizeof(double) * 2 * P));
  CK(cudaMalloc(&dh, sizeof(unsigned long long) * 512));
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(dv, lo.data(), sizeof(double) * P, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dv + P, hi.data(), sizeof(double) * P, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(dh, 0, sizeof(unsigned long long) * 512, s));
  CK(launch_eig_bounds(ctx->d, ctx->ids, dv, dv + P, dh, dh + 256, s));
  count_launch(ctx);
  std::vector<unsigned long long> hh(512);
  CK(cudaMemcpyAsync(hh.data(), dh, sizeof(unsigned long long) * 512, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  cudaFree(dv);
  cudaFree(dh);
  // (value, count) lists, ascending, equal values merged; each node counts once per DOF
  auto emit = [&](const std::vector<double>& val, const unsigned long long* h, double* ov, int64_t* oc, int* n) {
    std::vector<std::pair<double, long long>> e;
    for (int p = 0; p < P; ++p)
      if (h[p]) e.push_back({val[p], (long long)h[p] * ctx->d.c});
    std::sort(e.begin(), e.end());
    int k = 0;
    for (size_t i = 0; i < e.size(); ++i) {
      if (k > 0 && ov[k - 1] == e[i].first) {
        oc[k - 1] += e[i].second;
      } else {
        ov[k] = e[i].first;
        oc[k] = e[i].second;
        ++k;
      }
    }
    *n = k;
  };
  emit(lo, hh.data(), lo_values, lo_counts, n_lo);
  emit(hi, hh.data() + 256, hi_values, hi_counts, n_hi);
  return FEHOM_OK;
}

fehom_status fehom_fft_plan(const fehom_ctx* ctx, int precision, int* pairs, int* tc_y, int* tc_last, double* ms,
                            int* xy_fused) {
  if (!ctx) return FEHOM_E_INVALID;
  const auto& pl = ctx->plan[precision == FEHOM_MIXED ? 1 : 0];
  if (xy_fused) {
    const bool fp32 = precision == FEHOM_MIXED;
    const int a = (ctx->opt.fft_xy == 1 || (ctx->opt.fft_xy < 0 && pl.xy)) && fft_xy_supported(ctx->d, fp32);
    const int b = (ctx->opt.fft_xy == 1 || (ctx->opt.fft_xy < 0 && pl.last_reg)) && fft_last_rs_supported(ctx->d, fp32);
    *xy_fused = a | (b << 1);
  }
  if (pairs) *pairs = pl.pairs;
  if (tc_y) *tc_y = pl.tc_y;
  if (tc_last) *tc_last = pl.tc_last;
  if (ms)
    for (int i = 0; i < 3; ++i) ms[i] = pl.ms[i];
  return FEHOM_OK;
}

fehom_status fehom_stencil_plan(const fehom_ctx* ctx, int precision, int* rows, int* staging, double* ms) {
  if (!ctx) return FEHOM_E_INVALID;
  const auto& sp = ctx->stencil[precision == FEHOM_MIXED ? 1 : 0];
  if (rows) *rows = sp.rows != 0 ? sp.rows : (precision == FEHOM_MIXED ? 8 : 16);
  if (staging) *staging = sp.staging;
  if (ms)
    for (int i = 0; i < 4; ++i) ms[i] = sp.ms[i];
  return FEHOM_OK;
}

fehom_status fehom_set_reference(fehom_ctx* ctx, const double* C_ref) {
  if (!ctx || !C_ref) return FEHOM_E_INVALID;
  const int m = ctx->m;
  if (!spd(C_ref, m)) FAIL(FEHOM_E_INVALID, "C_ref must be symmetric positive definite");
  cudaStream_t s = ctx->stream;
  ctx->cref.assign(C_ref, C_ref + (size_t)m * m);
  std::vector<double> rm((size_t)ctx->D * ctx->D);
  grad_material(ctx, C_ref, rm.data());
  CK(cudaMemcpyAsync(ctx->rmats64, rm.data(), rm.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  ctx->iso_ref = false;
  double ri[kIsoStride];
  if (ctx->iso && iso_material(ctx, C_ref, ri)) {
    if (!ctx->riso64) CK(cudaMalloc(&ctx->riso64, kIsoStride * sizeof(double)));
    CK(cudaMemcpyAsync(ctx->riso64, ri, kIsoStride * sizeof(double), cudaMemcpyHostToDevice, s));
    ctx->iso_ref = true;
  }
  CK(cudaStreamSynchronize(s));
  ctx->built = false;
  return FEHOM_OK;
}

// Algorithm 1 (Newton) for the power-law conductivity of nl_element_kernel; linear solves by PCG with
// the FFT preconditioner of the volume-mean tangent, rebuilt every Newton step (Algorithm 2).
fehom_status fehom_newton_solve(fehom_ctx* ctx, const double* e, const double* power_n, double g0, double tol_cg,
                                double eta_nw, int max_newton, double* fluct_out, int fluct_on_device,
                                double* mean_flux_out, fehom_newton_info* info) {
  if (!ctx || !e || !power_n || !info) return FEHOM_E_INVALID;
  if (ctx->physics != FEHOM_SCALAR || ctx->d.elem != HEX8_3D)
    FAIL(FEHOM_E_INVALID, "fehom_newton_solve: scalar conductivity on FEHOM_HEX8_3D only");
  if (!(g0 > 0.0) || !(tol_cg > 0.0 && tol_cg < 1.0) || !(eta_nw > 0.0) || max_newton < 1 || max_newton > 32)
    FAIL(FEHOM_E_INVALID, "need g0 > 0, 0 < tol_cg < 1, eta_nw > 0, 1 <= max_newton <= 32");
  const int P = ctx->n_phases;
  std::vector<double> kp(P), np(power_n, power_n + P);
  for (int p = 0; p < P; ++p) {
    const double* C = &ctx->moduli[(size_t)p * 9];
    const bool iso = C[1] == 0 && C[2] == 0 && C[3] == 0 && C[5] == 0 && C[6] == 0 && C[7] == 0 && C[0] == C[4] &&
                     C[4] == C[8];
    if (!iso) FAIL(FEHOM_E_INVALID, "fehom_newton_solve: phase conductivities must be isotropic (k I)");
    if (!(np[p] > 0.0) || !std::isfinite(np[p])) FAIL(FEHOM_E_INVALID, "power_n must be positive");
    kp[p] = C[0];
  }
  std::memset(info, 0, sizeof(*info));
  cudaStream_t s = ctx->stream;
  TRY(grow64(ctx, 1));
  const long long N = ctx->d.N;
  const int nb = nl_blocks(N), vb = nl_vec_blocks();
  double *u = nullptr, *T = nullptr, *E = nullptr, *z = nullptr, *dk = nullptr, *dpart = nullptr;
  struct Free {
    std::vector<void*> p;
    ~Free() { for (void* q : p) cudaFree(q); }
  } guard;
  auto dalloc = [&](double** q, size_t n) -> cudaError_t {
    cudaError_t r = cudaMalloc(q, n * sizeof(double));
    if (r == cudaSuccess) guard.p.push_back(*q);
    return r;
  };
  CK(dalloc(&u, N));
  CK(dalloc(&T, (size_t)N * 48));
  CK(dalloc(&E, (size_t)N * 8));
  CK(dalloc(&z, N));
  CK(dalloc(&dk, 2 * P));
  CK(dalloc(&dpart, (size_t)std::max(nb * 9, vb)));
  CK(cudaMemcpyAsync(dk, kp.data(), P * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dk + P, np.data(), P * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(u, 0, N * sizeof(double), s));
  NlArgs base{};
  base.d = ctx->d;
  for (int i = 0; i < 3; ++i) base.h[i] = ctx->h[i];
  base.vvox = ctx->vol;
  base.ids = ctx->ids;
  base.kp = dk;
  base.np = dk + P;
  base.g0 = g0;
  base.T = T;
  base.E = E;
  base.partial = dpart;
  for (int i = 0; i < 3; ++i) base.e[i] = e[i];
  const double volY = ctx->vol * (double)N;
  std::vector<double> hp((size_t)std::max(nb * 9, vb));
  auto sum_partials = [&](int blocks, int stride, int r, double* out) -> fehom_status {
    CK(cudaMemcpyAsync(hp.data(), dpart, sizeof(double) * blocks * stride, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double acc = 0.0;
    for (int b = 0; b < blocks; ++b) acc += hp[(size_t)b * stride + r];
    *out = acc;
    return FEHOM_OK;
  };
  auto dot = [&](const double* x, const double* y, double* out) -> fehom_status {
    CK(launch_nl_dot(N, x, y, dpart, s));
    return sum_partials(vb, 1, 0, out);
  };
  auto flux_and_tangent = [&](double* qbar, double* Abar) -> fehom_status {
    NlArgs a = base;
    a.x = u;
    CK(launch_nl_element(a, 0, s));
    count_launch(ctx);
    for (int r = 0; r < 3; ++r) TRY(sum_partials(nb, 9, r, &qbar[r]));
    for (int r = 0; r < 6; ++r) TRY(sum_partials(nb, 9, 3 + r, &Abar[r]));
    for (int r = 0; r < 3; ++r) qbar[r] /= volY;
    for (int r = 0; r < 6; ++r) Abar[r] /= volY;
    return FEHOM_OK;
  };
  auto grad_norm2 = [&](const double* x, double* out) -> fehom_status {
    NlArgs a = base;
    a.x = x;
    CK(launch_nl_element(a, 2, s));
    count_launch(ctx);
    return sum_partials(nb, 1, 0, out);
  };
  auto precond = [&](const double* r, double* zz) -> fehom_status {
    FftArgs f;
    fill_dims_args(ctx, f, false, 1);
    CK(precond_passes<double>(ctx, f, FX_PLAIN, FX_PLAIN, const_cast<double*>(r), nullptr, zz, nullptr, s));
    return FEHOM_OK;
  };
  double qbar[3], Abar[6];
  for (int it = 0; it < max_newton; ++it) {
    // residual R(u) = D^T W q(e + D u) (b = -R) and the tangent at u
    TRY(flux_and_tangent(qbar, Abar));
    {
      NlArgs a = base;
      a.y = ctx->b64;
      CK(launch_nl_gather(a, -1.0, 0, s));
      count_launch(ctx);
    }
    double bb;
    TRY(dot(ctx->b64, ctx->b64, &bb));
    info->residual[it] = std::sqrt(bb);
    // reference material = volume mean of the tangent; Algorithm 2 again
    const double Cref[9] = {Abar[0], Abar[5], Abar[4], Abar[5], Abar[1], Abar[3], Abar[4], Abar[3], Abar[2]};
    TRY(fehom_set_reference(ctx, Cref));
    TRY(fehom_precond_build(ctx));
    // PCG on K_t delta = b, delta in x64 (stopping test of Sec. 6, normalised by b)
    CK(cudaMemsetAsync(ctx->x64, 0, N * sizeof(double), s));
    CK(cudaMemcpyAsync(ctx->r64, ctx->b64, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TRY(precond(ctx->r64, z));
    double rz;
    TRY(dot(ctx->r64, z, &rz));
    const double bz = rz;
    int k = 0;
    if (bz > 0.0) {
      CK(cudaMemcpyAsync(ctx->p64, z, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      for (k = 1; k <= ctx->opt.max_iter; ++k) {
        NlArgs a = base;
        a.x = ctx->p64;
        CK(launch_nl_element(a, 1, s));
        a.y = ctx->ap64;
        CK(launch_nl_gather(a, 1.0, 1, s));
        count_launch(ctx, 2);
        double pAp;
        TRY(sum_partials(nb, 1, 0, &pAp));
        if (!(pAp > 0.0) || !std::isfinite(pAp)) FAIL(FEHOM_E_BREAKDOWN, "Newton: non-positive curvature in PCG");
        const double alpha = rz / pAp;
        CK(launch_nl_axpby(N, alpha, ctx->p64, 1.0, ctx->x64, nullptr, nullptr, s));
        CK(launch_nl_axpby(N, -alpha, ctx->ap64, 1.0, ctx->r64, nullptr, nullptr, s));
        TRY(precond(ctx->r64, z));
        double rz_new;
        TRY(dot(ctx->r64, z, &rz_new));
        count_launch(ctx, 3);
        if (std::sqrt(std::max(rz_new, 0.0)) <= tol_cg * std::sqrt(bz)) break;
        CK(launch_nl_axpby(N, 1.0, z, rz_new / rz, ctx->p64, nullptr, nullptr, s));
        count_launch(ctx);
        rz = rz_new;
      }
      if (k > ctx->opt.max_iter) k = ctx->opt.max_iter;
    }
    info->pcg_per_step[it] = k;
    info->pcg_iterations += k;
    CK(launch_nl_axpby(N, 1.0, ctx->x64, 1.0, u, nullptr, nullptr, s));
    count_launch(ctx);
    double dd, uu;
    TRY(grad_norm2(ctx->x64, &dd));
    TRY(grad_norm2(u, &uu));
    const double ratio = uu > 0.0 ? std::sqrt(dd / uu) : 0.0;
    info->increment[it] = ratio;
    info->newton_iterations = it + 1;
    info->n_hist = it + 1;
    if (ratio <= eta_nw) {
      info->converged = 1;
      break;
    }
  }
  // outputs at the final u
  TRY(flux_and_tangent(qbar, Abar));
  if (mean_flux_out)
    for (int r = 0; r < 3; ++r) mean_flux_out[r] = qbar[r];
  TRY(ensure_partial(ctx, (size_t)ctx->d.c * 2 * 152));
  CK(launch_sub_mean(u, 1, N, 1, N, ctx->partial, s));
  count_launch(ctx, 2);
  if (fluct_out)
    CK(cudaMemcpyAsync(fluct_out, u, N * sizeof(double), fluct_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       s));
  CK(cudaStreamSynchronize(s));
  return info->converged ? FEHOM_OK : FEHOM_E_NOT_CONVERGED;
}

fehom_status fehom_effective_energy(const fehom_ctx* ctx, double* c_eff) {
  if (!ctx || !c_eff) return FEHOM_E_INVALID;
  if (ctx->c_eff_energy.empty()) return FEHOM_E_STATE;
  std::memcpy(c_eff, ctx->c_eff_energy.data(), ctx->c_eff_energy.size() * sizeof(double));
  return FEHOM_OK;
}

fehom_status fehom_launch_count(const fehom_ctx* ctx, int64_t* count) {
  if (!ctx || !count) return FEHOM_E_INVALID;
  *count = ctx->launches;
  return FEHOM_OK;
}

fehom_status fehom_query(const fehom_ctx* ctx, int* c, int* m, int64_t* N, int64_t* nxh) {
  if (!ctx) return FEHOM_E_INVALID;
  if (c) *c = ctx->d.c;
  if (m) *m = ctx->m;
  if (N) *N = ctx->d.N;
  if (nxh) *nxh = ctx->d.nxh;
  return FEHOM_OK;
}

void fehom_destroy(fehom_ctx* ctx) {
  if (!ctx) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->events_made)
    for (int i = 0; i < kChunk; ++i)
      for (int k = 0; k < FEHOM_K_COUNT; ++k)
        for (int j = 0; j < 2; ++j) cudaEventDestroy(ctx->ev[i][k][j]);
  dfree(ctx->ids); dfree(ctx->mats64); dfree(ctx->mats32); dfree(ctx->iso64); dfree(ctx->iso32); dfree(ctx->isodf);
  dfree(ctx->rmats64); dfree(ctx->riso64); dfree(ctx->tune_st);
  for (int i = 0; i < 3; ++i) { dfree(ctx->tw64[i]); dfree(ctx->tw32[i]); }
  dfree(ctx->sym64); dfree(ctx->sym32);
  dfree(ctx->x64); dfree(ctx->r64); dfree(ctx->p64); dfree(ctx->ap64); dfree(ctx->b64); dfree(ctx->spec64);
  dfree(ctx->x32); dfree(ctx->r32); dfree(ctx->p32); dfree(ctx->ap32); dfree(ctx->spec32);
  dfree(ctx->st); dfree(ctx->red.partial); dfree(ctx->red.count); dfree(ctx->red.hist);
  dfree(ctx->tau); dfree(ctx->taudf); dfree(ctx->partial);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  cudaSetDevice(prev);
  delete ctx;
}

static fehom_status setup_impl(fehom_ctx* ctx, int elem, int physics, const int64_t n[3], const double* cell,
                               const uint8_t* phase_ids, int ids_on_device, int n_phases, const double* phase_moduli,
                               const double* ref_material, const fehom_options* opt) {
  if (opt) ctx->opt = *opt;
  else fehom_default_options(&ctx->opt);
  if (ctx->opt.max_iter <= 0) ctx->opt.max_iter = 10000;
  if (!(ctx->opt.inner_tol > 0.0 && ctx->opt.inner_tol < 1.0)) ctx->opt.inner_tol = 1e-3;
  if (elem != FEHOM_P1TRI2_2D && elem != FEHOM_HEX8_3D && elem != FEHOM_Q1_2D && elem != FEHOM_P1TRI4_2D)
    FAIL(FEHOM_E_INVALID, "unknown element type");
  if (elem == FEHOM_P1TRI4_2D && physics != FEHOM_SCALAR)
    FAIL(FEHOM_E_INVALID, "the two-node stencil FEHOM_P1TRI4_2D is built for FEHOM_SCALAR only");
  if (physics != FEHOM_SCALAR && physics != FEHOM_ELASTIC) FAIL(FEHOM_E_INVALID, "unknown physics");
  if (!n || !phase_ids || !phase_moduli) FAIL(FEHOM_E_INVALID, "NULL argument");
  if (n_phases < 1 || n_phases > kMaxPhases) FAIL(FEHOM_E_INVALID, "n_phases must be in 1..256");
  const int dim = (elem == FEHOM_HEX8_3D) ? 3 : 2;
  if (dim == 2 && n[2] != 1) FAIL(FEHOM_E_UNSUPPORTED_SIZE, "2-D elements need n[2] == 1");
  for (int i = 0; i < dim; ++i)
    if (!size_ok(n[i])) FAIL(FEHOM_E_UNSUPPORTED_SIZE, "each grid size must be 2^k or 3*2^k in [2, 1024]");
  if (n[0] % 2) FAIL(FEHOM_E_UNSUPPORTED_SIZE, "n_x must be even");
  ctx->d.dim = dim;
  ctx->d.nx = (int)n[0];
  ctx->d.ny = (int)n[1];
  ctx->d.nz = dim == 3 ? (int)n[2] : 1;
  ctx->d.nxh = ctx->d.nx / 2 + 1;
  ctx->d.N = (long long)ctx->d.nx * ctx->d.ny * ctx->d.nz;
  ctx->d.Nh = (long long)ctx->d.nxh * ctx->d.ny * ctx->d.nz;
  ctx->d.c = physics == FEHOM_SCALAR ? 1 : dim;
  if (elem == FEHOM_P1TRI4_2D) ctx->d.c = 2;  // field blocks = node types (corner, centre)
  ctx->d.elem = elem;
  ctx->physics = physics;
  ctx->m = physics == FEHOM_SCALAR ? dim : dim * (dim + 1) / 2;
  ctx->D = (physics == FEHOM_SCALAR ? 1 : dim) * dim;
  ctx->vol = 1.0;
  for (int i = 0; i < 3; ++i) {
    const double l = (cell && i < dim) ? cell[i] : 1.0;
    if (!(l > 0.0) || !std::isfinite(l)) FAIL(FEHOM_E_INVALID, "cell lengths must be positive");
    ctx->h[i] = i < dim ? l / (double)n[i] : 1.0;
    if (i < dim) ctx->vol *= ctx->h[i];
  }
  const int m = ctx->m;
  ctx->n_phases = n_phases;
  ctx->moduli.assign(phase_moduli, phase_moduli + (size_t)n_phases * m * m);
  for (int p = 0; p < n_phases; ++p)
    if (!spd(&ctx->moduli[(size_t)p * m * m], m)) FAIL(FEHOM_E_INVALID, "phase moduli must be finite, symmetric, positive definite");

  CK(cudaGetDevice(&ctx->device));
  if (ctx->opt.stream) {
    ctx->stream = (cudaStream_t)ctx->opt.stream;
  } else {
    CK(cudaStreamCreate(&ctx->stream));  // blocking stream: ordered with the legacy default stream
    ctx->own_stream = true;
  }
  cudaStream_t s = ctx->stream;
  const long long N = ctx->d.N;
  CK(cudaMalloc(&ctx->ids, N));
  CK(cudaMemcpyAsync(ctx->ids, phase_ids, N, ids_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  // phase histogram: id range check and volume fractions
  unsigned long long* hist;
  CK(cudaMalloc(&hist, 256 * sizeof(unsigned long long)));
  CK(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), s));
  CK(launch_phase_histogram(ctx->ids, N, hist, s));
  count_launch(ctx);
  std::vector<unsigned long long> hh(256);
  CK(cudaMemcpyAsync(hh.data(), hist, 256 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  cudaFree(hist);
  for (int p = n_phases; p < 256; ++p)
    if (hh[p]) FAIL(FEHOM_E_INVALID, "phase id >= n_phases in phase_ids");
  ctx->frac.assign(n_phases, 0.0);
  for (int p = 0; p < n_phases; ++p) ctx->frac[p] = (double)hh[p] / (double)N;
  // reference material: given, or the volume mean (Sec. 6.2)
  ctx->cref.assign((size_t)m * m, 0.0);
  if (ref_material) {
    ctx->cref.assign(ref_material, ref_material + (size_t)m * m);
  } else {
    for (int p = 0; p < n_phases; ++p)
      for (int i = 0; i < m * m; ++i) ctx->cref[i] += ctx->frac[p] * ctx->moduli[(size_t)p * m * m + i];
  }
  if (!spd(ctx->cref.data(), m)) FAIL(FEHOM_E_INVALID, "reference material must be symmetric positive definite");
  // gradient-space materials
  const int D = ctx->D;
  std::vector<double> mats((size_t)n_phases * D * D);
  for (int p = 0; p < n_phases; ++p) grad_material(ctx, &ctx->moduli[(size_t)p * m * m], &mats[(size_t)p * D * D]);
  std::vector<float> mats32(mats.begin(), mats.end());
  CK(cudaMalloc(&ctx->mats64, mats.size() * sizeof(double)));
  CK(cudaMalloc(&ctx->mats32, mats.size() * sizeof(float)));
  CK(cudaMemcpyAsync(ctx->mats64, mats.data(), mats.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ctx->mats32, mats32.data(), mats32.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  std::vector<double> rm((size_t)D * D);
  grad_material(ctx, ctx->cref.data(), rm.data());
  CK(cudaMalloc(&ctx->rmats64, rm.size() * sizeof(double)));
  CK(cudaMemcpyAsync(ctx->rmats64, rm.data(), rm.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  // isotropic fast path (hex8 elasticity or conductivity on a cubic grid)
  if (elem == FEHOM_HEX8_3D && ctx->h[0] == ctx->h[1] && ctx->h[1] == ctx->h[2]) {
    bool all = true;
    std::vector<double> iso((size_t)kIsoStride * n_phases);
    for (int p = 0; p < n_phases && all; ++p)
      all = iso_material(ctx, &ctx->moduli[(size_t)p * m * m], &iso[(size_t)kIsoStride * p]);
    if (all) {
      ctx->iso = true;
      std::vector<float> iso32(iso.begin(), iso.end());
      CK(cudaMalloc(&ctx->iso64, iso.size() * sizeof(double)));
      CK(cudaMalloc(&ctx->iso32, iso.size() * sizeof(float)));
      CK(cudaMemcpyAsync(ctx->iso64, iso.data(), iso.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(ctx->iso32, iso32.data(), iso32.size() * sizeof(float), cudaMemcpyHostToDevice, s));
      if (physics == FEHOM_ELASTIC) {
        // double-float copy of the six constants, hi = fl(v), lo = fl(v - hi) (refinement residuals)
        std::vector<float> isodf((size_t)16 * n_phases, 0.0f);
        for (int p = 0; p < n_phases; ++p)
          for (int i = 0; i < 6; ++i) {
            const double v = iso[(size_t)kIsoStride * p + i];
            const float hi = (float)v;
            isodf[(size_t)16 * p + 2 * i] = hi;
            isodf[(size_t)16 * p + 2 * i + 1] = (float)(v - (double)hi);
          }
        CK(cudaMalloc(&ctx->isodf, isodf.size() * sizeof(float)));
        CK(cudaMemcpyAsync(ctx->isodf, isodf.data(), isodf.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));  // isodf is a local
      }
      CK(cudaStreamSynchronize(s));  // iso and iso32 are locals
    }
    double ri[kIsoStride];
    if (iso_material(ctx, ctx->cref.data(), ri)) {
      ctx->iso_ref = true;
      CK(cudaMalloc(&ctx->riso64, kIsoStride * sizeof(double)));
      CK(cudaMemcpyAsync(ctx->riso64, ri, kIsoStride * sizeof(double), cudaMemcpyHostToDevice, s));
    }
  }
  // twiddles
  const int lens[3] = {ctx->d.nx, ctx->d.ny, ctx->d.nz};
  for (int i = 0; i < dim; ++i) CK(make_twiddles(lens[i], &ctx->tw64[i], &ctx->tw32[i]));
  // PCG state and reduction scratch
  CK(cudaMalloc(&ctx->st, sizeof(PcgState) * kMaxLoads));
  ctx->red.max_blocks = kRedBlocks;
  CK(cudaMalloc(&ctx->red.partial, sizeof(double) * (size_t)kMaxLoads * kRedBlocks));
  CK(cudaMalloc(&ctx->red.count, sizeof(unsigned) * kMaxLoads));
  CK(cudaMalloc(&ctx->red.hist, sizeof(double) * (size_t)kMaxLoads * 2 * kHist));
  CK(cudaMemsetAsync(ctx->red.count, 0, sizeof(unsigned) * kMaxLoads, s));
  TRY(grow64(ctx, 1));
  CK(cudaStreamSynchronize(s));
  return FEHOM_OK;
}

fehom_status fehom_setup(fehom_ctx** out, int elem, int physics, const int64_t n[3], const double* cell,
                         const uint8_t* phase_ids, int ids_on_device, int n_phases, const double* phase_moduli,
                         const double* ref_material, const fehom_options* opt) {
  if (!out) return FEHOM_E_INVALID;
  *out = nullptr;
  fehom_ctx* ctx = new (std::nothrow) fehom_ctx();
  if (!ctx) return FEHOM_E_OOM;
  const fehom_status st = setup_impl(ctx, elem, physics, n, cell, phase_ids, ids_on_device, n_phases, phase_moduli,
                                     ref_material, opt);
  if (st != FEHOM_OK) {
    g_setup_error = ctx->err;  // readable through fehom_last_error(NULL)
    fehom_destroy(ctx);
    return st;
  }
  g_setup_error.clear();
  *out = ctx;
  return FEHOM_OK;
}

fehom_status fehom_precond_build(fehom_ctx* ctx) {
  if (!ctx) return FEHOM_E_INVALID;
  const int c = ctx->d.c;
  cudaStream_t s = ctx->stream;
  TRY(grow64(ctx, c));
  const long long cN = (long long)c * ctx->d.N;
  // Algorithm 2: the columns K_ref i^beta for the unit impulses i^beta at node 0 of component beta
  // (one "load" per beta).  K_ref i^beta is nonzero only on the 3^d nodes around node 0, so when
  // every axis has at least 4 nodes it is computed on a periodic 4^d proxy grid of the same spacing
  // (same element tables) and placed into the full grid; otherwise on the full grid itself.
  const bool proxy = ctx->d.nx >= 4 && ctx->d.ny >= 4 && (ctx->d.dim == 2 || ctx->d.nz >= 4);
  StencilArgs a{};
  a.ids = nullptr;  // uniform reference material
  a.mats = ctx->rmats64;
  a.iso = (ctx->iso_ref && ctx->iso) ? ctx->riso64 : nullptr;
  a.n_phases = 1;
  a.n_loads = c;
  a.y_scale = 1.0;
  a.red = ctx->red;
  const double one = 1.0;
  if (proxy) {
    Dims pd = ctx->d;
    pd.nx = pd.ny = 4;
    pd.nz = ctx->d.dim == 3 ? 4 : 1;
    pd.nxh = 3;
    pd.N = (long long)pd.nx * pd.ny * pd.nz;
    pd.Nh = (long long)pd.nxh * pd.ny * pd.nz;
    const long long pcN = (long long)c * pd.N;
    TRY(ensure_partial(ctx, (size_t)std::max<long long>(2 * c * pcN, 4 * 2 * 152)));
    double* px = ctx->partial;
    double* py = ctx->partial + c * pcN;
    CK(cudaMemsetAsync(px, 0, sizeof(double) * c * pcN, s));
    for (int be = 0; be < c; ++be)
      CK(cudaMemcpyAsync(px + be * pcN + (long long)be * pd.N, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    a.d = pd;
    a.x = px;
    a.y = py;
    a.load_stride = pcN;
    CK(launch_stiffness<double>(a, s));
    count_launch(ctx);
    CK(cudaMemsetAsync(ctx->ap64, 0, sizeof(double) * cN * c, s));
    CK(launch_impulse_scatter(py, pd, ctx->d, c, ctx->ap64, s));
    count_launch(ctx);
  } else {
    CK(cudaMemsetAsync(ctx->x64, 0, sizeof(double) * cN * c, s));
    for (int be = 0; be < c; ++be)
      CK(cudaMemcpyAsync(ctx->x64 + be * cN + (long long)be * ctx->d.N, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    a.d = ctx->d;
    a.x = ctx->x64;
    a.y = ctx->ap64;
    a.load_stride = cN;
    CK(launch_stiffness<double>(a, s));
    count_launch(ctx);
  }
  // forward FFT of every component of every column -> spec64[beta][alpha][Nh]
  FftArgs f;
  fill_dims_args(ctx, f, false, c);
  f.sym = nullptr;
  f.mode = FX_PLAIN;
  f.f0 = ctx->ap64;
  CK(launch_fft_x_fwd<double>(f, s));
  count_launch(ctx);
  if (ctx->d.dim == 3) {
    CK(launch_fft_y<double>(f, 0, s));
    count_launch(ctx);
  }
  CK(launch_fft_last_solve<double>(f, s));
  count_launch(ctx);
  // per-wavevector inverse
  const long long Nh = ctx->d.Nh;
  const bool herm = ctx->d.elem == P1TRI4_2D;
  const int ne = herm ? 4 : c * (c + 1) / 2;
  if (!ctx->sym64) {
    CK(cudaMalloc(&ctx->sym64, sizeof(double) * ne * Nh));
    CK(cudaMalloc(&ctx->sym32, sizeof(float) * ne * Nh));
  }
  TRY(ensure_partial(ctx, 4 * 2 * 152));
  SymbolArgs sa{};
  sa.d = ctx->d;
  sa.spec = ctx->spec64;
  sa.sym64 = ctx->sym64;
  sa.sym32 = ctx->sym32;
  sa.partial = ctx->partial;
  sa.zero_tol = 1e-12;
  sa.herm = herm ? 1 : 0;
  int blocks = 0;
  CK(launch_symbol_build(sa, &blocks, s));
  count_launch(ctx);
  std::vector<double> hp(4 * blocks);
  CK(cudaMemcpyAsync(hp.data(), ctx->partial, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  // the k = 0 block
  std::vector<double2> k0(c * c);
  for (int be = 0; be < c; ++be)
    for (int al = 0; al < c; ++al)
      CK(cudaMemcpyAsync(&k0[be * c + al], ctx->spec64 + ((long long)be * c + al) * Nh, sizeof(double2),
                         cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double mx_im = 0, mx_asym = 0, mx_abs = 0, mn_piv = 1e300;
  for (int b = 0; b < blocks; ++b) {
    mx_im = std::max(mx_im, hp[4 * b]);
    mx_asym = std::max(mx_asym, hp[4 * b + 1]);
    mx_abs = std::max(mx_abs, hp[4 * b + 2]);
    mn_piv = std::min(mn_piv, hp[4 * b + 3]);
  }
  char msg[256];
  if (!(mx_abs > 0) || mx_im > 1e-9 * mx_abs || mx_asym > 1e-9 * mx_abs) {
    std::snprintf(msg, sizeof msg, "reference symbol not real symmetric (Hermitian for the two-node stencil): "
                  "max|Im| %.3e, asym %.3e, max %.3e", mx_im,
                  mx_asym, mx_abs);
    FAIL(FEHOM_E_INVALID, msg);
  }
  if (ctx->d.Nh > 1 && !(mn_piv > 1e-13 * mx_abs)) {
    std::snprintf(msg, sizeof msg, "reference symbol singular away from k = 0 (min pivot %.3e)", mn_piv);
    FAIL(FEHOM_E_INVALID, msg);
  }
  // Moore-Penrose pseudo-inverse of the k = 0 block, singular values cut relative to max |K_hat|
  std::vector<double> A(c * c), V, ev;
  for (int al = 0; al < c; ++al)
    for (int be = 0; be < c; ++be) A[al * c + be] = 0.5 * (k0[be * c + al].x + k0[al * c + be].x);
  jacobi_eig(c, A, V, ev);
  std::vector<double> pinv(c * c, 0.0);
  for (int k = 0; k < c; ++k) {
    if (std::fabs(ev[k]) <= 1e-12 * mx_abs) continue;
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) pinv[i * c + j] += V[i * c + k] * V[j * c + k] / ev[k];
  }
  const int pi3[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
  const int pi2[3][2] = {{0, 0}, {1, 1}, {0, 1}};
  const double invN = 1.0 / (double)ctx->d.N;
  for (int e = 0; e < ne; ++e) {
    const int i = c == 3 ? pi3[e][0] : (c == 2 ? pi2[std::min(e, 2)][0] : 0);
    const int j = c == 3 ? pi3[e][1] : (c == 2 ? pi2[std::min(e, 2)][1] : 0);
    const double v = (herm && e == 3) ? 0.0 : pinv[i * c + j] * invN;  // Im of the k = 0 block: 0
    const float vf = (float)v;
    CK(cudaMemcpyAsync(ctx->sym64 + (long long)e * Nh, &v, sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->sym32 + (long long)e * Nh, &vf, sizeof(float), cudaMemcpyHostToDevice, s));
  }
  CK(cudaStreamSynchronize(s));
  ctx->built = true;
  return FEHOM_OK;
}

fehom_status fehom_apply_stiffness(fehom_ctx* ctx, const void* x, void* y, int precision) {
  if (!ctx || !x || !y) return FEHOM_E_INVALID;
  StencilArgs a = stencil_args(ctx, precision == FEHOM_MIXED, 1);
  a.x = x;
  a.y = y;
  if (precision == FEHOM_MIXED) CK(launch_stiffness<float>(a, ctx->stream));
  else CK(launch_stiffness<double>(a, ctx->stream));
  count_launch(ctx);
  CK(cudaStreamSynchronize(ctx->stream));
  return FEHOM_OK;
}

fehom_status fehom_rhs(fehom_ctx* ctx, const double* e, double* b) {
  if (!ctx || !e || !b) return FEHOM_E_INVALID;
  TRY(upload_tau(ctx, 1, e));
  return residual_stats(ctx, 1, nullptr, b, nullptr, nullptr);
}

fehom_status fehom_residual_update(fehom_ctx* ctx, const float* d, const double* r_in, double* r_out,
                                   double* sums_out) {
  if (!ctx || !d || !r_in || !r_out) return FEHOM_E_INVALID;
  if (!residual_df_supported(ctx))
    FAIL(FEHOM_E_UNSUPPORTED_SIZE, "fehom_residual_update: hex8 elasticity with isotropic phases on cubic voxels only");
  std::vector<double> y2, dT, fl;
  TRY(residual_update_df(ctx, 1, d, r_in, r_out, &y2, &dT));
  if (sums_out) {
    sums_to_flux(ctx, 1, dT, &fl);
    sums_out[0] = y2[0];
    for (int i = 0; i < ctx->m; ++i) sums_out[1 + i] = fl[i];
  }
  return FEHOM_OK;
}

fehom_status fehom_rhs_df(fehom_ctx* ctx, const double* e, double* b) {
  if (!ctx || !e || !b) return FEHOM_E_INVALID;
  if (!residual_df_supported(ctx))
    FAIL(FEHOM_E_UNSUPPORTED_SIZE, "fehom_rhs_df: hex8 elasticity with isotropic phases on cubic voxels only");
  for (int i = 0; i < ctx->m; ++i)
    if (!std::isfinite(e[i])) FAIL(FEHOM_E_INVALID, "non-finite load");
  TRY(upload_tau(ctx, 1, e));
  std::vector<double> y2, T;
  return rhs_df(ctx, 1, b, &y2, &T);
}

fehom_status fehom_apply_precond(fehom_ctx* ctx, const void* r, void* z, int precision) {
  if (!ctx || !r || !z) return FEHOM_E_INVALID;
  if (!ctx->built) FAIL(FEHOM_E_STATE, "fehom_apply_precond before fehom_precond_build");
  const bool fp32 = precision == FEHOM_MIXED;
  if (fp32) TRY(grow32(ctx, 1));
  FftArgs f;
  fill_dims_args(ctx, f, fp32, 1);
  if (fp32) CK(precond_passes<float>(ctx, f, FX_PLAIN, FX_PLAIN, const_cast<void*>(r), nullptr, z, nullptr, ctx->stream));
  else CK(precond_passes<double>(ctx, f, FX_PLAIN, FX_PLAIN, const_cast<void*>(r), nullptr, z, nullptr, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FEHOM_OK;
}

// Running PCG states of the operator-level PCG entry points (the stencil tuner's array, never the
// solve's): state RUN, the given <r, z> and alpha, no stopping test (tol^2 = 0), no iteration cap.
static fehom_status op_states(fehom_ctx* ctx, int n_loads, const double* rz, const double* alpha) {
  if (!ctx->tune_st) CK(cudaMalloc(&ctx->tune_st, sizeof(PcgState) * kMaxLoads));
  std::vector<PcgState> hs(n_loads);
  for (int l = 0; l < n_loads; ++l) {
    std::memset(&hs[l], 0, sizeof(PcgState));
    hs[l].state = ST_RUN;
    hs[l].rz = rz ? rz[l] : 0.0;
    hs[l].alpha = alpha ? alpha[l] : 0.0;
    hs[l].bnorm2 = 1.0;
    hs[l].max_iter = 1 << 30;
  }
  CK(cudaMemcpyAsync(ctx->tune_st, hs.data(), sizeof(PcgState) * n_loads, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FEHOM_OK;
}

static fehom_status op_read_states(fehom_ctx* ctx, int n_loads, std::vector<PcgState>* hs) {
  hs->resize(n_loads);
  CK(cudaMemcpyAsync(hs->data(), ctx->tune_st, sizeof(PcgState) * n_loads, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FEHOM_OK;
}

fehom_status fehom_pcg_apply_stiffness(fehom_ctx* ctx, int precision, int n_loads, const void* p, void* ap,
                                       const double* rz, int rows, int staging, double* pAp, double* alpha) {
  if (!ctx || !p || !ap || !rz) return FEHOM_E_INVALID;
  if (n_loads < 1 || n_loads > kMaxLoads) FAIL(FEHOM_E_INVALID, "fehom_pcg_apply_stiffness: n_loads out of range");
  if (rows != 0 && rows != 8 && rows != 16) FAIL(FEHOM_E_INVALID, "fehom_pcg_apply_stiffness: rows must be 0, 8 or 16");
  if (staging < 0 || staging > 3) FAIL(FEHOM_E_INVALID, "fehom_pcg_apply_stiffness: staging must be 0..3");
  if (precision != FEHOM_FP64 && precision != FEHOM_MIXED) FAIL(FEHOM_E_INVALID, "bad precision");
  for (int l = 0; l < n_loads; ++l)
    if (!std::isfinite(rz[l])) FAIL(FEHOM_E_INVALID, "fehom_pcg_apply_stiffness: non-finite <r, z>");
  const bool fp32 = precision == FEHOM_MIXED;
  TRY(op_states(ctx, n_loads, rz, nullptr));
  StencilArgs a = stencil_args(ctx, fp32, n_loads);
  a.x = p;
  a.y = ap;
  a.st = ctx->tune_st;
  a.red.hist = nullptr;
  if (rows) a.tile_rows = rows;
  if (staging != 0) a.staging = staging;  // 0: the context's plan
  const cudaError_t le = fp32 ? launch_stiffness<float>(a, ctx->stream) : launch_stiffness<double>(a, ctx->stream);
  if (le == cudaErrorInvalidValue && staging != 0)
    FAIL(FEHOM_E_UNSUPPORTED_SIZE, "fehom_pcg_apply_stiffness: this staging / tile height is not available here");
  CK(le);
  count_launch(ctx);
  std::vector<PcgState> hs;
  TRY(op_read_states(ctx, n_loads, &hs));
  bool broke = false;
  for (int l = 0; l < n_loads; ++l) {
    if (pAp) pAp[l] = hs[l].pAp;
    if (alpha) alpha[l] = hs[l].alpha;
    broke = broke || hs[l].state == ST_BREAK;
    if (hs[l].err) FAIL(FEHOM_E_CUDA, "fehom_pcg_apply_stiffness: a bounded wait of the kernel gave up");
  }
  if (broke) FAIL(FEHOM_E_BREAKDOWN, "fehom_pcg_apply_stiffness: <p, K p> not positive and finite for a load");
  return FEHOM_OK;
}

fehom_status fehom_pcg_precond_step(fehom_ctx* ctx, int precision, int n_loads, void* r, const void* ap, void* x,
                                    void* p, const double* alpha, const double* rz, double* rz_new, double* beta) {
  if (!ctx || !r || !p) return FEHOM_E_INVALID;
  if (!ctx->built) FAIL(FEHOM_E_STATE, "fehom_pcg_precond_step before fehom_precond_build");
  if (n_loads < 1 || n_loads > kMaxLoads) FAIL(FEHOM_E_INVALID, "fehom_pcg_precond_step: n_loads out of range");
  if (precision != FEHOM_FP64 && precision != FEHOM_MIXED) FAIL(FEHOM_E_INVALID, "bad precision");
  const bool init = alpha == nullptr;
  if (!init && (!ap || !x || !rz)) FAIL(FEHOM_E_INVALID, "fehom_pcg_precond_step: ap, x and rz are needed with alpha");
  if (!init)
    for (int l = 0; l < n_loads; ++l)
      if (!std::isfinite(alpha[l]) || !std::isfinite(rz[l]))
        FAIL(FEHOM_E_INVALID, "fehom_pcg_precond_step: non-finite alpha or <r, z>");
  const bool fp32 = precision == FEHOM_MIXED;
  if (fp32) TRY(grow32(ctx, n_loads));
  else TRY(grow64(ctx, n_loads));
  TRY(op_states(ctx, n_loads, rz, alpha));
  FftArgs f;
  fill_dims_args(ctx, f, fp32, n_loads);
  f.st = ctx->tune_st;
  f.red.hist = nullptr;
  f.init = init ? 1 : 0;
  const int fm = init ? FX_PLAIN : FX_PCG, im = init ? FX_PCG_INIT : FX_PCG;
  void* xi = init ? nullptr : x;
  if (fp32) CK(precond_passes<float>(ctx, f, fm, im, r, ap, xi, p, ctx->stream));
  else CK(precond_passes<double>(ctx, f, fm, im, r, ap, xi, p, ctx->stream));
  std::vector<PcgState> hs;
  TRY(op_read_states(ctx, n_loads, &hs));
  bool bad = false;
  for (int l = 0; l < n_loads; ++l) {
    if (rz_new) rz_new[l] = hs[l].rz;
    if (beta) beta[l] = init ? 0.0 : hs[l].beta;
    bad = bad || hs[l].state == ST_BREAK;
  }
  if (bad) FAIL(FEHOM_E_BREAKDOWN, "fehom_pcg_precond_step: non-finite <r, z> for a load");
  return FEHOM_OK;
}

fehom_status fehom_get_symbol_inverse(fehom_ctx* ctx, double* out) {
  if (!ctx || !out) return FEHOM_E_INVALID;
  if (!ctx->built) FAIL(FEHOM_E_STATE, "fehom_get_symbol_inverse before fehom_precond_build");
  const int ne = ctx->d.elem == P1TRI4_2D ? 4 : ctx->d.c * (ctx->d.c + 1) / 2;
  CK(cudaMemcpyAsync(out, ctx->sym64, sizeof(double) * ne * ctx->d.Nh, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FEHOM_OK;
}

fehom_status fehom_mean_flux_noalloc(fehom_ctx* ctx, const double* e, const double* u, double* out) {
  if (!ctx || !e || !u || !out) return FEHOM_E_INVALID;
  for (int i = 0; i < ctx->m; ++i)
    if (!std::isfinite(e[i])) FAIL(FEHOM_E_INVALID, "non-finite load");
  const int D = ctx->D, W = 1 + D, P = ctx->n_phases;
  const int ctas = stiffness_ctas(ctx->d, 1);
  const long long need = (long long)ctas * W + W + (long long)P * D;
  if (need > kNoallocDoubles) {
    char msg[200];
    std::snprintf(msg, sizeof msg,
                  "fehom_mean_flux_noalloc: this grid needs %lld scratch doubles, the fixed array holds %d", need,
                  kNoallocDoubles);
    FAIL(FEHOM_E_UNSUPPORTED_SIZE, msg);
  }
  cudaStream_t s = ctx->stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    FAIL(FEHOM_E_STATE, "fehom_mean_flux_noalloc: the context's stream is being captured (the call copies "
                        "between host and device and waits for the stream)");
  double* scratch = nullptr;
  TRY(noalloc_scratch(ctx, &scratch));
  const int dim = ctx->d.dim, m = ctx->m;
  double Pm[6 * 9];
  flux_map_into(dim, ctx->physics, Pm);
  double w, sc[3];
  kernel_scales(ctx, &w, sc);
  double tau[kMaxPhases * 9];  // host stack: per-phase prestress w S P^T C e of the load, [P][D]
  for (int ph = 0; ph < P; ++ph) {
    const double* C = &ctx->moduli[(size_t)ph * m * m];
    for (int q = 0; q < D; ++q) {
      double acc = 0.0;
      for (int I = 0; I < m; ++I)
        for (int J = 0; J < m; ++J) acc += Pm[I * D + q] * C[I * m + J] * e[J];
      tau[ph * D + q] = w * sc[q % dim] * acc;
    }
  }
  double* tau_d = scratch + (long long)ctas * W + W;
  CK(cudaMemcpyAsync(tau_d, tau, sizeof(double) * P * D, cudaMemcpyHostToDevice, s));
  StencilArgs a = stencil_args(ctx, false, 1);
  a.x = u;
  a.y = nullptr;  // sums only: no field is written
  a.tau = tau_d;
  a.y_scale = -1.0;
  a.stats = scratch;
  int got = 0;
  CK(launch_stiffness<double>(a, s, &got));
  count_launch(ctx);
  if (got != ctas) FAIL(FEHOM_E_CUDA, "stiffness statistics: CTA count mismatch");
  noalloc_sum_kernel<<<1, 32, 0, s>>>(scratch, ctas, W);
  CK(cudaGetLastError());
  count_launch(ctx);
  double sums[1 + 9];
  CK(cudaMemcpyAsync(sums, scratch + (long long)ctas * W, sizeof(double) * W, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double cell = 1.0;
  const int n3[3] = {ctx->d.nx, ctx->d.ny, ctx->d.nz};
  for (int i = 0; i < dim; ++i) cell *= ctx->h[i] * n3[i];
  for (int I = 0; I < ctx->m; ++I) {
    double v = 0.0;
    for (int q = 0; q < D; ++q) v += Pm[I * D + q] * sums[1 + q] / sc[q % dim];
    out[I] = v / cell;
  }
  return FEHOM_OK;
}

fehom_status fehom_mean_flux(fehom_ctx* ctx, const double* e, const double* u, double* out) {
  if (!ctx || !e || !u || !out) return FEHOM_E_INVALID;
  TRY(upload_tau(ctx, 1, e));
  std::vector<double> flux;
  TRY(residual_stats(ctx, 1, u, ctx->ap64, nullptr, &flux));
  std::memcpy(out, flux.data(), sizeof(double) * ctx->m);
  return FEHOM_OK;
}

// fields (mean removed), <sigma> and C_eff of a finished solve; flux: the mean fluxes of the final x
// C = E^-1 B for the m x m row-major E (rows = loads) by Gaussian elimination with partial pivoting;
// false when E is singular.
static bool solve_loads(int m, std::vector<double> E, std::vector<double>& B) {
  for (int col = 0; col < m; ++col) {
    int piv = col;
    for (int r = col + 1; r < m; ++r)
      if (std::fabs(E[r * m + col]) > std::fabs(E[piv * m + col])) piv = r;
    if (std::fabs(E[piv * m + col]) < 1e-300) return false;
    for (int k = 0; k < m; ++k) {
      std::swap(E[col * m + k], E[piv * m + k]);
      std::swap(B[col * m + k], B[piv * m + k]);
    }
    for (int r = 0; r < m; ++r) {
      if (r == col) continue;
      const double f = E[r * m + col] / E[col * m + col];
      for (int k = 0; k < m; ++k) {
        E[r * m + k] -= f * E[col * m + k];
        B[r * m + k] -= f * B[col * m + k];
      }
    }
  }
  for (int r = 0; r < m; ++r)
    for (int k = 0; k < m; ++k) B[r * m + k] /= E[r * m + r];
  return true;
}

// Energy form of C_eff (m loads e_l, fields x_l, right-hand sides b_l, true residuals r_l): for any x,
//   sum_q w_q (e_i + D x_i)^T C (e_j + D x_j) = |Y| e_i^T <C> e_j - x_j . b_i - x_i . r_j,
// (b = -D^T W C e, r = b - K x), stationary at the solution, so its error is second order in the
// solve error.  Since x_j . b_i = -sum_q w_q (D x_j)^T C e_i = -|Y| e_i^T (<sigma>_j - <C> e_j), with
// <sigma>_j the volume average of the same quadrature, the form equals |Y| e_i^T <sigma>_j - x_i . r_j:
// the stress average plus a correction from the residual, so only the dots x_i . r_j are formed.
// A = E C_eff E^T  ->  C_eff = E^-1 A E^-T.
static fehom_status energy_c_eff(fehom_ctx* ctx, int m, const double* loads, const double* res,
                                 const std::vector<double>& flux) {
  ctx->c_eff_energy.clear();
  if (!res || m > 6 || flux.size() < (size_t)m * ctx->m) return FEHOM_OK;
  cudaStream_t s = ctx->stream;
  const long long cN = (long long)ctx->d.c * ctx->d.N;
  TRY(ensure_partial(ctx, (size_t)m * m * 304 + m * m));
  double* out = ctx->partial + (size_t)m * m * 304;
  CK(launch_pair_dots(ctx->x64, res, m, cN, ctx->partial, out, s));
  count_launch(ctx, 2);
  std::vector<double> dots(m * m);
  CK(cudaMemcpyAsync(dots.data(), out, sizeof(double) * dots.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<double> A(m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double es = 0.0;  // e_i^T <sigma>_j
      for (int a = 0; a < m; ++a) es += loads[i * m + a] * flux[(size_t)j * m + a];
      // dots[i m + j] = x_i . r_j
      A[i * m + j] = es - dots[i * m + j] / (ctx->vol * (double)ctx->d.N);
    }
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) A[i * m + j] = A[j * m + i] = 0.5 * (A[i * m + j] + A[j * m + i]);
  std::vector<double> E(loads, loads + m * m);
  if (!solve_loads(m, E, A)) return FEHOM_OK;  // A <- E^-1 A
  std::vector<double> T(m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) T[i * m + j] = A[j * m + i];
  if (!solve_loads(m, E, T)) return FEHOM_OK;  // E^-1 (E^-1 A)^T = E^-1 A E^-T (A symmetric)
  ctx->c_eff_energy = T;
  return FEHOM_OK;
}

static fehom_status finish_outputs(fehom_ctx* ctx, int n_loads, const double* loads, double* fluct_out,
                                   int fluct_on_device, double* mean_flux_out, double* c_eff_out,
                                   const std::vector<double>& flux, const double* res) {
  cudaStream_t s = ctx->stream;
  const long long cN = (long long)ctx->d.c * ctx->d.N;
  ctx->c_eff_energy.clear();
  if (c_eff_out && n_loads == ctx->m) TRY(energy_c_eff(ctx, n_loads, loads, res, flux));
  TRY(ensure_partial(ctx, (size_t)n_loads * ctx->d.c * 2 * 152));
  CK(sub_mean_fields(ctx, ctx->x64, n_loads, s));
  count_launch(ctx, 2);
  if (mean_flux_out) std::memcpy(mean_flux_out, flux.data(), flux.size() * sizeof(double));
  if (c_eff_out && n_loads == ctx->m) {
    // C_eff = S E^-1 with S[:, l] = flux_l, E[:, l] = e_l  ->  solve E^T C_eff^T = S^T
    const int m = ctx->m;
    std::vector<double> Et(m * m), St(m * m);
    for (int l = 0; l < m; ++l)
      for (int i = 0; i < m; ++i) {
        Et[l * m + i] = loads[l * m + i];  // row l of E^T = e_l
        St[l * m + i] = flux[l * m + i];
      }
    // Gaussian elimination with partial pivoting on [Et | St]
    bool ok = true;
    for (int col = 0; col < m && ok; ++col) {
      int piv = col;
      for (int r = col + 1; r < m; ++r)
        if (std::fabs(Et[r * m + col]) > std::fabs(Et[piv * m + col])) piv = r;
      if (std::fabs(Et[piv * m + col]) < 1e-300) { ok = false; break; }
      for (int k = 0; k < m; ++k) {
        std::swap(Et[col * m + k], Et[piv * m + k]);
        std::swap(St[col * m + k], St[piv * m + k]);
      }
      for (int r = 0; r < m; ++r) {
        if (r == col) continue;
        const double f = Et[r * m + col] / Et[col * m + col];
        for (int k = 0; k < m; ++k) {
          Et[r * m + k] -= f * Et[col * m + k];
          St[r * m + k] -= f * St[col * m + k];
        }
      }
    }
    if (ok) {
      // row l of C_eff^T = St[l] / Et[l][l]  ->  C_eff[i][l] = St[l][i] / Et[l][l]
      for (int l = 0; l < m; ++l)
        for (int i = 0; i < m; ++i) c_eff_out[i * m + l] = St[l * m + i] / Et[l * m + l];
    }
  }
  if (fluct_out) {
    CK(cudaMemcpyAsync(fluct_out, ctx->x64, sizeof(double) * cN * n_loads,
                       fluct_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  return FEHOM_OK;
}

// Warm start x0 (already in x64, mean removed): x64[l] *= <b, x0> / <x0, K x0> per load, in FP64.
fehom_status scale_warm_start(fehom_ctx* ctx, int n_loads) {
  if (!ctx->opt.x0_scaling) return FEHOM_OK;
  cudaStream_t s = ctx->stream;
  const long long cN = (long long)ctx->d.c * ctx->d.N;
  StencilArgs a = stencil_args(ctx, false, n_loads);
  a.x = ctx->x64;
  a.y = ctx->ap64;
  CK(launch_stiffness<double>(a, s));
  TRY(ensure_partial(ctx, (size_t)n_loads * 2 * 304));
  CK(launch_galerkin_scale(ctx->x64, ctx->ap64, ctx->b64, n_loads, cN, ctx->partial, s));
  count_launch(ctx, 3);
  return FEHOM_OK;
}

// One solve of one context, split into phases so that the PCG iterations of several contexts can
// run from one captured graph (fehom_solve_batch) as well as alone (fehom_solve).
//   FP64:  begin (tuner, b, initial preconditioner apply) -> iterations -> end_step (true residual)
//   mixed: begin (tuner, b) -> { begin_step (FP64 residual, FP32 initial apply, per-load decision)
//                                -> iterations -> end_step (x += d) } until every load is done
struct SolveRun {
  fehom_ctx* ctx = nullptr;
  int n_loads = 0;
  const double* loads = nullptr;
  double tol = 0;
  const double* x0 = nullptr;
  bool mixed = false;
  std::vector<PcgState> hs;
  std::vector<int> outer_it, inner_it;
  std::vector<double> relM, flux, rel2, bn2, rn2, bnorm2;
  std::vector<double> tsum;  // mixed: dual sums of the current x (+ e), updated with each correction
  bool df = false;           // mixed: refinement residuals r -= K d in double-float arithmetic
  std::vector<bool> done;
  int total_inner = 0;
  int steps = 0;
  bool stats_current = false;
  bool finished = false;
  const double* last_res = nullptr;  // buffer holding b - K x of the current x (FP64)

  fehom_status begin() {
    cudaStream_t s = ctx->stream;
    const long long cN = (long long)ctx->d.c * ctx->d.N;
    TRY(grow64(ctx, n_loads));
    if (mixed) TRY(grow32(ctx, n_loads));
    if (mixed) TRY(autotune_fft<float>(ctx, n_loads));
    else TRY(autotune_fft<double>(ctx, n_loads));
    if (mixed) TRY(autotune_stencil<float>(ctx, n_loads));
    else TRY(autotune_stencil<double>(ctx, n_loads));
    TRY(upload_tau(ctx, n_loads, loads));
    df = mixed && ctx->opt.residual_df != 0 && residual_df_supported(ctx);
    if (df) TRY(rhs_df(ctx, n_loads, ctx->b64, &bn2, &tsum));  // b = -D^T W C e, double-float
    else TRY(residual_stats(ctx, n_loads, nullptr, ctx->b64, &bn2, nullptr, &tsum));  // FP64
    outer_it.assign(n_loads, 0);
    inner_it.assign(n_loads, 0);
    relM.assign(n_loads, 1.0);
    hs.assign(n_loads, PcgState{});
    if (mixed) {
      if (x0) {
        CK(cudaMemcpyAsync(ctx->x64, x0, sizeof(double) * cN * n_loads, cudaMemcpyDeviceToDevice, s));
        TRY(ensure_partial(ctx, (size_t)n_loads * ctx->d.c * 2 * 152));
        CK(sub_mean_fields(ctx, ctx->x64, n_loads, s));
        count_launch(ctx, 2);
        TRY(scale_warm_start(ctx, n_loads));
      } else {
        CK(cudaMemsetAsync(ctx->x64, 0, sizeof(double) * cN * n_loads, s));
      }
      bnorm2.assign(n_loads, -1.0);
      done.assign(n_loads, false);
      return FEHOM_OK;
    }
    if (x0) {
      // <b, K_ref^+ b> first (normalisation of the stopping test), then r0 = b - K x0
      TRY(set_states(ctx, n_loads, tol, ctx->opt.max_iter, -1.0));
      CK(cudaMemcpyAsync(ctx->r64, ctx->b64, sizeof(double) * cN * n_loads, cudaMemcpyDeviceToDevice, s));
      TRY(pcg_init<double>(ctx, n_loads, ctx->r64, ctx->p64));
      std::vector<PcgState> h0(n_loads);
      CK(cudaMemcpyAsync(h0.data(), ctx->st, sizeof(PcgState) * n_loads, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      CK(cudaMemcpyAsync(ctx->x64, x0, sizeof(double) * cN * n_loads, cudaMemcpyDeviceToDevice, s));
      TRY(ensure_partial(ctx, (size_t)n_loads * ctx->d.c * 2 * 152));
      CK(sub_mean_fields(ctx, ctx->x64, n_loads, s));
      count_launch(ctx, 2);
      TRY(scale_warm_start(ctx, n_loads));
      TRY(residual_stats(ctx, n_loads, ctx->x64, ctx->r64, nullptr, nullptr));
      std::vector<PcgState> hs0(n_loads);
      for (int l = 0; l < n_loads; ++l) {
        std::memset(&hs0[l], 0, sizeof(PcgState));
        hs0[l].bnorm2 = h0[l].bnorm2;
        hs0[l].tol2_rel = tol * tol;
        hs0[l].state = ST_RUN;
        hs0[l].max_iter = ctx->opt.max_iter;
      }
      CK(cudaMemcpyAsync(ctx->st, hs0.data(), sizeof(PcgState) * n_loads, cudaMemcpyHostToDevice, s));
    } else {
      CK(cudaMemcpyAsync(ctx->r64, ctx->b64, sizeof(double) * cN * n_loads, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemsetAsync(ctx->x64, 0, sizeof(double) * cN * n_loads, s));
      TRY(set_states(ctx, n_loads, tol, ctx->opt.max_iter, -1.0));
    }
    TRY(pcg_init<double>(ctx, n_loads, ctx->r64, ctx->p64));
    return FEHOM_OK;
  }

  // Prepares the next PCG run; *need = false when the solve is complete (nothing to iterate).
  fehom_status begin_step(bool* need) {
    *need = false;
    if (finished) return FEHOM_OK;
    if (!mixed) {
      *need = steps == 0;
      return FEHOM_OK;
    }
    cudaStream_t s = ctx->stream;
    const long long cN = (long long)ctx->d.c * ctx->d.N;
    const double* r64 = ctx->b64;
    if (steps > 0 && df) {
      // r = b - K x updated by the last correction d (x += d in FP64): r -= K d with K d in
      // double-float arithmetic (FP32 pairs), ||r||^2 and <sigma> from the dual sums of x + e
      std::vector<double> dT;
      TRY(residual_update_df(ctx, n_loads, ctx->x32, (steps == 1 && !x0) ? ctx->b64 : ctx->r64, ctx->r64, &rn2,
                             &dT));
      for (size_t i = 0; i < tsum.size(); ++i) tsum[i] += dT[i];
      sums_to_flux(ctx, n_loads, tsum, &flux);
      r64 = ctx->r64;
      stats_current = true;
      last_res = ctx->r64;
    } else if (steps > 0 || x0) {
      // true residual r = b - K x = -D^T W C (e + D x) in FP64, with ||r||^2 and <sigma>
      TRY(residual_stats(ctx, n_loads, ctx->x64, ctx->r64, &rn2, &flux, &tsum));
      r64 = ctx->r64;
      stats_current = true;
      last_res = ctx->r64;
    }
    if (steps == 0 && x0) {
      // normalisation <b, K_ref^+ b> from b itself
      CK(launch_cast_d2f(ctx->b64, ctx->r32, 1.0, cN * n_loads, s));
      count_launch(ctx);
      TRY(set_states(ctx, n_loads, ctx->opt.inner_tol, 1, -1.0));
      TRY(pcg_init<float>(ctx, n_loads, ctx->r32, ctx->p32));
      std::vector<PcgState> h0(n_loads);
      CK(cudaMemcpyAsync(h0.data(), ctx->st, sizeof(PcgState) * n_loads, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int l = 0; l < n_loads; ++l) bnorm2[l] = h0[l].rz_init;
    }
    CK(launch_cast_d2f(r64, ctx->r32, 1.0, cN * n_loads, s));
    count_launch(ctx);
    CK(cudaMemsetAsync(ctx->x32, 0, sizeof(float) * cN * n_loads, s));
    const int remaining = std::max(1, ctx->opt.max_iter - total_inner);
    TRY(set_states(ctx, n_loads, ctx->opt.inner_tol, remaining, -1.0));
    TRY(pcg_init<float>(ctx, n_loads, ctx->r32, ctx->p32));
    std::vector<PcgState> h(n_loads);
    CK(cudaMemcpyAsync(h.data(), ctx->st, sizeof(PcgState) * n_loads, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool all = true;
    for (int l = 0; l < n_loads; ++l) {
      if (done[l]) {
        h[l].state = ST_DONE;
        continue;
      }
      if (bnorm2[l] < 0) bnorm2[l] = h[l].rz_init;
      relM[l] = bnorm2[l] > 0 ? std::sqrt(std::max(h[l].rz_init, 0.0) / bnorm2[l]) : 0.0;
      if (bnorm2[l] <= 0 || h[l].rz_init <= tol * tol * bnorm2[l]) {
        done[l] = true;
        h[l].state = ST_DONE;
      } else {
        all = false;
        outer_it[l] += 1;
        if (h[l].state != ST_RUN) h[l].state = ST_RUN;  // inner criterion met at start: still do >= 1 step
        // inner stopping point: the relative reduction inner_tol, or (if less work) half the distance
        // to the outer target tol * sqrt(<b, K_ref^+ b>)
        h[l].tol2 = std::max(h[l].tol2, 0.25 * tol * tol * bnorm2[l]);
      }
    }
    if (all || total_inner >= ctx->opt.max_iter || steps >= 60) return finish_mixed();
    CK(cudaMemcpyAsync(ctx->st, h.data(), sizeof(PcgState) * n_loads, cudaMemcpyHostToDevice, s));
    *need = true;
    return FEHOM_OK;
  }

  // After the PCG run: hs holds the device states at its end.
  fehom_status end_step() {
    ++steps;
    if (!mixed) {
      TRY(residual_stats(ctx, n_loads, ctx->x64, ctx->ap64, &rn2, &flux));  // true residual + averages
      last_res = ctx->ap64;
      rel2.resize(n_loads);
      for (int l = 0; l < n_loads; ++l) rel2[l] = bn2[l] > 0 ? std::sqrt(rn2[l] / bn2[l]) : 0.0;
      finished = true;
      return FEHOM_OK;
    }
    const long long cN = (long long)ctx->d.c * ctx->d.N;
    int mx = 0;
    for (int l = 0; l < n_loads; ++l) {
      if (!done[l]) inner_it[l] += hs[l].iter;
      mx = std::max(mx, hs[l].iter);
    }
    total_inner += mx;
    CK(launch_add_f2d(ctx->x32, ctx->x64, 1.0, cN * n_loads, ctx->stream));
    count_launch(ctx);
    stats_current = false;
    return FEHOM_OK;
  }

  fehom_status finish_mixed() {
    if (!stats_current) {
      TRY(residual_stats(ctx, n_loads, ctx->x64, ctx->ap64, &rn2, &flux));
      last_res = ctx->ap64;
    }
    rel2.resize(n_loads);
    for (int l = 0; l < n_loads; ++l) {
      hs[l].iter = inner_it[l];
      hs[l].state = done[l] ? ST_DONE : ST_MAXIT;
      rel2[l] = bn2[l] > 0 ? std::sqrt(rn2[l] / bn2[l]) : 0.0;
    }
    finished = true;
    return FEHOM_OK;
  }

  // outputs, info and status of the finished solve
  fehom_status report(double* fluct_out, int fluct_on_device, double* mean_flux_out, double* c_eff_out,
                      fehom_solve_info* info, float ms) {
    TRY(finish_outputs(ctx, n_loads, loads, fluct_out, fluct_on_device, mean_flux_out, c_eff_out, flux, last_res));
    bool brk = false, notconv = false;
    for (int l = 0; l < n_loads; ++l) {
      if (hs[l].state == ST_BREAK) brk = true;
      if (hs[l].state != ST_DONE) notconv = true;
      if (info) {
        info[l].iterations = hs[l].iter;
        info[l].refinements = mixed ? outer_it[l] : 0;
        info[l].converged = hs[l].state == ST_DONE;
        info[l].rel_residual_M =
            mixed ? relM[l] : (hs[l].bnorm2 > 0 ? std::sqrt(std::max(hs[l].rz, 0.0) / hs[l].bnorm2) : 0.0);
        info[l].rel_residual_2 = rel2[l];
        info[l].solve_ms = ms;
      }
    }
    if (brk) FAIL(FEHOM_E_BREAKDOWN, "PCG breakdown (non-positive or non-finite curvature)");
    if (notconv) FAIL(FEHOM_E_NOT_CONVERGED, "PCG did not reach the tolerance within max_iter");
    ctx->err.clear();
    return FEHOM_OK;
  }
};

static fehom_status check_solve_args(fehom_ctx* ctx, int n_loads, const double* loads, double tol) {
  if (!ctx->built) FAIL(FEHOM_E_STATE, "fehom_solve before fehom_precond_build");
  if (n_loads < 1 || n_loads > kMaxLoads || !loads) FAIL(FEHOM_E_INVALID, "n_loads must be in 1..64 with loads given");
  if (!(tol > 0.0 && tol < 1.0)) FAIL(FEHOM_E_INVALID, "tol must be in (0, 1)");
  for (int i = 0; i < n_loads * ctx->m; ++i)
    if (!std::isfinite(loads[i])) FAIL(FEHOM_E_INVALID, "non-finite load");
  return FEHOM_OK;
}

// ----------------------------------------------------------------------------------------------------
// batches of contexts: their PCG iterations replayed from one CUDA graph, one branch per context
// ----------------------------------------------------------------------------------------------------
}  // extern "C"

struct fehom_batch {
  std::vector<fehom_ctx*> ctxs;
  cudaStream_t main = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  PcgState* st = nullptr;                      // [n_ctx][kMaxLoads], the contexts' states during a batch
  cudaGraphExec_t exec[2] = {nullptr, nullptr}; // per precision (FP64, FP32)
  int exec_loads[2] = {0, 0};
  int per_ctx_launches[2] = {0, 0};
  std::string err;
};

namespace {

#define BCK(call)                                                                 \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      b->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return e_ == cudaErrorMemoryAllocation ? FEHOM_E_OOM : FEHOM_E_CUDA;        \
    }                                                                             \
  } while (0)

fehom_status mark_done(fehom_ctx* ctx, int n_loads) {
  std::vector<PcgState> h(n_loads);
  for (auto& x : h) {
    std::memset(&x, 0, sizeof(x));
    x.state = ST_DONE;
  }
  CK(cudaMemcpyAsync(ctx->st, h.data(), sizeof(PcgState) * n_loads, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FEHOM_OK;
}

template <typename T> T* buf_x(fehom_ctx* c) { if constexpr (sizeof(T) == 4) return c->x32; else return c->x64; }
template <typename T> T* buf_r(fehom_ctx* c) { if constexpr (sizeof(T) == 4) return c->r32; else return c->r64; }
template <typename T> T* buf_p(fehom_ctx* c) { if constexpr (sizeof(T) == 4) return c->p32; else return c->p64; }
template <typename T> T* buf_ap(fehom_ctx* c) { if constexpr (sizeof(T) == 4) return c->ap32; else return c->ap64; }

// PCG iterations of every context of the batch until all their loads are finished
template <typename T>
fehom_status run_iterations_batch(fehom_batch* b, std::vector<SolveRun>& runs, int n_loads, int max_iter) {
  const int prec = sizeof(T) == 4 ? 1 : 0;
  const int nc = (int)b->ctxs.size();
  if (!b->exec[prec] || b->exec_loads[prec] != n_loads) {
    if (b->exec[prec]) cudaGraphExecDestroy(b->exec[prec]);
    b->exec[prec] = nullptr;
    cudaGraph_t g;
    BCK(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b->fork, b->main);
    int launches = 0;
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
      fehom_ctx* ctx = b->ctxs[c];
      e = cudaStreamWaitEvent(ctx->stream, b->fork, 0);
      const long long before = ctx->launches;
      for (int i = 0; i < kChunk && e == cudaSuccess; ++i)
        e = pcg_iteration<T>(ctx, n_loads, buf_x<T>(ctx), buf_r<T>(ctx), buf_p<T>(ctx), buf_ap<T>(ctx), ctx->stream);
      launches = (int)(ctx->launches - before);
      ctx->launches = before;  // counted per replay
      if (e == cudaSuccess) e = cudaEventRecord(b->joins[c], ctx->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->joins[c], 0);
    }
    const cudaError_t e2 = cudaStreamEndCapture(b->main, &g);
    BCK(e);
    BCK(e2);
    BCK(cudaGraphInstantiate(&b->exec[prec], g, 0));
    cudaGraphDestroy(g);
    b->exec_loads[prec] = n_loads;
    b->per_ctx_launches[prec] = launches;
  }
  // the contexts' set-up work (on their own streams) precedes the replays
  for (int c = 0; c < nc; ++c) {
    BCK(cudaEventRecord(b->joins[c], b->ctxs[c]->stream));
    BCK(cudaStreamWaitEvent(b->main, b->joins[c], 0));
  }
  std::vector<PcgState> hs((size_t)nc * kMaxLoads);
  for (int done = 0; done < max_iter + kChunk;) {
    BCK(cudaGraphLaunch(b->exec[prec], b->main));
    for (auto* ctx : b->ctxs) ctx->launches += b->per_ctx_launches[prec];
    done += kChunk;
    BCK(cudaMemcpyAsync(hs.data(), b->st, sizeof(PcgState) * hs.size(), cudaMemcpyDeviceToHost, b->main));
    BCK(cudaStreamSynchronize(b->main));
    bool all = true;
    for (int c = 0; c < nc; ++c)
      for (int l = 0; l < n_loads; ++l) {
        const int st = hs[(size_t)c * kMaxLoads + l].state;
        if (st == ST_RUN || st == ST_CONV || st == ST_FIN_MAX) all = false;
      }
    if (all) break;
  }
  for (int c = 0; c < nc; ++c) {
    runs[c].hs.assign(hs.begin() + (size_t)c * kMaxLoads, hs.begin() + (size_t)c * kMaxLoads + n_loads);
    for (int l = 0; l < n_loads; ++l) b->ctxs[c]->hist_count[l] = std::min(runs[c].hs[l].iter, kHist);
  }
  return FEHOM_OK;
}

}  // namespace

extern "C" {

fehom_status fehom_batch_create(fehom_batch** out, int n_ctx, fehom_ctx* const* ctxs) {
  if (!out || n_ctx < 1 || !ctxs) return FEHOM_E_INVALID;
  *out = nullptr;
  for (int c = 0; c < n_ctx; ++c)
    if (!ctxs[c]) return FEHOM_E_INVALID;
  fehom_batch* b = new (std::nothrow) fehom_batch();
  if (!b) return FEHOM_E_OOM;
  b->ctxs.assign(ctxs, ctxs + n_ctx);
  auto fail = [&](fehom_status st) {
    g_setup_error = b->err;
    fehom_batch_destroy(b);
    return st;
  };
  const int dev = ctxs[0]->device;
  const int prec = ctxs[0]->opt.precision;
  for (int c = 0; c < n_ctx; ++c) {
    if (ctxs[c]->device != dev) {
      b->err = "all contexts of a batch must live on one device";
      return fail(FEHOM_E_INVALID);
    }
    if (ctxs[c]->opt.precision != prec) {
      b->err = "all contexts of a batch must use the same precision";
      return fail(FEHOM_E_INVALID);
    }
    for (int k = 0; k < c; ++k)
      if (ctxs[k] == ctxs[c]) {
        b->err = "a context appears twice in the batch";
        return fail(FEHOM_E_INVALID);
      }
  }
  cudaError_t e = cudaStreamCreate(&b->main);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  b->joins.resize(n_ctx, nullptr);
  for (int c = 0; c < n_ctx && e == cudaSuccess; ++c) e = cudaEventCreateWithFlags(&b->joins[c], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&b->st, sizeof(PcgState) * (size_t)n_ctx * kMaxLoads);
  if (e != cudaSuccess) {
    b->err = std::string("fehom_batch_create: ") + cudaGetErrorString(e);
    return fail(e == cudaErrorMemoryAllocation ? FEHOM_E_OOM : FEHOM_E_CUDA);
  }
  *out = b;
  return FEHOM_OK;
}

void fehom_batch_destroy(fehom_batch* b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  for (int p = 0; p < 2; ++p)
    if (b->exec[p]) cudaGraphExecDestroy(b->exec[p]);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto ev : b->joins)
    if (ev) cudaEventDestroy(ev);
  if (b->st) cudaFree(b->st);
  if (b->main) cudaStreamDestroy(b->main);
  delete b;
}

const char* fehom_batch_last_error(const fehom_batch* b) { return b ? b->err.c_str() : g_setup_error.c_str(); }

fehom_status fehom_solve_batch(fehom_batch* b, int n_loads, const double* loads, double tol, double* mean_flux_out,
                               double* c_eff_out, fehom_solve_info* info) {
  if (!b) return FEHOM_E_INVALID;
  const int nc = (int)b->ctxs.size();
  for (int c = 0; c < nc; ++c) {
    const fehom_status st = check_solve_args(b->ctxs[c], n_loads, loads, tol);
    if (st != FEHOM_OK) {
      b->err = "context " + std::to_string(c) + ": " + b->ctxs[c]->err;
      return st;
    }
  }
  const bool mixed = b->ctxs[0]->opt.precision == FEHOM_MIXED;
  // every context keeps its PCG states in the batch's array while the batch runs
  std::vector<PcgState*> saved(nc);
  for (int c = 0; c < nc; ++c) {
    saved[c] = b->ctxs[c]->st;
    b->ctxs[c]->st = b->st + (size_t)c * kMaxLoads;
  }
  auto body = [&]() -> fehom_status {
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    BCK(cudaEventRecord(e0, b->main));
    std::vector<SolveRun> runs(nc);
    for (int c = 0; c < nc; ++c) {
      SolveRun& r = runs[c];
      r.ctx = b->ctxs[c];
      r.n_loads = n_loads;
      r.loads = loads;
      r.tol = tol;
      r.mixed = mixed;
      const fehom_status st = r.begin();
      if (st != FEHOM_OK) {
        b->err = "context " + std::to_string(c) + ": " + r.ctx->err;
        return st;
      }
    }
    int max_iter = 0;
    for (auto* ctx : b->ctxs) max_iter = std::max(max_iter, ctx->opt.max_iter);
    for (;;) {
      bool any = false;
      for (int c = 0; c < nc; ++c) {
        bool need = false;
        fehom_status st = runs[c].begin_step(&need);
        if (st == FEHOM_OK && !need) st = mark_done(runs[c].ctx, n_loads);
        if (st != FEHOM_OK) {
          b->err = "context " + std::to_string(c) + ": " + runs[c].ctx->err;
          return st;
        }
        any = any || need;
      }
      if (!any) break;
      const fehom_status st = mixed ? run_iterations_batch<float>(b, runs, n_loads, max_iter)
                                    : run_iterations_batch<double>(b, runs, n_loads, max_iter);
      if (st != FEHOM_OK) return st;
      for (int c = 0; c < nc; ++c) {
        if (runs[c].finished) continue;
        const fehom_status st2 = runs[c].end_step();
        if (st2 != FEHOM_OK) {
          b->err = "context " + std::to_string(c) + ": " + runs[c].ctx->err;
          return st2;
        }
      }
    }
    for (auto* ctx : b->ctxs) {
      BCK(cudaEventRecord(b->joins[0], ctx->stream));
      BCK(cudaStreamWaitEvent(b->main, b->joins[0], 0));
    }
    BCK(cudaEventRecord(e1, b->main));
    BCK(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    fehom_status worst = FEHOM_OK;
    const int m = b->ctxs[0]->m;
    for (int c = 0; c < nc; ++c) {
      const int mc = b->ctxs[c]->m;
      const fehom_status st = runs[c].report(nullptr, 0, mean_flux_out ? mean_flux_out + (size_t)c * n_loads * mc : nullptr,
                                             c_eff_out ? c_eff_out + (size_t)c * mc * mc : nullptr,
                                             info ? info + (size_t)c * n_loads : nullptr, ms);
      if (st != FEHOM_OK && (worst == FEHOM_OK || st == FEHOM_E_CUDA)) {
        worst = st;
        b->err = "context " + std::to_string(c) + ": " + runs[c].ctx->err;
      }
    }
    (void)m;
    if (worst == FEHOM_OK) b->err.clear();
    return worst;
  };
  const fehom_status st = body();
  for (int c = 0; c < nc; ++c) b->ctxs[c]->st = saved[c];
  return st;
}

fehom_status fehom_solve(fehom_ctx* ctx, int n_loads, const double* loads, double tol, const double* x0,
                         double* fluct_out, int fluct_on_device, double* mean_flux_out, double* c_eff_out,
                         fehom_solve_info* info) {
  if (!ctx) return FEHOM_E_INVALID;
  TRY(check_solve_args(ctx, n_loads, loads, tol));
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  SolveRun run;
  run.ctx = ctx;
  run.n_loads = n_loads;
  run.loads = loads;
  run.tol = tol;
  run.x0 = x0;
  run.mixed = ctx->opt.precision == FEHOM_MIXED;
  TRY(run.begin());
  for (;;) {
    bool need = false;
    TRY(run.begin_step(&need));
    if (!need) break;
    if (run.mixed) TRY(run_iterations<float>(ctx, n_loads, ctx->x32, ctx->r32, ctx->p32, ctx->ap32,
                                             std::max(1, ctx->opt.max_iter - run.total_inner), run.hs));
    else TRY(run_iterations<double>(ctx, n_loads, ctx->x64, ctx->r64, ctx->p64, ctx->ap64, ctx->opt.max_iter, run.hs));
    TRY(run.end_step());
  }
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return run.report(fluct_out, fluct_on_device, mean_flux_out, c_eff_out, info, ms);
}

}  // extern "C"
