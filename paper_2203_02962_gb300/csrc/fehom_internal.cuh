// Internal declarations shared by the translation units of libfehom.so.
//
// Layout in device memory (one context = one periodic cell):
//   fields   T[load][comp][N]            x fastest inside a component (N = nx ny nz)
//   spectra  complex<T>[load][comp][Nh]   half spectrum, kx = 0..nx/2 fastest (Nh = nxh ny nz)
//   symbol   T[entry][Nh]                packed symmetric K_hat^+(k) / N (Sec. 5.3)
//   ids      uint8[N]                    phase id per pixel/voxel
//   mats     T[phase][D*D]               gradient-space material (see stencil.cu)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fehom {

constexpr int kMaxLoads = 64;      // loads solved as one batch
constexpr int kMaxPhases = 256;

enum Elem { P1TRI2_2D = 1, HEX8_3D = 2, Q1_2D = 3, P1TRI4_2D = 4 };  // P1TRI4_2D: two node types per pixel (c = 2 blocks)

struct Dims {
  int dim;        // 2 or 3
  int nx, ny, nz; // nz == 1 in 2-D
  int nxh;        // nx / 2 + 1
  long long N;    // nx ny nz
  long long Nh;   // nxh ny nz
  int c;          // DOF per node
  int elem;
};

// Per-load PCG scalars, resident in device memory (written by the last CTA of a reduction).
struct PcgState {
  double rz;       // <r, z> of the current iterate
  double pAp;      // <p, K p>
  double alpha, beta;
  double bnorm2;   // <b, K_ref^+ b>; negative = take <r0, z0> (zero initial guess)
  double tol2_rel; // tol^2
  double tol2;     // tol^2 * bnorm2
  double rz_init;  // <r0, z0>
  int state;       // see ST_*
  int iter;
  int max_iter;
  int err;         // nonzero: a kernel gave up a bounded wait for this load (state is ST_BREAK)
};

// RUN: iterating; CONV / FIN_MAX: converged / out of iterations, finishing the current iteration
// (x update still due); DONE / MAXIT: finished; BREAK: breakdown (non-positive or non-finite curvature).
enum { ST_RUN = 0, ST_CONV = 1, ST_DONE = 2, ST_BREAK = 3, ST_MAXIT = 4, ST_FIN_MAX = 5 };

// Reduction scratch: per-load partial sums written by each CTA, plus per-load arrival counters.
struct RedScratch {
  double* partial;   // [kMaxLoads][max_blocks]
  unsigned* count;   // [kMaxLoads] arrival counters (self-resetting)
  int max_blocks;
  double* hist;      // PCG coefficients [load][2][kHist] (alpha_j, beta_j) or nullptr
};

constexpr int kHist = 2048;  // PCG coefficients kept per load (for the Lanczos / Ritz check)

// Dot-product accumulator of the FP32 kernels.  On GB300 an FP64 instruction costs 64 FP32 lanes, so
// the FP32 kernels do not accumulate in FP64 directly: each product is split exactly into float
// head + tail (fma), the heads are added with Knuth's TwoSum, their rounding errors and the product
// tails -- both of order 2^-24 of the heads -- are summed plainly into a compensation term, and the
// per-thread (sum, compensation) pair is converted to FP64 once.  The per-thread result carries
// FP64-level accuracy (relative error of order 2^-48 of the sum of magnitudes); the CTA and grid
// reductions that follow are FP64.  The FP64 kernels accumulate in FP64.
template <typename T> struct DotAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(T a, T b) { s = fma((double)a, (double)b, s); }
  __device__ __forceinline__ void add_scaled(T a, T b, double w) { s = fma(w * (double)a, (double)b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<float> {
  float s = 0.0f, c = 0.0f;  // head sum; TwoSum errors and product tails
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;  // a b = p + fma(a, b, -p) exactly
    const float t = s + p;  // s + p = t + ((s - (t - z)) + (p - z)) exactly (TwoSum)
    const float z = t - s;
    c += ((s - (t - z)) + (p - z)) + fmaf(a, b, -p);
    s = t;
  }
  // w = 1 or 2 (Parseval weights): exact in float
  __device__ __forceinline__ void add_scaled(float a, float b, double w) { add((float)w * a, b); }
  __device__ __forceinline__ void scale2() { s += s; c += c; }  // exact
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// The same accumulation for the real and imaginary parts of complex FP32 products at once, in packed
// FP32x2 instructions (Blackwell FADD2 / FMUL2 / FFMA2, each rounding exactly like the scalar operation):
// add(a, b) accumulates a.x b.x and a.y b.y.
struct DotAcc2 {
  float2 s = make_float2(0.0f, 0.0f), c = make_float2(0.0f, 0.0f);
  __device__ __forceinline__ void add(float2 a, float2 b) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 p = __fmul2_rn(a, b);
    const float2 t = __fadd2_rn(s, p);
    const float2 z = __ffma2_rn(s, m1, t);                                            // t - s
    const float2 e = __fadd2_rn(__ffma2_rn(__ffma2_rn(z, m1, t), m1, s), __ffma2_rn(z, m1, p));  // TwoSum error
    c = __fadd2_rn(c, __fadd2_rn(e, __ffma2_rn(a, b, __fmul2_rn(p, m1))));            // + the product tails
    s = t;
  }
  __device__ __forceinline__ void scale2() {  // exact
    s = __fadd2_rn(s, s);
    c = __fadd2_rn(c, c);
  }
  __device__ __forceinline__ double value() const {
    return ((double)s.x + (double)c.x) + ((double)s.y + (double)c.y);
  }
};

// ------------------------------------------------------------------------------------------------
// stencil.cu
// ------------------------------------------------------------------------------------------------
// Isotropic cubic fast path: per phase lambda', mu' (the material in gradient coordinates) and the
// constants of the closed-form hex8 duals: [lambda', mu', 2 mu', lambda'/3, mu'/3, (lambda' + 4 mu')/9, 0, 0].
constexpr int kIsoStride = 8;
inline void iso_entry(double lam, double mu, double* out) {
  out[0] = lam; out[1] = mu; out[2] = 2.0 * mu; out[3] = lam / 3.0; out[4] = mu / 3.0;
  out[5] = (lam + 4.0 * mu) / 9.0; out[6] = 0.0; out[7] = 0.0;
}
// Scalar conductivity k' I (gradient coordinates): the hex8 duals are k' (q1, q2, q3), (2/3) k' (q4, q5, q6)
// and (1/3) k' q7 (each of q4..q6 enters two linear monomials weighted 1/3, q7 three bilinear ones weighted 1/9).
inline void iso_entry_scalar(double k, double* out) {
  out[0] = k; out[1] = 2.0 * k / 3.0; out[2] = k / 3.0;
  for (int i = 3; i < kIsoStride; ++i) out[i] = 0.0;
}

struct StencilArgs {
  Dims d;
  const void* x;        // [load][c][N] or nullptr (treated as zero)
  void* y;              // [load][c][N]
  const uint8_t* ids;   // [N]; nullptr = every voxel is phase 0 (uniform material)
  const void* mats;     // [phase][D*D] gradient-space material, T
  const void* iso;      // [phase][kIsoStride] (iso_entry / iso_entry_scalar) for the isotropic cubic fast path, or nullptr
  const double* tau;    // [load][phase][D] prestress of the macroscopic load (FP64), or nullptr
  int n_phases;
  int n_loads;
  long long load_stride;  // elements between loads in x / y
  double y_scale;         // y = y_scale * D^T W C (D x + e)
  int tile_rows;          // hex8 PCG apply: node rows per tile, 8 or 16 (0 = the precision's default)
  int staging;            // FP32 hex8 PCG apply, node-plane staging: 0 = cp.async copies (16-byte row copies
                          // where every x tile is full, else 4-byte), 1 = 4-byte cp.async copies, 2 = 16-byte
                          // row copies, 3 = one tensor-memory-accelerator box per plane (2 and 3: every x
                          // tile full, else refused)
  // fused PCG reduction <x, y> -> pAp, alpha = rz / pAp (nullptr = off)
  PcgState* st;
  RedScratch red;
  // fused statistics (nullptr = off): per load and CTA, sum y^2 and the sum of the monomial-1 duals
  // of the CTA's elements, [load][cta][1 + c * dim] doubles; with y == nullptr only the sums are made
  double* stats;
};

// Launches y = D^T W C (D x + e) for every load (blockIdx.z).  T = double or float.  ctas (optional)
// receives the number of CTAs per load (the stride of the statistics partials).
template <typename T>
cudaError_t launch_stiffness(const StencilArgs& a, cudaStream_t s, int* ctas = nullptr);

// CTAs per load of a stiffness launch (the stride of the statistics partials)
int stiffness_ctas(const Dims& d, int n_loads);  // CTAs per load of an FP64 launch over n_loads loads
// Refinement residual r_out = r_in - K d in double-float arithmetic (stencil.cu): a.x = d (float),
// a.y = r_out (double, may alias r_in), a.iso = the double-float isotropic table ([phase][16] floats:
// lambda', mu', 2 mu', lambda'/3, mu'/3, (lambda' + 4 mu')/9 as hi, lo pairs), a.stats = partial sums
// [load][cta][1 + 9] (sum r_out^2, sums of the monomial-1 duals of d); hex8 elasticity only.
// With taudf (per-load, per-phase prestress as float pairs, [load][phase][9][2]) instead: r_out = the
// right-hand side b = -D^T W C e (a.x, r_in unused), with sum b^2 and the prestress sums.
cudaError_t launch_residual_df(const StencilArgs& a, const double* r_in, const float* taudf, cudaStream_t s,
                               int* ctas);
int residual_df_ctas(const Dims& d, int n_loads);

cudaError_t launch_phase_histogram(const uint8_t* ids, long long N, unsigned long long* hist,
                                   cudaStream_t s);

// Sec. 4.3 bounds: per node, the phase whose lo (hi) value is smallest (largest) over the voxels that
// contain the node; histograms of those phases, [256] each (zeroed by the caller)
cudaError_t launch_eig_bounds(const Dims& d, const uint8_t* ids, const double* lo, const double* hi,
                              unsigned long long* hist_lo, unsigned long long* hist_hi, cudaStream_t s);

// ------------------------------------------------------------------------------------------------
// fft.cu
// ------------------------------------------------------------------------------------------------
struct Twiddles {  // W_L^m = exp(-2 pi i m / L) for the x (length nx), y, z axes
  const void* x;
  const void* y;
  const void* z;
};

enum FxMode {
  FX_PLAIN = 0,     // forward: spectrum of the field; inverse: write the field
  FX_PCG = 1,       // forward: r -= alpha Ap first; inverse: x += alpha p, p = z + beta p
  FX_PCG_INIT = 2   // inverse only: p = z (first preconditioner apply of PCG)
};

struct FftArgs {
  Dims d;
  int n_loads;
  long long load_stride_f;  // field stride between loads (c * N)
  long long load_stride_s;  // spectrum stride between loads (c * Nh), in complex elements
  void* spec;               // complex<T>
  Twiddles tw;
  // x-pass operands
  void* f0;          // forward: r (in/out); inverse: x (in/out) or output z (FX_PLAIN)
  const void* f1;    // forward: Ap; inverse: unused
  void* f2;          // inverse: p (in/out)
  int mode;
  // solve pass
  const void* sym;   // [entry][Nh] packed K_hat^+ / N (T)
  PcgState* st;      // nullptr = no PCG bookkeeping
  RedScratch red;
  int init;          // solve pass: 1 = first apply (sets rz, bnorm2)
  // launch plan (0 = built-in choice): x-line pairs per CTA (4, 8 or 16), columns per CTA of the y pass
  // and of the last-axis pass (2, 4, 8 or 16)
  int pairs, tc_y, tc_last;
  int herm;      // 1: Hermitian 2 x 2 symbol blocks (two-node stencil), packed (00, 11, Re 01, Im 01)
  int xy;        // 1: fused x-y passes (launch_fft_xy) in place of the separate x and y passes
  int last_reg;  // 1: register-split last-axis pass (FP32 3-D, nz = 32, 64, 96, 128 or 256, c = 1 or 3) with the block solve
};

template <typename T> cudaError_t launch_fft_x_fwd(const FftArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_fft_x_inv(const FftArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_fft_y(const FftArgs& a, int inverse, cudaStream_t s);
// last axis (z in 3-D, y in 2-D): forward FFT, z^ = K_hat^+ r^ / N, <r, z>, inverse FFT.
// sym == nullptr: forward only (used by Algorithm 2).
template <typename T> cudaError_t launch_fft_last_solve(const FftArgs& a, cudaStream_t s);
// Fused x-y passes (one CTA per z-plane and component; FP32 3-D fields with n x n planes, n = 32, 64,
// 96 or 128):
// forward = x forward (with the FX_PCG update) + y forward; inverse = y inverse + x inverse (with the
// FX_PCG / FX_PCG_INIT updates and the iteration bookkeeping).  cudaErrorInvalidValue when unsupported.
template <typename T> cudaError_t launch_fft_xy(const FftArgs& a, int inverse, cudaStream_t s);
bool fft_xy_supported(const Dims& d, bool fp32);
bool fft_last_rs_supported(const Dims& d, bool fp32);

// Algorithm 2 tail: spectra of the c impulse responses -> packed FP64 K_hat blocks, with the
// largest |Im| and largest asymmetry recorded; then per-wavevector inverse.
struct SymbolArgs {
  Dims d;
  const void* spec;  // complex<double>[beta][alpha][Nh]: spectrum of component alpha of K_ref i^beta
  double* sym64;     // [entry][Nh] output K_hat^+ / N
  float* sym32;      // [entry][Nh] output (float copy) or nullptr
  double* diag;      // [4]: max |Im|, max asymmetry, max |K_hat|, min eigenvalue ratio (atomic max/min via partials)
  double* partial;   // [blocks][4]
  double zero_tol;   // relative cut for the k = 0 pseudo-inverse
  int herm;          // 1: two-node stencil, Hermitian 2 x 2 blocks packed (00, 11, Re 01, Im 01)
};
cudaError_t launch_symbol_build(const SymbolArgs& a, int* blocks_out, cudaStream_t s);

cudaError_t make_twiddles(int L, double2** d64, float2** d32);

// ------------------------------------------------------------------------------------------------
// vec.cu: small vector kernels used by the solve driver
// ------------------------------------------------------------------------------------------------
cudaError_t launch_cast_d2f(const double* x, float* y, double scale, long long n, cudaStream_t s);
cudaError_t launch_add_f2d(const float* x, double* y, double scale, long long n, cudaStream_t s);
// Algorithm 2 on a proxy grid: copies the 3^d-node neighbourhood of node 0 of the impulse responses
// computed on the 4^d proxy `pd` (py: [beta][alpha][pd.N]) into zeroed full-grid columns
// (out: [beta][alpha][full.N])
cudaError_t launch_impulse_scatter(const double* py, const Dims& pd, const Dims& full, int c, double* out,
                                   cudaStream_t s);

// removes the mean of every (component, load); partial: scratch of n_loads * c * 304 doubles (two launches)
cudaError_t launch_sub_mean(double* x, int c, long long N, int n_loads, long long load_stride, double* partial,
                            cudaStream_t s);
// out[(i L + j) 2 + k] = x_i . b_j (k = 0), x_i . r_j (k = 1) for i, j < L <= 6, slices of n doubles;
// partial: scratch of L * 2 L * 304 doubles; out: 2 L^2 doubles (device).  Fixed summation order.
cudaError_t launch_pair_dots(const double* x, const double* r, int L, long long n, double* partial, double* out,
                             cudaStream_t s);
// x[l] *= gamma_l = <x[l], b[l]> / <x[l], kx[l]> (0 when <x[l], kx[l]> <= 0), l < n_loads, slices of n doubles;
// partial: scratch of n_loads * 2 * 304 doubles (two launches, fixed summation order)
cudaError_t launch_galerkin_scale(double* x, const double* kx, const double* b, int n_loads, long long n,
                                  double* partial, cudaStream_t s);

// ------------------------------------------------------------------------------------------------
// Newton's method for a nonlinear scalar conductivity (hex8, per-Gauss-point tangents, FP64)
// ------------------------------------------------------------------------------------------------
struct NlArgs {
  Dims d;
  double h[3];          // voxel edges
  double vvox;          // voxel volume
  const double* x;      // element kernels: the nodal field; gather: the dot partner
  double e[3];          // macroscopic gradient (flux mode)
  const uint8_t* ids;   // phase per voxel (nullptr: phase 0)
  const double* kp;     // per phase: k
  const double* np;     // per phase: n
  double g0;
  double* T;            // [N][8][6] tangents per Gauss point (xx, yy, zz, yz, xz, xy)
  double* E;            // [N][8] element contributions per corner
  double* y;            // gather output [N]
  double* partial;      // block partials
};
int nl_blocks(long long n);
int nl_vec_blocks();
// mode 0: flux + tangent at x (partials: sum w q (3), sum w A (6) per block); 1: tangent apply to x;
// 2: partials of sum w |D x|^2
cudaError_t launch_nl_element(const NlArgs& a, int mode, cudaStream_t s);
cudaError_t launch_nl_gather(const NlArgs& a, double scale, int dot, cudaStream_t s);
cudaError_t launch_nl_axpby(long long n, double alpha, const double* x, double beta, double* y, const double* z,
                            double* partial, cudaStream_t s);
cudaError_t launch_nl_dot(long long n, const double* x, const double* y, double* partial, cudaStream_t s);

}  // namespace fehom
