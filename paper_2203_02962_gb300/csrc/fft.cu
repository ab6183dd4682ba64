// Fourier-space application of the reference-material preconditioner (Sec. 4.2, Eq. M_inverse) and
// the Fourier part of Algorithm 2 (Sec. 5.2), as shared-memory Stockham FFT passes.
//
// Transform convention: unnormalised forward DFT exp(-2 pi i k.x / n); the inverse DFT's 1/N is
// folded into the stored symbol K_hat^+ / N.  A real field is stored as its half spectrum
// (kx = 0 .. nx/2) per component.
//
// Passes (3-D; in 2-D the last axis is y and there is no middle pass):
//   x forward  : two real lines packed into one complex line (re = line 2q, im = line 2q+1), one
//                complex FFT of length nx, split into the two half spectra.  Fused PCG update
//                r <- r - alpha Ap in front (FX_PCG).
//   y forward / inverse : complex FFT along y of a tile of TC consecutive half-spectrum columns.
//   last axis  : forward FFT, per-wavevector block solve z^ = K_hat^+ r^ / N (c x c real symmetric,
//                Sec. 5.3, Eq. block_inversion), Parseval partial sum <r, z>, inverse FFT, for all c
//                components of the same columns in one CTA.  Without a symbol: forward only.
//   x inverse  : two half spectra -> one complex line (Hermitian completion), inverse FFT, split into
//                the two real lines.  Fused PCG update x <- x + alpha p, p <- z + beta p (FX_PCG).
//
// Stockham autosort stages in shared memory: a stage of radix R with span Ns reads butterfly j's
// inputs at j + r L/R, multiplies input r by W^(r (j mod Ns)) of the length-(Ns R) transform, does
// an R-point DFT in registers and writes output r to (j / Ns) Ns R + (j mod Ns) + r Ns.  Radices
// 3 (once, for 3 * 2^k), 8, 4, 2.  Twiddles come from a per-axis table W_L^m = exp(-2 pi i m / L)
// computed on the host in long double from octant symmetry.
#include "fehom_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace fehom {
namespace {

template <typename T> struct V2;
template <> struct V2<double> { using t = double2; };
template <> struct V2<float> { using t = float2; };

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
// FP32 complex additions as one packed FP32x2 instruction each (a - b as fma(b, -1, a): the same rounding)
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  return mk<C>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// multiply by -i (forward) or +i (inverse)
template <typename C, bool INV> __device__ __forceinline__ C rot(C a) {
  return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}

// R-point DFT in registers (sign -1 forward, +1 inverse), natural order in and out.
template <typename C, int R, bool INV> __device__ __forceinline__ void dft(C (&v)[R]);

template <typename C, bool INV> __device__ __forceinline__ void dft2(C& a, C& b) {
  const C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <typename C, bool INV> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  const C a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), d = rot<C, INV>(csub(v1, v3));
  v0 = cadd(a, c);
  v2 = csub(a, c);
  v1 = cadd(b, d);
  v3 = csub(b, d);
}

// FP32: the four sums and differences as packed FP32x2 instructions; the butterflies with the +-i
// rotation mix the real and imaginary parts, so they stay scalar (the negation folds into the add)
template <> __device__ __forceinline__ void dft4<float2, false>(float2& v0, float2& v1, float2& v2, float2& v3) {
  const float2 a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), e = csub(v1, v3);
  v0 = cadd(a, c);
  v2 = csub(a, c);
  v1 = make_float2(b.x + e.y, b.y - e.x);  // b + (-i) e
  v3 = make_float2(b.x - e.y, b.y + e.x);
}
template <> __device__ __forceinline__ void dft4<float2, true>(float2& v0, float2& v1, float2& v2, float2& v3) {
  const float2 a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), e = csub(v1, v3);
  v0 = cadd(a, c);
  v2 = csub(a, c);
  v1 = make_float2(b.x - e.y, b.y + e.x);  // b + i e
  v3 = make_float2(b.x + e.y, b.y - e.x);
}

template <typename C, int R, bool INV> struct Dft;
template <typename C, bool INV> struct Dft<C, 2, INV> {
  __device__ static void run(C (&v)[2]) { dft2<C, INV>(v[0], v[1]); }
};
template <typename C, bool INV> struct Dft<C, 4, INV> {
  __device__ static void run(C (&v)[4]) { dft4<C, INV>(v[0], v[1], v[2], v[3]); }
};
template <typename C, bool INV> struct Dft<C, 8, INV> {
  // one radix-2 decimation-in-frequency step, then two 4-point DFTs
  __device__ static void run(C (&v)[8]) {
    using T = decltype(C::x);
    const T r2 = T(0.70710678118654752440);
    C a[4], b[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      a[n] = cadd(v[n], v[n + 4]);
      b[n] = csub(v[n], v[n + 4]);
    }
    // b[n] *= W_8^n  (forward W_8 = (1 - i)/sqrt 2; inverse: conjugate)
    b[1] = INV ? mk<C>(r2 * (b[1].x - b[1].y), r2 * (b[1].x + b[1].y))
               : mk<C>(r2 * (b[1].x + b[1].y), r2 * (b[1].y - b[1].x));
    b[2] = rot<C, INV>(b[2]);
    b[3] = INV ? mk<C>(-r2 * (b[3].x + b[3].y), r2 * (b[3].x - b[3].y))
               : mk<C>(r2 * (b[3].y - b[3].x), -r2 * (b[3].x + b[3].y));
    dft4<C, INV>(a[0], a[1], a[2], a[3]);
    dft4<C, INV>(b[0], b[1], b[2], b[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = a[k];
      v[2 * k + 1] = b[k];
    }
  }
};
template <typename C, bool INV> struct Dft<C, 3, INV> {
  __device__ static void run(C (&v)[3]) {
    using T = decltype(C::x);
    const T s3 = T(0.86602540378443864676);  // sin(2 pi / 3)
    const C t1 = cadd(v[1], v[2]);
    const C d = csub(v[1], v[2]);
    const C m = mk<C>(fma(T(-0.5), t1.x, v[0].x), fma(T(-0.5), t1.y, v[0].y));
    // t2 = (v1 - v2) * (-i sin(2 pi/3)) forward, (+i ...) inverse
    const C t2 = INV ? mk<C>(-s3 * d.y, s3 * d.x) : mk<C>(s3 * d.y, -s3 * d.x);
    v[0] = cadd(v[0], t1);
    v[1] = cadd(m, t2);
    v[2] = csub(m, t2);
  }
};

// One Stockham stage over NCOLS independent columns held element-major in shared memory
// (element e of column col at e * LD + col).  Ns (the span of the stages done so far) is a power of
// two: the radix-3 stage, when there is one, runs last.
template <typename C, int R, bool INV, int NCOLS, int LD>
__device__ __forceinline__ void stage(const C* __restrict__ in, C* __restrict__ out, int L, int Ns,
                                      const C* __restrict__ tw) {
  const int nb = L / R;
  const int tstride = L / (Ns * R);
  const int nw = NCOLS * nb;
  for (int w = threadIdx.x; w < nw; w += blockDim.x) {
    const int col = w % NCOLS, j = w / NCOLS;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[(j + r * nb) * LD + col];
    const int kk = j & (Ns - 1);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const C w_ = __ldg(tw + kk * r * tstride);
        v[r] = INV ? cmulc(v[r], w_) : cmul(v[r], w_);
      }
    }
    Dft<C, R, INV>::run(v);
    const int base = (j - kk) * R + kk;
#pragma unroll
    for (int r = 0; r < R; ++r) out[(base + r * Ns) * LD + col] = v[r];
  }
  __syncthreads();
}

// Full length-L transform (L = 2^k or 3 * 2^k) of NCOLS columns held in b0; returns the buffer
// holding the result (b0 or b1).
template <typename C, bool INV, int NCOLS, int LD>
__device__ C* fft_smem(C* b0, C* b1, int L, const C* tw) {
  int Ns = 1;
  int rem = (L % 3 == 0) ? L / 3 : L;
  C* in = b0;
  C* out = b1;
  auto swap = [&] { C* t = in; in = out; out = t; };
  while (rem % 8 == 0 && rem != 16) {  // 16 = 4 * 4 is cheaper than 8 * 2
    stage<C, 8, INV, NCOLS, LD>(in, out, L, Ns, tw);
    Ns *= 8; rem /= 8;
    swap();
  }
  while (rem % 4 == 0) {
    stage<C, 4, INV, NCOLS, LD>(in, out, L, Ns, tw);
    Ns *= 4; rem /= 4;
    swap();
  }
  if (rem % 2 == 0) {
    stage<C, 2, INV, NCOLS, LD>(in, out, L, Ns, tw);
    Ns *= 2; rem /= 2;
    swap();
  }
  if (L % 3 == 0) {
    stage<C, 3, INV, NCOLS, LD>(in, out, L, Ns, tw);
    swap();
  }
  return in;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double t = 0.0;
  if (w == 0) {
    t = (l < nw) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (l == 0) sh[0] = t;
  }
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

__device__ bool finish_reduction(double part, double* partial, unsigned* counter, int nblk, int bid, double* sh,
                                 double* total) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partial[bid] = part;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    last = (prev == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += ((volatile double*)partial)[b];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    *total = t;
    *counter = 0u;
  }
  return true;
}

__device__ __forceinline__ bool first_half_active(const PcgState* st, int load) {
  return st == nullptr || st[load].state == ST_RUN;
}
__device__ __forceinline__ bool second_half_active(const PcgState* st, int load) {
  if (st == nullptr) return true;
  const int s = st[load].state;
  return s == ST_RUN || s == ST_CONV || s == ST_FIN_MAX;
}

constexpr int XT = 256;  // threads of the x passes
constexpr int ST = 256;  // threads of the strided passes

// (line, position) of a flat index over lines of length n, x fastest; shift/mask when n = 2^k
struct LineIdx {
  int n, lg;
  bool pow2;
  __device__ explicit LineIdx(int n_) : n(n_), lg(0), pow2((n_ & (n_ - 1)) == 0) {
    while ((2 << lg) <= n) ++lg;
  }
  __device__ __forceinline__ void split(int idx, int& q, int& x) const {
    if (pow2) {
      q = idx >> lg;
      x = idx & (n - 1);
    } else {
      q = idx / n;
      x = idx - q * n;
    }
  }
};

// ------------------------------------------------------------------------------------------------
// x passes: P pairs of real lines per CTA, each pair packed into one complex line; shared memory
// holds the P complex lines element-major with a padded stride P + 1 (conflict-free both when the
// lines are read along x and when the butterflies run across the P columns).
// ------------------------------------------------------------------------------------------------
template <typename T, bool UPDATE, int P>
__global__ void __launch_bounds__(XT) fft_x_fwd_kernel(FftArgs a) {
  using C = typename V2<T>::t;
  constexpr int LD = P + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = a.d;
  const int nx = d.nx, nxh = d.nxh;
  C* b0 = reinterpret_cast<C*>(smem_raw);
  C* b1 = b0 + nx * LD;
  const int comp = blockIdx.y, load = blockIdx.z;
  if (UPDATE && !first_half_active(a.st, load)) return;
  const long long nlines = (long long)d.ny * d.nz;
  const long long foff = (long long)load * a.load_stride_f + (long long)comp * d.N;
  T* r = reinterpret_cast<T*>(a.f0) + foff;
  const T* ap = UPDATE ? reinterpret_cast<const T*>(a.f1) + foff : nullptr;
  C* spec = reinterpret_cast<C*>(a.spec) + (long long)load * a.load_stride_s + (long long)comp * d.Nh;
  const T alpha = UPDATE ? T(a.st[load].alpha) : T(0);
  const long long line_base = 2LL * blockIdx.x * P;
  const LineIdx li(nx);
  // BL indices per step: their global loads are issued before any of their stores, so that they are in
  // flight together (an odd line count leaves the last line unpaired)
  constexpr int BL = 4;
  for (int idx0 = threadIdx.x; idx0 < P * nx; idx0 += BL * XT) {
    T v0[BL], v1[BL];
    [[maybe_unused]] T a0[BL], a1[BL];
#pragma unroll
    for (int b = 0; b < BL; ++b) {
      v0[b] = v1[b] = T(0);
      if (UPDATE) a0[b] = a1[b] = T(0);
      const int idx = idx0 + b * XT;
      if (idx >= P * nx) continue;
      int q, xx;
      li.split(idx, q, xx);
      const long long l0 = line_base + 2 * q;
      if (l0 < nlines) {
        const bool has1 = l0 + 1 < nlines;
        const long long g0 = l0 * nx + xx, g1 = g0 + nx;
        v0[b] = r[g0];
        if (has1) v1[b] = r[g1];
        if (UPDATE) {
          a0[b] = ap[g0];
          if (has1) a1[b] = ap[g1];
        }
      }
    }
#pragma unroll
    for (int b = 0; b < BL; ++b) {
      const int idx = idx0 + b * XT;
      if (idx >= P * nx) continue;
      int q, xx;
      li.split(idx, q, xx);
      const long long l0 = line_base + 2 * q;
      T w0 = v0[b], w1 = v1[b];
      if (UPDATE && l0 < nlines) {
        const bool has1 = l0 + 1 < nlines;
        const long long g0 = l0 * nx + xx, g1 = g0 + nx;
        w0 = fma(-alpha, a0[b], w0);
        r[g0] = w0;
        if (has1) {
          w1 = fma(-alpha, a1[b], w1);
          r[g1] = w1;
        }
      }
      b0[xx * LD + q] = mk<C>(w0, w1);
    }
  }
  __syncthreads();
  const C* res = fft_smem<C, false, P, LD>(b0, b1, nx, reinterpret_cast<const C*>(a.tw.x));
  // split Z = FFT(a + i b) into the half spectra A = (Z_k + conj Z_-k)/2, B = (Z_k - conj Z_-k)/(2i)
  for (int idx = threadIdx.x; idx < P * nxh; idx += XT) {
    const int k = idx / P, q = idx % P;
    const long long l0 = line_base + 2 * q;
    if (l0 >= nlines) continue;
    const C zk = res[k * LD + q];
    const C zn = res[(k == 0 ? 0 : nx - k) * LD + q];
    const T h = T(0.5);
    spec[l0 * nxh + k] = mk<C>(h * (zk.x + zn.x), h * (zk.y - zn.y));
    if (l0 + 1 < nlines) spec[(l0 + 1) * nxh + k] = mk<C>(h * (zk.y + zn.y), h * (zn.x - zk.x));
  }
}

template <typename T, int MODE, int P>
__global__ void __launch_bounds__(XT) fft_x_inv_kernel(FftArgs a) {
  using C = typename V2<T>::t;
  constexpr int LD = P + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  const Dims d = a.d;
  const int nx = d.nx, nxh = d.nxh, half = nx / 2;
  C* b0 = reinterpret_cast<C*>(smem_raw);
  C* b1 = b0 + nx * LD;
  const int comp = blockIdx.y, load = blockIdx.z;
  if (MODE != FX_PLAIN && !second_half_active(a.st, load)) return;
  const long long nlines = (long long)d.ny * d.nz;
  const long long foff = (long long)load * a.load_stride_f + (long long)comp * d.N;
  const C* spec = reinterpret_cast<const C*>(a.spec) + (long long)load * a.load_stride_s + (long long)comp * d.Nh;
  const long long line_base = 2LL * blockIdx.x * P;
  const LineIdx li(nx);
  for (int idx = threadIdx.x; idx < P * nx; idx += XT) {
    int q, k;
    li.split(idx, q, k);
    const long long l0 = line_base + 2 * q;
    C z = mk<C>(T(0), T(0));
    if (l0 < nlines) {
      // Hermitian completion of the two half spectra, then Z = A + i B
      const bool has1 = l0 + 1 < nlines;
      const bool lo = k <= half;
      const int kk = lo ? k : nx - k;
      C A = spec[l0 * nxh + kk];
      C B = has1 ? spec[(l0 + 1) * nxh + kk] : mk<C>(T(0), T(0));
      if (!lo) {
        A.y = -A.y;
        B.y = -B.y;
      } else if (k == 0 || k == half) {
        A.y = T(0);
        B.y = T(0);
      }
      z = mk<C>(A.x - B.y, A.y + B.x);
    }
    b0[k * LD + q] = z;
  }
  __syncthreads();
  const C* res = fft_smem<C, true, P, LD>(b0, b1, nx, reinterpret_cast<const C*>(a.tw.x));
  T* f0 = reinterpret_cast<T*>(a.f0) + foff;
  T* f2 = (MODE != FX_PLAIN) ? reinterpret_cast<T*>(a.f2) + foff : nullptr;
  const T alpha = (MODE == FX_PCG) ? T(a.st[load].alpha) : T(0);
  const T beta = (MODE == FX_PCG) ? T(a.st[load].beta) : T(0);
  // BL indices per step: the x and p loads of FX_PCG are issued before any of the stores
  constexpr int BL = 4;
  for (int idx0 = threadIdx.x; idx0 < P * nx; idx0 += BL * XT) {
    [[maybe_unused]] T p0[BL], p1[BL], x0[BL], x1[BL];
    if constexpr (MODE == FX_PCG) {
#pragma unroll
      for (int b = 0; b < BL; ++b) {
        const int idx = idx0 + b * XT;
        if (idx >= P * nx) continue;
        int q, xx;
        li.split(idx, q, xx);
        const long long l0 = line_base + 2 * q;
        if (l0 >= nlines) continue;
        const long long g0 = l0 * nx + xx, g1 = g0 + nx;
        p0[b] = f2[g0];
        x0[b] = f0[g0];
        if (l0 + 1 < nlines) {
          p1[b] = f2[g1];
          x1[b] = f0[g1];
        }
      }
    }
#pragma unroll
    for (int b = 0; b < BL; ++b) {
      const int idx = idx0 + b * XT;
      if (idx >= P * nx) continue;
      int q, xx;
      li.split(idx, q, xx);
      const long long l0 = line_base + 2 * q;
      if (l0 >= nlines) continue;
      const C zc = res[xx * LD + q];
      const bool has1 = l0 + 1 < nlines;
      const long long g0 = l0 * nx + xx, g1 = g0 + nx;
      if (MODE == FX_PLAIN) {
        f0[g0] = zc.x;
        if (has1) f0[g1] = zc.y;
      } else if (MODE == FX_PCG_INIT) {
        f2[g0] = zc.x;
        if (has1) f2[g1] = zc.y;
      } else {
        f0[g0] = fma(alpha, p0[b], x0[b]);
        f2[g0] = fma(beta, p0[b], zc.x);
        if (has1) {
          f0[g1] = fma(alpha, p1[b], x1[b]);
          f2[g1] = fma(beta, p1[b], zc.y);
        }
      }
    }
  }
  if (MODE != FX_PLAIN && a.st != nullptr) {
    // the last CTA over all components finalises the iteration bookkeeping
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    double total;
    __syncthreads();
    if (finish_reduction(0.0, a.red.partial + (long long)load * a.red.max_blocks, a.red.count + load, nblk, bid,
                         red_sh, &total)) {
      if (threadIdx.x == 0) {
        PcgState& s = a.st[load];
        if (MODE == FX_PCG) s.iter += 1;
        if (s.state == ST_CONV) s.state = ST_DONE;
        else if (s.state == ST_FIN_MAX) s.state = ST_MAXIT;
      }
    }
  }
}

// ------------------------------------------------------------------------------------------------
// strided passes: columns cf = 0..ncols-1 of the half spectrum; element e of column cf at
//   (cf / nxh) * outer + e * estride + (cf % nxh).  A CTA holds TC consecutive columns; their base
//   offsets are computed once per CTA.
// ------------------------------------------------------------------------------------------------
struct ColMap {
  int L;             // transform length (axis size)
  int ncols;         // number of columns
  long long outer;   // stride of cf / nxh
  long long estride; // stride along the axis
};

template <int TC>
__device__ __forceinline__ void column_bases(const ColMap& m, int nxh, int cf0, long long* base, int* kx) {
  if (threadIdx.x < TC) {
    const int cf = cf0 + threadIdx.x;
    if (cf < m.ncols) {
      base[threadIdx.x] = (long long)(cf / nxh) * m.outer + (cf % nxh);
      kx[threadIdx.x] = cf % nxh;
    } else {
      base[threadIdx.x] = -1;
      kx[threadIdx.x] = 0;
    }
  }
  __syncthreads();
}

template <typename T, bool INV, int TC>
__global__ void __launch_bounds__(ST) fft_strided_kernel(FftArgs a, ColMap m, const typename V2<T>::t* tw) {
  using C = typename V2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long base[TC];
  __shared__ int kxs[TC];
  C* b0 = reinterpret_cast<C*>(smem_raw);
  C* b1 = b0 + m.L * TC;
  const int comp = blockIdx.y, load = blockIdx.z;
  if (a.st != nullptr) {
    if (!INV && !first_half_active(a.st, load)) return;
    if (INV && !second_half_active(a.st, load)) return;
  }
  C* spec = reinterpret_cast<C*>(a.spec) + (long long)load * a.load_stride_s + (long long)comp * a.d.Nh;
  column_bases<TC>(m, a.d.nxh, blockIdx.x * TC, base, kxs);
  for (int idx = threadIdx.x; idx < m.L * TC; idx += ST) {
    const int e = idx / TC, t = idx % TC;
    const long long cb = base[t];
    b0[idx] = cb >= 0 ? spec[cb + (long long)e * m.estride] : mk<C>(T(0), T(0));
  }
  __syncthreads();
  const C* res = fft_smem<C, INV, TC, TC>(b0, b1, m.L, tw);
  for (int idx = threadIdx.x; idx < m.L * TC; idx += ST) {
    const int e = idx / TC, t = idx % TC;
    const long long cb = base[t];
    if (cb >= 0) spec[cb + (long long)e * m.estride] = res[idx];
  }
}

// Last axis with the block solve.  3-D: axis z, columns cf = ky * nxh + kx.  2-D: axis y, cf = kx.
// Shared memory: [e][component][TC] (all c components of the same columns).
template <typename T, int NC, bool SOLVE, int TC>
__global__ void __launch_bounds__(ST) fft_last_kernel(FftArgs a, ColMap m, const typename V2<T>::t* tw) {
  using C = typename V2<T>::t;
  constexpr int W = NC * TC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  __shared__ long long base[TC];
  __shared__ int kxs[TC];
  C* b0 = reinterpret_cast<C*>(smem_raw);
  C* b1 = b0 + m.L * W;
  const int load = blockIdx.z;
  if (!first_half_active(a.st, load)) return;
  C* spec = reinterpret_cast<C*>(a.spec) + (long long)load * a.load_stride_s;
  const long long Nh = a.d.Nh;
  const int half = a.d.nx / 2;
  column_bases<TC>(m, a.d.nxh, blockIdx.x * TC, base, kxs);
  constexpr int BL = 4;  // the loads of BL elements per step are in flight together
  for (int idx0 = threadIdx.x; idx0 < m.L * W; idx0 += BL * ST) {
    C v[BL];
#pragma unroll
    for (int b = 0; b < BL; ++b) {
      const int idx = idx0 + b * ST;
      if (idx >= m.L * W) continue;
      const int e = idx / W, rem = idx % W, comp = rem / TC, t = rem % TC;
      const long long cb = base[t];
      v[b] = cb >= 0 ? spec[comp * Nh + cb + (long long)e * m.estride] : mk<C>(T(0), T(0));
    }
#pragma unroll
    for (int b = 0; b < BL; ++b)
      if (idx0 + b * ST < m.L * W) b0[idx0 + b * ST] = v[b];
  }
  __syncthreads();
  C* res = fft_smem<C, false, W, W>(b0, b1, m.L, tw);
  C* other = (res == b0) ? b1 : b0;
  if (!SOLVE) {
    for (int idx = threadIdx.x; idx < m.L * W; idx += ST) {
      const int e = idx / W, rem = idx % W, comp = rem / TC, t = rem % TC;
      const long long cb = base[t];
      if (cb >= 0) spec[comp * Nh + cb + (long long)e * m.estride] = res[idx];
    }
    return;
  }
  const T* sym = reinterpret_cast<const T*>(a.sym);
  DotAcc<T> dot;
  // the block solve z = K_hat^+ r and the Parseval sum at one wavevector (k: the symbol entries there)
  auto solve_point = [&](int idx, const T* k) {
    const int e = idx / TC, t = idx % TC;
    const int kx = kxs[t];
    const T wgt = (kx == 0 || kx == half) ? T(1) : T(2);
    C r[NC], z[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) r[c] = res[e * W + c * TC + t];
    if constexpr (NC == 1) {
      z[0] = mk<C>(k[0] * r[0].x, k[0] * r[0].y);
    } else if constexpr (NC == 2) {
      const T k00 = k[0], k11 = k[1], k01 = k[2];
      if (a.herm) {  // z0 = k00 r0 + k01 r1, z1 = conj(k01) r0 + k11 r1 with complex k01
        const T k01i = k[3];
        z[0] = mk<C>(fma(k00, r[0].x, fma(k01, r[1].x, -k01i * r[1].y)), fma(k00, r[0].y, fma(k01, r[1].y, k01i * r[1].x)));
        z[1] = mk<C>(fma(k11, r[1].x, fma(k01, r[0].x, k01i * r[0].y)), fma(k11, r[1].y, fma(k01, r[0].y, -k01i * r[0].x)));
      } else {
        z[0] = mk<C>(fma(k00, r[0].x, k01 * r[1].x), fma(k00, r[0].y, k01 * r[1].y));
        z[1] = mk<C>(fma(k01, r[0].x, k11 * r[1].x), fma(k01, r[0].y, k11 * r[1].y));
      }
    } else {
      const T k00 = k[0], k11 = k[1], k22 = k[2], k12 = k[3], k02 = k[4], k01 = k[5];
      z[0] = mk<C>(fma(k00, r[0].x, fma(k01, r[1].x, k02 * r[2].x)), fma(k00, r[0].y, fma(k01, r[1].y, k02 * r[2].y)));
      z[1] = mk<C>(fma(k01, r[0].x, fma(k11, r[1].x, k12 * r[2].x)), fma(k01, r[0].y, fma(k11, r[1].y, k12 * r[2].y)));
      z[2] = mk<C>(fma(k02, r[0].x, fma(k12, r[1].x, k22 * r[2].x)), fma(k02, r[0].y, fma(k12, r[1].y, k22 * r[2].y)));
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      dot.add(wgt * r[c].x, z[c].x);  // wgt in {1, 2}: exact
      dot.add(wgt * r[c].y, z[c].y);
      res[e * W + c * TC + t] = z[c];
    }
  };
  // symbol entries per wavevector: 1, 3 (4 with the Hermitian coupling) or 6
  constexpr int E = NC == 1 ? 1 : (NC == 2 ? 4 : 6);
  constexpr int BS = NC == 1 ? 4 : 2;  // the symbol loads of BS points per step are in flight together
  const int ne = NC == 2 ? (a.herm ? 4 : 3) : E;
  for (int idx0 = threadIdx.x; idx0 < m.L * TC; idx0 += BS * ST) {
    T k[BS][E];
#pragma unroll
    for (int b = 0; b < BS; ++b) {
      const int idx = idx0 + b * ST;
      if (idx >= m.L * TC) continue;
      const int e = idx / TC, t = idx % TC;
      const long long cb = base[t];
      if (cb < 0) continue;
      const long long ti = cb + (long long)e * m.estride;
#pragma unroll
      for (int j = 0; j < E; ++j)
        if (j < ne) k[b][j] = sym[j * Nh + ti];
    }
#pragma unroll
    for (int b = 0; b < BS; ++b) {
      const int idx = idx0 + b * ST;
      if (idx >= m.L * TC || base[idx % TC] < 0) continue;
      solve_point(idx, k[b]);
    }
  }
  __syncthreads();
  const C* out = fft_smem<C, true, W, W>(res, other, m.L, tw);
  for (int idx = threadIdx.x; idx < m.L * W; idx += ST) {
    const int e = idx / W, rem = idx % W, comp = rem / TC, t = rem % TC;
    const long long cb = base[t];
    if (cb >= 0) spec[comp * Nh + cb + (long long)e * m.estride] = out[idx];
  }
  if (a.st != nullptr) {
    const double part = block_sum(dot.value(), red_sh);
    double total;
    if (finish_reduction(part, a.red.partial + (long long)load * a.red.max_blocks, a.red.count + load, gridDim.x,
                         blockIdx.x, red_sh, &total)) {
      if (threadIdx.x == 0) {
        PcgState& s = a.st[load];
        if (a.init) {
          s.rz = total;
          s.rz_init = total;
          if (s.bnorm2 < 0.0) s.bnorm2 = total;  // zero initial guess: <b, K_ref^+ b> = <r0, z0>
          s.tol2 = s.tol2_rel * s.bnorm2;
          s.alpha = 0.0;
          s.beta = 0.0;
          if (!isfinite(total)) s.state = ST_BREAK;
          else if (total <= s.tol2) s.state = ST_CONV;
        } else {
          s.beta = (s.rz > 0.0) ? total / s.rz : 0.0;
          if (a.red.hist != nullptr && s.iter < kHist) a.red.hist[((long long)load * 2 + 1) * kHist + s.iter] = s.beta;
          s.rz = total;
          if (!isfinite(total)) s.state = ST_BREAK;
          else if (total <= s.tol2) s.state = ST_CONV;
          else if (s.iter + 1 >= s.max_iter) s.state = ST_FIN_MAX;
        }
      }
    }
  }
}


// ------------------------------------------------------------------------------------------------
// Register-split FP32 passes for axes of N = 16 Q points (N = 32, 64, 96 or 128).  Each transform is
// split N = 16 x Q: a 16-point DFT in registers over the stride-Q subsequence, the twiddles
// W_N^(j k1), one shared-memory exchange, then Q-point DFTs (output index k1 + 16 k2).
// Fused x-y passes for 3-D fields with N x N planes: one CTA transforms one z-plane of one
// component, so the half spectrum crosses HBM once per direction instead of twice.
//   forward: rows 2q, 2q+1 -> one complex line (fused r -= alpha Ap); the y pass splits the two half
//            spectra on the fly; the real columns kx = 0 and kx = N/2 share one complex column and
//            are separated after the transform.
//   inverse: columns kx = 0 and kx = N/2 (whose inverse transforms are real) share one complex
//            column; the x pass completes the Hermitian lines and applies the PCG updates of FX_PCG.
// Threads 4 N: the 16 N stage-2 tasks of a pass (N/2 lines or columns x 16 k1) in two rounds; the
// N^2/32 16-point DFTs of stage 1 (N/2 lines x Q subsequences) use all of them for N = 128 and
// 3/4, 1/2, 1/4 of them for N = 96, 64, 32.
// ------------------------------------------------------------------------------------------------
template <int N>
struct RS {
  static_assert(N == 32 || N == 64 || N == 96 || N == 128, "register-split axis lengths: 32, 64, 96, 128");
  static constexpr int Q = N / 16;   // the Q-point stage
  static constexpr int H = N / 2 + 1;  // half-spectrum width
  static constexpr int NP = N / 2;   // line pairs of the x pass, packed columns of the y pass
  static constexpr int NT = 4 * N;   // threads of the fused x-y passes
  static constexpr int MIN_CTAS = 1152 / NT > 2 ? 1152 / NT : 2;  // resident CTAs per SM the registers allow
  // Shared-memory strides (complex unless noted), padded against bank conflicts (the 128 values
  // measured, the others picked with a bank model of these access patterns):
  //   LDQ  line stride of the x-pass buffer, [k1][Q + 1] per line
  //   LDT  column stride of the y-pass buffer, [k1][Q + 1] per column
  //   LDP  row stride of the y-inverse result plane (N/2 columns used)
  //   LDF_F, LDF_I  row strides (floats) of the forward / inverse row staging, which aliases the
  //   line buffer: the N/2 line pairs as two float arrays (rows 2q and 2q + 1)
  static constexpr int LDQ = N == 128 ? 148 : N == 96 ? 118 : N == 64 ? 84 : 50;
  static constexpr int LDT = N == 128 ? 145 : N == 96 ? 113 : N == 64 ? 81 : 49;
  static constexpr int LDP = N == 128 ? 66 : N == 96 ? 50 : N == 64 ? 34 : 17;
  static constexpr int LDF_F = N == 128 ? 136 : N == 96 ? 100 : N == 64 ? 68 : 36;
  static constexpr int LDF_I = N == 128 ? 144 : N == 96 ? 112 : N == 64 ? 80 : 48;
  static constexpr int BUF = NP * LDQ;
  static constexpr size_t SMEM = (BUF + N) * sizeof(float2);
  static_assert(LDQ >= 16 * (Q + 1) && LDT >= 16 * (Q + 1) && LDP >= NP, "strides hold their rows");
  static_assert(LDF_F >= N && LDF_I >= N && LDF_F % 4 == 0 && LDF_I % 4 == 0, "16-byte aligned float rows");
  static_assert(2 * NP * LDF_F <= 2 * BUF && 2 * NP * LDF_I <= 2 * BUF, "row staging fits in the line buffer");
  static_assert(N * LDP <= BUF && NT * 2 == NP * 16, "y-inverse plane fits; two stage-2 rounds");
};

template <typename C, bool INV> struct Dft<C, 6, INV> {
  // one radix-2 decimation-in-frequency step, then two 3-point DFTs
  __device__ static void run(C (&v)[6]) {
    using T = decltype(C::x);
    const T h = T(0.5), s3 = T(0.86602540378443864676);  // W_6 = (1/2, -sin(pi/3)) forward
    C a[3], b[3];
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      a[n] = cadd(v[n], v[n + 3]);
      b[n] = csub(v[n], v[n + 3]);
    }
    b[1] = cmul(b[1], mk<C>(h, INV ? s3 : -s3));
    b[2] = cmul(b[2], mk<C>(-h, INV ? s3 : -s3));
    Dft<C, 3, INV>::run(a);
    Dft<C, 3, INV>::run(b);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      v[2 * k] = a[k];
      v[2 * k + 1] = b[k];
    }
  }
};

// 16-point DFT in registers, natural order in and out: n = n1 + 4 n2, k = 4 k1 + k2
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
  const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, r2 = 0.70710678118654752440f;
  float2 y[4][4];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    y[n1][0] = v[n1];
    y[n1][1] = v[n1 + 4];
    y[n1][2] = v[n1 + 8];
    y[n1][3] = v[n1 + 12];
    dft4<float2, INV>(y[n1][0], y[n1][1], y[n1][2], y[n1][3]);
  }
  // y[n1][k2] *= W_16^(n1 k2) (forward); conjugate for the inverse
  const float sg = INV ? 1.0f : -1.0f;
  y[1][1] = cmul(y[1][1], mk<float2>(c1, sg * s1));
  y[1][2] = cmul(y[1][2], mk<float2>(r2, sg * r2));
  y[1][3] = cmul(y[1][3], mk<float2>(s1, sg * c1));
  y[2][1] = cmul(y[2][1], mk<float2>(r2, sg * r2));
  y[2][2] = rot<float2, INV>(y[2][2]);
  y[2][3] = cmul(y[2][3], mk<float2>(-r2, sg * r2));
  y[3][1] = cmul(y[3][1], mk<float2>(s1, sg * c1));
  y[3][2] = cmul(y[3][2], mk<float2>(-r2, sg * r2));
  y[3][3] = cmul(y[3][3], mk<float2>(-c1, -sg * s1));
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    float2 a0 = y[0][k2], a1 = y[1][k2], a2 = y[2][k2], a3 = y[3][k2];
    dft4<float2, INV>(a0, a1, a2, a3);
    v[k2] = a0;
    v[4 + k2] = a1;
    v[8 + k2] = a2;
    v[12 + k2] = a3;
  }
}

// the 16-point DFT as the Q-point stage of the last-axis pass for nz = 256
template <bool INV> struct Dft<float2, 16, INV> {
  __device__ static void run(float2 (&v)[16]) { dft16<INV>(v); }
};

template <int N, bool UPDATE>
__global__ void __launch_bounds__(RS<N>::NT, RS<N>::MIN_CTAS) fft_xy_fwd_rs_kernel(FftArgs a) {
  using P = RS<N>;
  constexpr int Q = P::Q, NP = P::NP, NT = P::NT, H = P::H;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* S = reinterpret_cast<float2*>(smem_raw);
  float2* Cz = S + P::BUF;
  const int z = blockIdx.x, comp = blockIdx.y, load = blockIdx.z;
  if (UPDATE && !first_half_active(a.st, load)) return;
  const long long foff = (long long)load * a.load_stride_f + (long long)comp * a.d.N + (long long)z * N * N;
  float* r = reinterpret_cast<float*>(a.f0) + foff;
  const float* ap = UPDATE ? reinterpret_cast<const float*>(a.f1) + foff : nullptr;
  float2* spec = reinterpret_cast<float2*>(a.spec) + (long long)load * a.load_stride_s + (long long)comp * a.d.Nh +
                 (long long)z * N * H;
  const float alpha = UPDATE ? float(a.st[load].alpha) : 0.0f;
  const float2* twx = reinterpret_cast<const float2*>(a.tw.x);
  const float2* twy = reinterpret_cast<const float2*>(a.tw.y);
  const int t = threadIdx.x;
  const bool s1_thread = t < NP * Q;  // stage 1: line (or column pair index) x subsequence
  {  // x, stage 0: rows to shared memory (16-byte accesses along each row pair), r -= alpha Ap
    float* Rre = reinterpret_cast<float*>(S);
    float* Rim = Rre + NP * P::LDF_F;
    // the r and Ap loads of a batch of row pieces are issued before any of its stores, so that they are
    // in flight together
    constexpr int IT = N / 32, B = IT < 2 ? IT : 2;
#pragma unroll
    for (int it0 = 0; it0 < IT; it0 += B) {
      float4 v0[B], v1[B];
      [[maybe_unused]] float4 a0[B], a1[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        if (it0 + b < IT) {
          const int task = t + NT * (it0 + b);
          const int q = task / (N / 4), x = 4 * (task % (N / 4));
          v0[b] = *reinterpret_cast<const float4*>(r + 2 * q * N + x);
          v1[b] = *reinterpret_cast<const float4*>(r + (2 * q + 1) * N + x);
          if (UPDATE) {
            a0[b] = __ldg(reinterpret_cast<const float4*>(ap + 2 * q * N + x));
            a1[b] = __ldg(reinterpret_cast<const float4*>(ap + (2 * q + 1) * N + x));
          }
        }
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        if (it0 + b >= IT) continue;
        const int task = t + NT * (it0 + b);
        const int q = task / (N / 4), x = 4 * (task % (N / 4));
        float4 w0 = v0[b], w1 = v1[b];
        if (UPDATE) {
          w0 = make_float4(fmaf(-alpha, a0[b].x, w0.x), fmaf(-alpha, a0[b].y, w0.y), fmaf(-alpha, a0[b].z, w0.z),
                           fmaf(-alpha, a0[b].w, w0.w));
          w1 = make_float4(fmaf(-alpha, a1[b].x, w1.x), fmaf(-alpha, a1[b].y, w1.y), fmaf(-alpha, a1[b].z, w1.z),
                           fmaf(-alpha, a1[b].w, w1.w));
          *reinterpret_cast<float4*>(r + 2 * q * N + x) = w0;
          *reinterpret_cast<float4*>(r + (2 * q + 1) * N + x) = w1;
        }
        *reinterpret_cast<float4*>(Rre + q * P::LDF_F + x) = w0;
        *reinterpret_cast<float4*>(Rim + q * P::LDF_F + x) = w1;
      }
    }
  }
  __syncthreads();
  {  // x, stage 1: line q = rows (2q, 2q+1), subsequence j
    const int q = t / Q, j = t % Q;
    float2 v[16];
    if (s1_thread) {
      const float* Rre = reinterpret_cast<const float*>(S) + q * P::LDF_F + j;
      const float* Rim = Rre + NP * P::LDF_F;
#pragma unroll
      for (int m = 0; m < 16; ++m) v[m] = make_float2(Rre[Q * m], Rim[Q * m]);
    }
    __syncthreads();  // every row has been gathered before the line buffer overwrites it
    if (s1_thread) {
      dft16<false>(v);
      float2* Sq = S + q * P::LDQ;
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) Sq[k1 * (Q + 1) + j] = k1 == 0 ? v[0] : cmul(v[k1], __ldg(twx + j * k1));
    }
  }
  __syncthreads();
#pragma unroll
  for (int round = 0; round < 2; ++round) {  // x, stage 2: a warp holds both lines it rewrites
    const int task = t + NT * round;
    const int q = task >> 4, k1 = task & 15;
    float2* Sq = S + q * P::LDQ;
    float2 v[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) v[j] = Sq[k1 * (Q + 1) + j];
    __syncwarp();
    Dft<float2, Q, false>::run(v);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) Sq[k1 + 16 * k2] = v[k2];
    __syncwarp();
  }
  __syncthreads();
  {  // y, stage 1: column kx (kx = 0 carries kx = 0 and kx = N/2), subsequence j of the rows
    const int kx = t % NP, j = t / NP;
    const int sodd = j & 1, q0 = j >> 1;  // row j + Q m = 2 (q0 + (Q/2) m) + sodd (Q is even)
    float2 v[16];
    if (s1_thread) {
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const float2* Sq = S + (q0 + (Q / 2) * m) * P::LDQ;
        if (kx == 0) {
          const float2 z0 = Sq[0], zh = Sq[NP];
          v[m] = sodd ? make_float2(z0.y, zh.y) : make_float2(z0.x, zh.x);
        } else {
          const float2 zk = Sq[kx], zn = Sq[N - kx];
          v[m] = sodd ? make_float2(0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x))
                      : make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
        }
      }
    }
    __syncthreads();  // every line has been read before the column buffer overwrites it
    if (s1_thread) {
      dft16<false>(v);
      float2* Tc = S + kx * P::LDT;
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) Tc[k1 * (Q + 1) + j] = k1 == 0 ? v[0] : cmul(v[k1], __ldg(twy + j * k1));
    }
  }
  __syncthreads();
#pragma unroll
  for (int round = 0; round < 2; ++round) {  // y, stage 2 -> half spectrum (packed column to Cz)
    const int task = t + NT * round;
    const int kx = task % NP, k1 = task / NP;
    const float2* Tc = S + kx * P::LDT;
    float2 v[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) v[j] = Tc[k1 * (Q + 1) + j];
    Dft<float2, Q, false>::run(v);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
      const int ky = k1 + 16 * k2;
      if (kx == 0) Cz[ky] = v[k2];
      else spec[ky * H + kx] = v[k2];
    }
  }
  __syncthreads();
  if (t < N) {  // separate the spectra of the real columns kx = 0 and kx = N/2
    const float2 c = Cz[t], cn = Cz[t == 0 ? 0 : N - t];
    spec[t * H] = make_float2(0.5f * (c.x + cn.x), 0.5f * (c.y - cn.y));
    spec[t * H + NP] = make_float2(0.5f * (c.y + cn.y), 0.5f * (cn.x - c.x));
  }
}

template <int N, int MODE>
__global__ void __launch_bounds__(RS<N>::NT, RS<N>::MIN_CTAS) fft_xy_inv_rs_kernel(FftArgs a) {
  using P = RS<N>;
  constexpr int Q = P::Q, NP = P::NP, NT = P::NT, H = P::H;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  float2* S = reinterpret_cast<float2*>(smem_raw);
  const int z = blockIdx.x, comp = blockIdx.y, load = blockIdx.z;
  if (MODE != FX_PLAIN && !second_half_active(a.st, load)) return;
  const long long foff = (long long)load * a.load_stride_f + (long long)comp * a.d.N + (long long)z * N * N;
  const float2* spec = reinterpret_cast<const float2*>(a.spec) + (long long)load * a.load_stride_s +
                       (long long)comp * a.d.Nh + (long long)z * N * H;
  const float2* twx = reinterpret_cast<const float2*>(a.tw.x);
  const float2* twy = reinterpret_cast<const float2*>(a.tw.y);
  const int t = threadIdx.x;
  const bool s1_thread = t < NP * Q;
  if (s1_thread) {  // y inverse, stage 1: column kx (kx = 0 carries kx = 0 and kx = N/2 as real and imaginary parts)
    const int kx = t % NP, j = t / NP;
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int ky = j + Q * m;
      if (kx == 0) {
        const float2 s0 = spec[ky * H], sh = spec[ky * H + NP];
        v[m] = make_float2(s0.x - sh.y, s0.y + sh.x);
      } else {
        v[m] = spec[ky * H + kx];
      }
    }
    dft16<true>(v);
    float2* Tc = S + kx * P::LDT;
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) Tc[k1 * (Q + 1) + j] = k1 == 0 ? v[0] : cmulc(v[k1], __ldg(twy + j * k1));
  }
  __syncthreads();
  {  // y inverse, stage 2 -> plane P[y][kx]
    float2 w[2][Q];
#pragma unroll
    for (int round = 0; round < 2; ++round) {
      const int task = t + NT * round;
      const int kx = task % NP, k1 = task / NP;
#pragma unroll
      for (int j = 0; j < Q; ++j) w[round][j] = S[kx * P::LDT + k1 * (Q + 1) + j];
    }
    __syncthreads();
#pragma unroll
    for (int round = 0; round < 2; ++round) {
      const int task = t + NT * round;
      const int kx = task % NP, k1 = task / NP;
      Dft<float2, Q, true>::run(w[round]);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) S[(k1 + 16 * k2) * P::LDP + kx] = w[round][k2];
    }
  }
  __syncthreads();
  {  // x inverse, stage 1: line q = rows (2q, 2q+1), Hermitian completion, Z = A + i B
    const int q = t / Q, j = t % Q;
    float2 v[16];
    if (s1_thread) {
      const float2* PA = S + 2 * q * P::LDP;
      const float2* PB = PA + P::LDP;
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int k = j + Q * m;
        float2 A, B;
        if (k == 0) {
          A = make_float2(PA[0].x, 0.0f);
          B = make_float2(PB[0].x, 0.0f);
        } else if (k == NP) {
          A = make_float2(PA[0].y, 0.0f);
          B = make_float2(PB[0].y, 0.0f);
        } else if (k < NP) {
          A = PA[k];
          B = PB[k];
        } else {
          A = PA[N - k];
          B = PB[N - k];
          A.y = -A.y;
          B.y = -B.y;
        }
        v[m] = make_float2(A.x - B.y, A.y + B.x);
      }
    }
    __syncthreads();  // the plane has been read before the line buffer overwrites it
    if (s1_thread) {
      dft16<true>(v);
      float2* Sq = S + q * P::LDQ;
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) Sq[k1 * (Q + 1) + j] = k1 == 0 ? v[0] : cmulc(v[k1], __ldg(twx + j * k1));
    }
  }
  __syncthreads();
  {  // x inverse, stage 2: Q-point DFTs, rows (2q, 2q+1) of z to the row buffers (aliasing the lines)
    float2 w[2][Q];
#pragma unroll
    for (int round = 0; round < 2; ++round) {
      const int task = t + NT * round;
      const int q = task >> 4, k1 = task & 15;
#pragma unroll
      for (int j = 0; j < Q; ++j) w[round][j] = S[q * P::LDQ + k1 * (Q + 1) + j];
    }
    __syncthreads();  // every line has been read before the row buffers overwrite it
    float* Rre = reinterpret_cast<float*>(S);
    float* Rim = Rre + NP * P::LDF_I;
#pragma unroll
    for (int round = 0; round < 2; ++round) {
      const int task = t + NT * round;
      const int q = task >> 4, k1 = task & 15;
      Dft<float2, Q, true>::run(w[round]);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) {
        Rre[q * P::LDF_I + k1 + 16 * k2] = w[round][k2].x;
        Rim[q * P::LDF_I + k1 + 16 * k2] = w[round][k2].y;
      }
    }
  }
  __syncthreads();
  float* f0 = reinterpret_cast<float*>(a.f0) + foff;
  float* f2 = (MODE != FX_PLAIN) ? reinterpret_cast<float*>(a.f2) + foff : nullptr;
  const float alpha = (MODE == FX_PCG) ? float(a.st[load].alpha) : 0.0f;
  const float beta = (MODE == FX_PCG) ? float(a.st[load].beta) : 0.0f;
  // rows to global memory (16-byte accesses along each row) with the PCG updates; the x and p loads of
  // a batch of rows are issued before any of its stores, so that they are in flight together
  constexpr int IT = N / 16, B = IT < 4 ? IT : 4;
#pragma unroll
  for (int it0 = 0; it0 < IT; it0 += B) {
    [[maybe_unused]] float4 pv[B], xv[B];
    if constexpr (MODE == FX_PCG) {
#pragma unroll
      for (int b = 0; b < B; ++b) {
        if (it0 + b < IT) {
          const int task = t + NT * (it0 + b);
          const long long g = (long long)(task / (N / 4)) * N + 4 * (task % (N / 4));
          pv[b] = *reinterpret_cast<const float4*>(f2 + g);
          xv[b] = *reinterpret_cast<const float4*>(f0 + g);
        }
      }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      if (it0 + b >= IT) continue;
      const int task = t + NT * (it0 + b);
      const int row = task / (N / 4), x = 4 * (task % (N / 4));
      const float* R = reinterpret_cast<const float*>(S) + (row & 1) * NP * P::LDF_I + (row >> 1) * P::LDF_I + x;
      const float4 zv = *reinterpret_cast<const float4*>(R);
      const long long g = (long long)row * N + x;
      if (MODE == FX_PLAIN) {
        *reinterpret_cast<float4*>(f0 + g) = zv;
      } else if (MODE == FX_PCG_INIT) {
        *reinterpret_cast<float4*>(f2 + g) = zv;
      } else {
        const float4 p4 = pv[b], x4 = xv[b];
        *reinterpret_cast<float4*>(f0 + g) = make_float4(fmaf(alpha, p4.x, x4.x), fmaf(alpha, p4.y, x4.y),
                                                         fmaf(alpha, p4.z, x4.z), fmaf(alpha, p4.w, x4.w));
        *reinterpret_cast<float4*>(f2 + g) = make_float4(fmaf(beta, p4.x, zv.x), fmaf(beta, p4.y, zv.y),
                                                         fmaf(beta, p4.z, zv.z), fmaf(beta, p4.w, zv.w));
      }
    }
  }
  if (MODE != FX_PLAIN && a.st != nullptr) {
    // the last CTA over all planes and components finalises the iteration bookkeeping
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    double total;
    __syncthreads();
    if (finish_reduction(0.0, a.red.partial + (long long)load * a.red.max_blocks, a.red.count + load, nblk, bid,
                         red_sh, &total)) {
      if (threadIdx.x == 0) {
        PcgState& st = a.st[load];
        if (MODE == FX_PCG) st.iter += 1;
        if (st.state == ST_CONV) st.state = ST_DONE;
        else if (st.state == ST_FIN_MAX) st.state = ST_MAXIT;
      }
    }
  }
}

// Last axis (z) of FP32 3-D fields with nz = N = 16 Q (32, 64, 96, 128 or 256), 16 columns x NC components
// per CTA, with the block solve: the same 16 x Q split as the fused x-y passes.  Stage 1: 16-point
// DFTs of the stride-Q z subsequences read straight from the spectrum; stage 2, in place on every
// thread: (a) the Q-point DFTs of the 16 NC (k1, c) lines of each column, (b) the block solve and the
// Parseval sum at each wavevector kz = k1 + 16 k2, (c) the Q-point inverse DFTs with the conjugate
// twiddles; stage 3: 16-point inverse DFTs written straight back.  Shared memory is touched twice per
// direction instead of once per radix stage.  The symbol entries are read from L2 at the block
// solve: the grid runs the loads of one column group next to each other (load = blockIdx.x), so the
// slice comes from HBM once.
// Threads: 16 Q NC for stages 1 and 3, at least 256 (16 columns x 16 k1) for stage 2, a multiple of 32.
// Requires ny * nxh to be a multiple of 16 (no partial column groups).
template <int N, int NC>
__host__ __device__ constexpr int last_rs_threads() {
  return 16 * (N / 16) * NC > 256 ? (16 * (N / 16) * NC + 31) / 32 * 32 : 256;
}
template <int N, int NC>
__host__ __device__ constexpr size_t last_rs_smem() {
  return (size_t)NC * 16 * (N / 16) * 16 * sizeof(float2);
}

template <int N, int NC>
__global__ void __launch_bounds__(last_rs_threads<N, NC>(), 1152 / last_rs_threads<N, NC>() > 1 ? 1152 / last_rs_threads<N, NC>() : 1)
    fft_last_rs_kernel(FftArgs a) {
  constexpr int TCL = 16, Q = N / 16;
  constexpr int NT3 = last_rs_threads<N, NC>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  float2* S = reinterpret_cast<float2*>(smem_raw);  // S[c][k1][slot][t]: NC * 16 * Q * 16 complex
  const int load = blockIdx.x;
  if (!first_half_active(a.st, load)) return;
  float2* spec = reinterpret_cast<float2*>(a.spec) + (long long)load * a.load_stride_s;
  const long long Nh = a.d.Nh;
  const long long es = (long long)a.d.ny * a.d.nxh;
  const int nxh = a.d.nxh, half = a.d.nx / 2;
  const int cf0 = blockIdx.y * TCL;
  const float2* tw = reinterpret_cast<const float2*>(a.tw.z);
  const float* sym = reinterpret_cast<const float*>(a.sym);
  const int tid = threadIdx.x;
  if (tid < 16 * Q * NC) {  // stage 1: task (column t, subsequence j, component c)
    const int t = tid & 15, j = (tid >> 4) % Q, c = tid / (16 * Q);
    const int cf = cf0 + t;
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = spec[c * Nh + cf + (j + Q * m) * es];
    dft16<false>(v);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1)
      S[((c * 16 + k1) * Q + j) * TCL + t] = k1 == 0 ? v[0] : cmul(v[k1], __ldg(tw + j * k1));
  }
  __syncthreads();
  // stage 2, all threads, in place in S[c][k1][slot][t]: (a) the Q-point forward DFTs over the slot
  // index (j -> k2) of the 16 NC (k1, c) lines of each column; (b) the block solve z^ = K_hat^+ r^ / N
  // and the Parseval sum <r, z> at every (k1, k2) of the thread's column; (c) the Q-point inverse DFTs
  // (k2 -> j) with the conjugate twiddles W_N^(j k1) of the inverse split
  constexpr int UNITS = 16 * 16 * NC;  // (t, k1, c) lines of Q values
  auto line = [&](int w) { return S + ((w >> 4) * Q) * TCL + (w & 15); };  // w = (c * 16 + k1) * 16 + t
#pragma unroll
  for (int w = tid; w < UNITS; w += NT3) {
    float2* L = line(w);
    float2 z[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) z[j] = L[j * TCL];
    Dft<float2, Q, false>::run(z);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) L[k2 * TCL] = z[k2];
  }
  __syncthreads();
  DotAcc2 dot;
  const int t = tid & 15;  // NT3 is a multiple of 16: every point of this thread lies in column t
  {
    const int kx = (cf0 + t) % nxh;
    for (int pnt = tid; pnt < 16 * N; pnt += NT3) {
      const int k1 = (pnt >> 4) & 15, k2 = pnt >> 8;
      // the symbol entries of this wavevector, read from L2 where the loads of the column group meet
      // (the grid runs them next to each other): entry e at ks[e * Nh]
      const float* ks = sym + cf0 + t + (long long)(k1 + 16 * k2) * es;
      float2 r[NC], z[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) r[c] = S[((c * 16 + k1) * Q + k2) * TCL + t];
      // a real symmetric block scales the real and imaginary parts alike: packed FP32x2 products
      auto kk = [](float k) { return make_float2(k, k); };
      if constexpr (NC == 1) {
        z[0] = __fmul2_rn(kk(__ldg(ks)), r[0]);
      } else {
        const float2 k00 = kk(__ldg(ks)), k11 = kk(__ldg(ks + Nh)), k22 = kk(__ldg(ks + 2 * Nh));
        const float2 k12 = kk(__ldg(ks + 3 * Nh)), k02 = kk(__ldg(ks + 4 * Nh)), k01 = kk(__ldg(ks + 5 * Nh));
        z[0] = __ffma2_rn(k00, r[0], __ffma2_rn(k01, r[1], __fmul2_rn(k02, r[2])));
        z[1] = __ffma2_rn(k01, r[0], __ffma2_rn(k11, r[1], __fmul2_rn(k12, r[2])));
        z[2] = __ffma2_rn(k02, r[0], __ffma2_rn(k12, r[1], __fmul2_rn(k22, r[2])));
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        dot.add(r[c], z[c]);  // the column's Parseval weight is applied to the thread's sum below
        S[((c * 16 + k1) * Q + k2) * TCL + t] = z[c];
      }
    }
    if (kx != 0 && kx != half) dot.scale2();
  }
  __syncthreads();
#pragma unroll
  for (int w = tid; w < UNITS; w += NT3) {
    float2* L = line(w);
    const int k1 = (w >> 4) & 15;
    float2 z[Q];
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) z[k2] = L[k2 * TCL];
    Dft<float2, Q, true>::run(z);
    L[0] = z[0];
#pragma unroll
    for (int j = 1; j < Q; ++j) L[j * TCL] = cmulc(z[j], __ldg(tw + j * k1));
  }
  __syncthreads();
  if (tid < 16 * Q * NC) {  // stage 3: task (column t, subsequence j, component c): 16-point inverse DFT over k1
    const int tt = tid & 15, j = (tid >> 4) % Q, c = tid / (16 * Q);
    const int cff = cf0 + tt;
    float2 v[16];
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) v[kk] = S[((c * 16 + kk) * Q + j) * TCL + tt];
    dft16<true>(v);
#pragma unroll
    for (int m = 0; m < 16; ++m) spec[c * Nh + cff + (j + Q * m) * es] = v[m];
  }
  if (a.st != nullptr) {
    const double part = block_sum(dot.value(), red_sh);
    double total;
    if (finish_reduction(part, a.red.partial + (long long)load * a.red.max_blocks, a.red.count + load, gridDim.y,
                         blockIdx.y, red_sh, &total)) {
      if (threadIdx.x == 0) {
        PcgState& st = a.st[load];
        if (a.init) {
          st.rz = total;
          st.rz_init = total;
          if (st.bnorm2 < 0.0) st.bnorm2 = total;  // zero initial guess: <b, K_ref^+ b> = <r0, z0>
          st.tol2 = st.tol2_rel * st.bnorm2;
          st.alpha = 0.0;
          st.beta = 0.0;
          if (!isfinite(total)) st.state = ST_BREAK;
          else if (total <= st.tol2) st.state = ST_CONV;
        } else {
          st.beta = (st.rz > 0.0) ? total / st.rz : 0.0;
          if (a.red.hist != nullptr && st.iter < kHist) a.red.hist[((long long)load * 2 + 1) * kHist + st.iter] = st.beta;
          st.rz = total;
          if (!isfinite(total)) st.state = ST_BREAK;
          else if (total <= st.tol2) st.state = ST_CONV;
          else if (st.iter + 1 >= st.max_iter) st.state = ST_FIN_MAX;
        }
      }
    }
  }
}


// ------------------------------------------------------------------------------------------------
// Algorithm 2 tail: packed symbol, checks and per-wavevector inverse
// ------------------------------------------------------------------------------------------------
template <int NC>
__global__ void symbol_kernel(SymbolArgs a) {
  const long long Nh = a.d.Nh;
  const double2* sp = reinterpret_cast<const double2*>(a.spec);
  const double invN = 1.0 / (double)a.d.N;
  double mx_im = 0.0, mx_asym = 0.0, mx_abs = 0.0, mn_piv = 1e300;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < Nh; k += (long long)gridDim.x * blockDim.x) {
    double K[NC][NC];
#pragma unroll
    for (int al = 0; al < NC; ++al)
#pragma unroll
      for (int be = 0; be < NC; ++be) {
        const double2 v = sp[((long long)be * NC + al) * Nh + k];  // spectrum of comp alpha of K_ref i^beta
        K[al][be] = v.x;
        mx_im = fmax(mx_im, fabs(v.y));
        mx_abs = fmax(mx_abs, fabs(v.x));
      }
#pragma unroll
    for (int al = 0; al < NC; ++al)
#pragma unroll
      for (int be = al + 1; be < NC; ++be) {
        mx_asym = fmax(mx_asym, fabs(K[al][be] - K[be][al]));
        const double s = 0.5 * (K[al][be] + K[be][al]);
        K[al][be] = s;
        K[be][al] = s;
      }
    double inv[6] = {0, 0, 0, 0, 0, 0};  // packed (00, 11, 22, 12, 02, 01) / (00, 11, 01) / (00)
    if (k != 0) {
      if (NC == 1) {
        mn_piv = fmin(mn_piv, K[0][0]);
        inv[0] = 1.0 / K[0][0];
      } else if (NC == 2) {
        const double det = K[0][0] * K[1][1] - K[0][1] * K[0][1];
        mn_piv = fmin(mn_piv, fmin(K[0][0], det / K[0][0]));
        inv[0] = K[1][1] / det;
        inv[1] = K[0][0] / det;
        inv[2] = -K[0][1] / det;
      } else {
        const double A = K[0][0], B = K[1][1], Cc = K[2][2], D = K[1][2], E = K[0][2], F = K[0][1];
        const double c00 = B * Cc - D * D, c11 = A * Cc - E * E, c22 = A * B - F * F;
        const double c12 = E * F - A * D, c02 = D * F - B * E, c01 = D * E - Cc * F;
        const double det = A * c00 + F * c01 + E * c02;
        mn_piv = fmin(mn_piv, fmin(A, fmin(c22 / A, det / c22)));
        inv[0] = c00 / det; inv[1] = c11 / det; inv[2] = c22 / det;
        inv[3] = c12 / det; inv[4] = c02 / det; inv[5] = c01 / det;
      }
    }
    constexpr int NE_ = NC * (NC + 1) / 2;
#pragma unroll
    for (int e = 0; e < NE_; ++e) {
      a.sym64[e * Nh + k] = inv[e] * invN;
      if (a.sym32) a.sym32[e * Nh + k] = (float)(inv[e] * invN);
    }
  }
  // block maxima -> partials (host reduces)
  __shared__ double sh[4][256];
  sh[0][threadIdx.x] = mx_im;
  sh[1][threadIdx.x] = mx_asym;
  sh[2][threadIdx.x] = mx_abs;
  sh[3][threadIdx.x] = mn_piv;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][threadIdx.x + s]);
      sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + s]);
      sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + s]);
      sh[3][threadIdx.x] = fmin(sh[3][threadIdx.x], sh[3][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int i = 0; i < 4; ++i) a.partial[blockIdx.x * 4 + i] = sh[i][0];
}

// Two-node stencil: the 2 x 2 blocks are Hermitian (the centre node sits half a pixel off the corner
// grid, so the corner-centre coupling carries a phase).  Per k != 0 the regular inverse
// [[c, -b], [-conj b, a]] / (a c - |b|^2) of [[a, b], [conj b, c]]; k = 0 is set by the host.
// Packed (00, 11, Re 01, Im 01) / N.  Diagnostics: |Im| of the diagonal, |K01 - conj K10|.
__global__ void symbol_herm2_kernel(SymbolArgs a) {
  const long long Nh = a.d.Nh;
  const double2* sp = reinterpret_cast<const double2*>(a.spec);
  const double invN = 1.0 / (double)a.d.N;
  double mx_im = 0.0, mx_asym = 0.0, mx_abs = 0.0, mn_piv = 1e300;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < Nh; k += (long long)gridDim.x * blockDim.x) {
    const double2 k00 = sp[0 * Nh + k], k11 = sp[3 * Nh + k];
    const double2 k01 = sp[2 * Nh + k];  // component 0 of the response to the centre impulse
    const double2 k10 = sp[1 * Nh + k];  // component 1 of the response to the corner impulse
    mx_im = fmax(mx_im, fmax(fabs(k00.y), fabs(k11.y)));
    mx_asym = fmax(mx_asym, fmax(fabs(k01.x - k10.x), fabs(k01.y + k10.y)));
    mx_abs = fmax(mx_abs, fmax(fmax(fabs(k00.x), fabs(k11.x)), fmax(hypot(k01.x, k01.y), hypot(k10.x, k10.y))));
    const double A = k00.x, Cc = k11.x;
    const double bx = 0.5 * (k01.x + k10.x), by = 0.5 * (k01.y - k10.y);
    double inv[4] = {0, 0, 0, 0};
    if (k != 0) {
      const double det = A * Cc - (bx * bx + by * by);
      mn_piv = fmin(mn_piv, fmin(A, det / A));
      inv[0] = Cc / det;
      inv[1] = A / det;
      inv[2] = -bx / det;
      inv[3] = -by / det;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      a.sym64[e * Nh + k] = inv[e] * invN;
      if (a.sym32) a.sym32[e * Nh + k] = (float)(inv[e] * invN);
    }
  }
  __shared__ double sh[4][256];
  sh[0][threadIdx.x] = mx_im;
  sh[1][threadIdx.x] = mx_asym;
  sh[2][threadIdx.x] = mx_abs;
  sh[3][threadIdx.x] = mn_piv;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][threadIdx.x + s]);
      sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + s]);
      sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + s]);
      sh[3][threadIdx.x] = fmin(sh[3][threadIdx.x], sh[3][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int i = 0; i < 4; ++i) a.partial[blockIdx.x * 4 + i] = sh[i][0];
}

template <typename K>
cudaError_t set_smem(K kern, size_t bytes) {
  if (bytes > 32 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

constexpr size_t kSmemPair = 112 * 1024;  // two CTAs per SM
constexpr size_t kSmemMax = 200 * 1024;

// pairs of x lines per CTA: the planned value when it fits, else 8, or 4 when 8 does not fit
template <typename T> int x_pairs(const Dims& d, int planned) {
  using C = typename V2<T>::t;
  auto fits = [&](int P) { return 2ull * d.nx * (P + 1) * sizeof(C) <= 160 * 1024; };
  if ((planned == 4 || planned == 8 || planned == 16) && fits(planned)) return planned;
  return fits(8) ? 8 : 4;
}

// columns per CTA of a strided pass over nc components: the planned value when it fits, else
// 128-byte rows halved until two CTAs fit on an SM; 0 = no tile fits
template <typename T> int tile_cols(int L, int nc, int planned) {
  using C = typename V2<T>::t;
  auto bytes = [&](int TC) { return 2ull * L * nc * TC * sizeof(C); };
  if ((planned == 2 || planned == 4 || planned == 8 || planned == 16) && bytes(planned) <= kSmemMax) return planned;
  int TC = sizeof(T) == 4 ? 16 : 8;
  while (TC > 2 && bytes(TC) > kSmemPair) TC >>= 1;
  return bytes(TC) <= kSmemMax ? TC : 0;
}

template <typename K, typename... Args>
cudaError_t launch_with_smem(K kern, dim3 grid, int threads, size_t smem, cudaStream_t s, Args... args) {
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, smem, s>>>(args...);
  return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
template <typename T>
cudaError_t launch_fft_x_fwd(const FftArgs& a, cudaStream_t s) {
  using C = typename V2<T>::t;
  const int P = x_pairs<T>(a.d, a.pairs);
  const long long pairs = ((long long)a.d.ny * a.d.nz + 1) / 2;
  dim3 grid((unsigned)((pairs + P - 1) / P), a.d.c, a.n_loads);
  const size_t smem = 2ull * a.d.nx * (P + 1) * sizeof(C);
  const bool up = a.mode == FX_PCG;
  if (P == 16) return up ? launch_with_smem(fft_x_fwd_kernel<T, true, 16>, grid, XT, smem, s, a)
                         : launch_with_smem(fft_x_fwd_kernel<T, false, 16>, grid, XT, smem, s, a);
  if (P == 8) return up ? launch_with_smem(fft_x_fwd_kernel<T, true, 8>, grid, XT, smem, s, a)
                        : launch_with_smem(fft_x_fwd_kernel<T, false, 8>, grid, XT, smem, s, a);
  return up ? launch_with_smem(fft_x_fwd_kernel<T, true, 4>, grid, XT, smem, s, a)
            : launch_with_smem(fft_x_fwd_kernel<T, false, 4>, grid, XT, smem, s, a);
}

template <typename T>
cudaError_t launch_fft_x_inv(const FftArgs& a, cudaStream_t s) {
  using C = typename V2<T>::t;
  const int P = x_pairs<T>(a.d, a.pairs);
  const long long pairs = ((long long)a.d.ny * a.d.nz + 1) / 2;
  dim3 grid((unsigned)((pairs + P - 1) / P), a.d.c, a.n_loads);
  if (a.st != nullptr && (long long)grid.x * grid.y > a.red.max_blocks) return cudaErrorInvalidConfiguration;
  const size_t smem = 2ull * a.d.nx * (P + 1) * sizeof(C);
  if (P == 16) {
    if (a.mode == FX_PCG) return launch_with_smem(fft_x_inv_kernel<T, FX_PCG, 16>, grid, XT, smem, s, a);
    if (a.mode == FX_PCG_INIT) return launch_with_smem(fft_x_inv_kernel<T, FX_PCG_INIT, 16>, grid, XT, smem, s, a);
    return launch_with_smem(fft_x_inv_kernel<T, FX_PLAIN, 16>, grid, XT, smem, s, a);
  }
  if (P == 8) {
    if (a.mode == FX_PCG) return launch_with_smem(fft_x_inv_kernel<T, FX_PCG, 8>, grid, XT, smem, s, a);
    if (a.mode == FX_PCG_INIT) return launch_with_smem(fft_x_inv_kernel<T, FX_PCG_INIT, 8>, grid, XT, smem, s, a);
    return launch_with_smem(fft_x_inv_kernel<T, FX_PLAIN, 8>, grid, XT, smem, s, a);
  }
  if (a.mode == FX_PCG) return launch_with_smem(fft_x_inv_kernel<T, FX_PCG, 4>, grid, XT, smem, s, a);
  if (a.mode == FX_PCG_INIT) return launch_with_smem(fft_x_inv_kernel<T, FX_PCG_INIT, 4>, grid, XT, smem, s, a);
  return launch_with_smem(fft_x_inv_kernel<T, FX_PLAIN, 4>, grid, XT, smem, s, a);
}

template <typename T, bool INV>
static cudaError_t launch_strided_tc(const FftArgs& a, const ColMap& m, int TC, dim3 grid, size_t smem,
                                     const typename V2<T>::t* tw, cudaStream_t s) {
  switch (TC) {
    case 16: return launch_with_smem(fft_strided_kernel<T, INV, 16>, grid, ST, smem, s, a, m, tw);
    case 8: return launch_with_smem(fft_strided_kernel<T, INV, 8>, grid, ST, smem, s, a, m, tw);
    case 4: return launch_with_smem(fft_strided_kernel<T, INV, 4>, grid, ST, smem, s, a, m, tw);
    case 2: return launch_with_smem(fft_strided_kernel<T, INV, 2>, grid, ST, smem, s, a, m, tw);
    default: return cudaErrorInvalidConfiguration;
  }
}

template <typename T>
cudaError_t launch_fft_y(const FftArgs& a, int inverse, cudaStream_t s) {
  using C = typename V2<T>::t;
  // 3-D middle axis: columns (z, kx), element e = ky
  ColMap m{a.d.ny, a.d.nz * a.d.nxh, (long long)a.d.ny * a.d.nxh, (long long)a.d.nxh};
  const int TC = tile_cols<T>(m.L, 1, a.tc_y);
  if (TC == 0) return cudaErrorInvalidConfiguration;
  dim3 grid((m.ncols + TC - 1) / TC, a.d.c, a.n_loads);
  const size_t smem = 2ull * m.L * TC * sizeof(C);
  const C* tw = reinterpret_cast<const C*>(a.tw.y);
  return inverse ? launch_strided_tc<T, true>(a, m, TC, grid, smem, tw, s)
                 : launch_strided_tc<T, false>(a, m, TC, grid, smem, tw, s);
}

template <typename T, int NC, bool SOLVE>
static cudaError_t launch_last_tc(const FftArgs& a, const ColMap& m, int TC, dim3 grid, size_t smem,
                                  const typename V2<T>::t* tw, cudaStream_t s) {
  switch (TC) {
    case 16: return launch_with_smem(fft_last_kernel<T, NC, SOLVE, 16>, grid, ST, smem, s, a, m, tw);
    case 8: return launch_with_smem(fft_last_kernel<T, NC, SOLVE, 8>, grid, ST, smem, s, a, m, tw);
    case 4: return launch_with_smem(fft_last_kernel<T, NC, SOLVE, 4>, grid, ST, smem, s, a, m, tw);
    case 2: return launch_with_smem(fft_last_kernel<T, NC, SOLVE, 2>, grid, ST, smem, s, a, m, tw);
    default: return cudaErrorInvalidConfiguration;
  }
}

template <typename T, int NC>
static cudaError_t launch_last_nc(const FftArgs& a, cudaStream_t s) {
  using C = typename V2<T>::t;
  ColMap m;
  const C* tw;
  if (a.d.dim == 3) {
    m = ColMap{a.d.nz, a.d.ny * a.d.nxh, (long long)a.d.nxh, (long long)a.d.ny * a.d.nxh};
    tw = reinterpret_cast<const C*>(a.tw.z);
  } else {
    m = ColMap{a.d.ny, a.d.nxh, 0LL, (long long)a.d.nxh};
    tw = reinterpret_cast<const C*>(a.tw.y);
  }
  const int TC = tile_cols<T>(m.L, NC, a.tc_last);
  if (TC == 0) return cudaErrorInvalidConfiguration;
  dim3 grid((m.ncols + TC - 1) / TC, 1, a.n_loads);
  if (a.st != nullptr && (long long)grid.x > a.red.max_blocks) return cudaErrorInvalidConfiguration;
  const size_t smem = 2ull * m.L * NC * TC * sizeof(C);
  return a.sym ? launch_last_tc<T, NC, true>(a, m, TC, grid, smem, tw, s)
               : launch_last_tc<T, NC, false>(a, m, TC, grid, smem, tw, s);
}

static bool rs_length(int n) { return n == 32 || n == 64 || n == 96 || n == 128; }

bool fft_last_rs_supported(const Dims& d, bool fp32) {
  const bool len = rs_length(d.nz) || d.nz == 256;
  return fp32 && d.dim == 3 && len && (d.c == 1 || d.c == 3) && (d.ny * d.nxh) % 16 == 0;
}

template <int N>
static cudaError_t launch_last_rs(const FftArgs& a, dim3 grid, cudaStream_t s) {
  if (a.d.c == 1) return launch_with_smem(fft_last_rs_kernel<N, 1>, grid, last_rs_threads<N, 1>(), last_rs_smem<N, 1>(), s, a);
  return launch_with_smem(fft_last_rs_kernel<N, 3>, grid, last_rs_threads<N, 3>(), last_rs_smem<N, 3>(), s, a);
}

template <typename T>
cudaError_t launch_fft_last_solve(const FftArgs& a, cudaStream_t s) {
  if (sizeof(T) == 4 && a.last_reg && a.sym && fft_last_rs_supported(a.d, true)) {
    const int groups = (a.d.ny * a.d.nxh) / 16;
    if (groups > 65535) return cudaErrorInvalidConfiguration;
    const dim3 grid(a.n_loads, groups, 1);
    if (a.st != nullptr && (long long)groups > a.red.max_blocks) return cudaErrorInvalidConfiguration;
    switch (a.d.nz) {
      case 128: return launch_last_rs<128>(a, grid, s);
      case 96: return launch_last_rs<96>(a, grid, s);
      case 64: return launch_last_rs<64>(a, grid, s);
      case 32: return launch_last_rs<32>(a, grid, s);
      case 256: return launch_last_rs<256>(a, grid, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (a.d.c == 1) return launch_last_nc<T, 1>(a, s);
  if (a.d.c == 2) return launch_last_nc<T, 2>(a, s);
  if (a.d.c == 3) return launch_last_nc<T, 3>(a, s);
  return cudaErrorInvalidValue;
}

template <int N>
static cudaError_t launch_xy_rs(const FftArgs& a, int inverse, cudaStream_t s) {
  using P = RS<N>;
  const dim3 grid(a.d.nz, a.d.c, a.n_loads);
  if (!inverse && a.mode == FX_PCG) return launch_with_smem(fft_xy_fwd_rs_kernel<N, true>, grid, P::NT, P::SMEM, s, a);
  if (!inverse) return launch_with_smem(fft_xy_fwd_rs_kernel<N, false>, grid, P::NT, P::SMEM, s, a);
  if (a.st != nullptr && (long long)grid.x * grid.y > a.red.max_blocks) return cudaErrorInvalidConfiguration;
  if (a.mode == FX_PCG) return launch_with_smem(fft_xy_inv_rs_kernel<N, FX_PCG>, grid, P::NT, P::SMEM, s, a);
  if (a.mode == FX_PCG_INIT) return launch_with_smem(fft_xy_inv_rs_kernel<N, FX_PCG_INIT>, grid, P::NT, P::SMEM, s, a);
  return launch_with_smem(fft_xy_inv_rs_kernel<N, FX_PLAIN>, grid, P::NT, P::SMEM, s, a);
}

template <>
cudaError_t launch_fft_xy<float>(const FftArgs& a, int inverse, cudaStream_t s) {
  if (!fft_xy_supported(a.d, true)) return cudaErrorInvalidValue;
  switch (a.d.nx) {
    case 128: return launch_xy_rs<128>(a, inverse, s);
    case 96: return launch_xy_rs<96>(a, inverse, s);
    case 64: return launch_xy_rs<64>(a, inverse, s);
    case 32: return launch_xy_rs<32>(a, inverse, s);
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_fft_xy<double>(const FftArgs&, int, cudaStream_t) {
  return cudaErrorInvalidValue;
}

bool fft_xy_supported(const Dims& d, bool fp32) {
  return fp32 && d.dim == 3 && rs_length(d.nx) && d.ny == d.nx && d.nxh == d.nx / 2 + 1;
}

template cudaError_t launch_fft_x_fwd<double>(const FftArgs&, cudaStream_t);
template cudaError_t launch_fft_x_fwd<float>(const FftArgs&, cudaStream_t);
template cudaError_t launch_fft_x_inv<double>(const FftArgs&, cudaStream_t);
template cudaError_t launch_fft_x_inv<float>(const FftArgs&, cudaStream_t);
template cudaError_t launch_fft_y<double>(const FftArgs&, int, cudaStream_t);
template cudaError_t launch_fft_y<float>(const FftArgs&, int, cudaStream_t);
template cudaError_t launch_fft_last_solve<double>(const FftArgs&, cudaStream_t);
template cudaError_t launch_fft_last_solve<float>(const FftArgs&, cudaStream_t);

cudaError_t launch_symbol_build(const SymbolArgs& a, int* blocks_out, cudaStream_t s) {
  const int blocks = (int)std::min<long long>(2 * 152, (a.d.Nh + 255) / 256);
  *blocks_out = blocks;
  if (a.herm) symbol_herm2_kernel<<<blocks, 256, 0, s>>>(a);
  else if (a.d.c == 1) symbol_kernel<1><<<blocks, 256, 0, s>>>(a);
  else if (a.d.c == 2) symbol_kernel<2><<<blocks, 256, 0, s>>>(a);
  else symbol_kernel<3><<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// W_L^m = exp(-2 pi i m / L), m = 0..L-1, from cos/sin of the first octant in long double.
cudaError_t make_twiddles(int L, double2** d64, float2** d32) {
  std::vector<double2> h64(L);
  std::vector<float2> h32(L);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int m = 0; m < L; ++m) {
    // angle = 2 pi m / L reduced to [0, pi/4] by octant symmetry: exact at multiples of L/8
    long long num = (long long)m * 8;  // angle in units of (2 pi / (8 L)) * 8 = octants * L
    const int oct = (int)(num / L);    // 0..7
    long long rem = num - (long long)oct * L;  // 0..L-1, angle within the octant = (2 pi / 8) * rem / L
    // within-octant angle phi in [0, pi/4); use the reflected angle on odd octants
    long double phi = two_pi / 8.0L * (long double)rem / (long double)L;
    long double c = cosl(phi), sn = sinl(phi);
    long double cr = cosl(two_pi / 8.0L - phi), sr = sinl(two_pi / 8.0L - phi);
    long double cosv = 0, sinv = 0;
    switch (oct) {  // theta = oct * pi/4 + phi
      case 0: cosv = c; sinv = sn; break;
      case 1: cosv = sr; sinv = cr; break;          // theta = pi/2 - (pi/4 - phi)
      case 2: cosv = -sn; sinv = c; break;          // theta = pi/2 + phi
      case 3: cosv = -cr; sinv = sr; break;         // theta = pi - (pi/4 - phi)
      case 4: cosv = -c; sinv = -sn; break;         // theta = pi + phi
      case 5: cosv = -sr; sinv = -cr; break;        // theta = 3pi/2 - (pi/4 - phi)
      case 6: cosv = sn; sinv = -c; break;          // theta = 3pi/2 + phi
      default: cosv = cr; sinv = -sr; break;        // theta = 2pi - (pi/4 - phi)
    }
    h64[m] = make_double2((double)cosv, (double)(-sinv));
    h32[m] = make_float2((float)cosv, (float)(-sinv));
  }
  cudaError_t e = cudaMalloc(d64, sizeof(double2) * L);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(d32, sizeof(float2) * L);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(*d64, h64.data(), sizeof(double2) * L, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*d32, h32.data(), sizeof(float2) * L, cudaMemcpyHostToDevice);
}

}  // namespace fehom
