// Learned warm start: the periodic 3-D U-Net of fehom_unet.h, trained and evaluated on the GPU.
//
// The 3x3x3 convolutions are implicit GEMMs on the tcgen05 tensor cores (BF16 operands, FP32
// accumulators in tensor memory):
//   * conv3_tc_kernel (forward, and input gradient through flipped/transposed weights): one CTA
//     computes ZT (1, 2 or 4) output planes of a 16 x 8 (y, x) tile; each plane is the M = 128 rows
//     of its own MMAs and accumulator, N = up to 64 output channels.  Per 16-channel slice of the
//     input it stages the periodic halo ((ZT + 2) x 18 x 10 voxels) and the slice's weights once in
//     shared memory in the no-swizzle K-major core-matrix layout; each of the 27 taps of each plane
//     is then the same halo read through a shifted matrix descriptor (the 8 x-voxels of a core
//     matrix row are contiguous in the halo), so the taps cost no data movement.
//   * wgrad_tc_kernel (weight gradient): M = 128 rows = output channels (zero-padded), N = 16 input
//     channels, K = voxels of a tile; three x-shifted copies of the halo keep every tap a shifted
//     descriptor; the 27 taps accumulate in 27 x 16 TMEM columns across the CTA's tiles.
// Everything else (first layer with one input channel, pooling, upsampling/concatenation and their
// adjoints, ReLU masks, head and loss, bias sums, Adam) runs on CUDA cores.  Reductions are
// block partials summed in a fixed order, so results are deterministic.
//
// Every wait on an mbarrier is bounded (2 s of the global timer); a timeout sets the network's
// error flag, frees tensor memory and returns.
#include "../../include/fehom_unet.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace fehom_unet_impl {
namespace {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------------------------------------
// tcgen05, mbarrier and proxy-fence wrappers
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the completion of the phase with the given parity; false after 2 s.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  while (!mbar_test(bar, parity)) {
    if (global_ns() - t0 > 2000000000ull) return false;
    __nanosleep(32);
  }
  return true;
}

// Shared-memory matrix descriptor, no swizzle: start address, leading-dimension byte offset (between
// core matrices along K), stride-dimension byte offset (between 8-row groups along M or N), all >> 4;
// bit 46 = descriptor version of tcgen05.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 lanes x 16 columns of FP32 from tensor memory (this warp's lane quarter), waited in the same asm.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

__device__ __forceinline__ void unpack8(const uint4& u, float (&f)[8]) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 p = __bfloat1622float2(h[i]);
    f[2 * i] = p.x;
    f[2 * i + 1] = p.y;
  }
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
  uint4 u;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
  return u;
}

// ------------------------------------------------------------------------------------------------
// tensor-core 3x3x3 periodic convolution (forward / input gradient)
// ------------------------------------------------------------------------------------------------
struct ConvArgs {
  const bf16* x;      // [B][D][H][W][Cin]
  const bf16* w;      // [27][Cout][Cin]
  const float* bias;  // [Cout] or null
  const bf16* mask;   // [B][D][H][W][Cout] or null: output *= (mask > 0)
  bf16* y;            // [B][D][H][W][Cout] (bf16) or null
  float* y32;         // [B][D][H][W][Cout] (fp32) or null
  int D, H, W, Cin, Cout, relu;
  int* err;
};

constexpr int kHaloVox = 3 * 18 * 10;            // z-1..z+1, y0-1..y0+16, x0-1..x0+8 (one output plane)
constexpr int kPlaneVox = 18 * 10;
template <int ZT>
__host__ __device__ constexpr int conv_halo_vox() { return (ZT + 2) * kPlaneVox; }
template <int NT, int ZT>
__host__ __device__ constexpr int conv_stage_bytes() { return 2 * conv_halo_vox<ZT>() * 16 + 27 * NT * 32; }
template <int NT, int ZT>
__host__ __device__ constexpr int conv_smem_bytes() { return 2 * conv_stage_bytes<NT, ZT>() + 32; }
template <int NT, int ZT>
__host__ __device__ constexpr uint32_t conv_tmem_cols() {
  return NT * ZT <= 32 ? 32 : NT * ZT <= 64 ? 64 : NT * ZT <= 128 ? 128 : 256;
}

// One CTA: ZT consecutive output planes of a 16 x 8 (y, x) tile, NT output channels.  The weights of
// a 16-channel input slice are staged once and serve all ZT planes (ZT accumulators in TMEM).
template <int NT, int ZT>
__global__ void __launch_bounds__(128, 1) conv3_tc_kernel(ConvArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr int HV = conv_halo_vox<ZT>();
  constexpr int ABYTES = 2 * HV * 16;
  constexpr int STAGE = conv_stage_bytes<NT, ZT>();
  constexpr uint32_t NCOLS = conv_tmem_cols<NT, ZT>();
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * STAGE);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + 2 * STAGE + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tiles_x = (a.W + 7) >> 3;
  const int x0 = (blockIdx.x % tiles_x) * 8, y0 = (blockIdx.x / tiles_x) * 16;
  const int z0 = blockIdx.y * ZT;
  const int ntn = a.Cout / NT;
  const int b = blockIdx.z / ntn, n0 = (blockIdx.z % ntn) * NT;
  const long long V = static_cast<long long>(a.D) * a.H * a.W;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(slot, NCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  const bf16* xb = a.x + b * V * a.Cin;
  auto load_stage = [&](int kc, int s) {
    uint8_t* As = smem + s * STAGE;
    uint8_t* Bs = As + ABYTES;
    for (int idx = tid; idx < 2 * HV; idx += 128) {
      const int half = idx >= HV ? 1 : 0, h = idx - half * HV;
      const int zz = h / kPlaneVox, ry = (h % kPlaneVox) / 10, rx = h % 10;
      const int zi = wrapi(z0 + zz - 1, a.D), yi = wrapi(y0 + ry - 1, a.H), xi = wrapi(x0 + rx - 1, a.W);
      const uint4 v = *reinterpret_cast<const uint4*>(
          xb + ((static_cast<long long>(zi) * a.H + yi) * a.W + xi) * a.Cin + kc * 16 + half * 8);
      *reinterpret_cast<uint4*>(As + half * (HV * 16) + h * 16) = v;
    }
    for (int idx = tid; idx < 27 * NT * 2; idx += 128) {
      const int half = idx & 1, co = (idx >> 1) % NT, tap = (idx >> 1) / NT;
      const uint4 v = *reinterpret_cast<const uint4*>(a.w + (static_cast<long long>(tap) * a.Cout + n0 + co) * a.Cin +
                                                      kc * 16 + half * 8);
      *reinterpret_cast<uint4*>(Bs + tap * (NT * 32) + half * (NT * 16) + co * 16) = v;
    }
  };
  const uint32_t idesc = idesc_bf16(128, NT);
  auto issue = [&](int kc, int s) {
    const uint32_t As = smem_u32(smem + s * STAGE), Bs = As + ABYTES;
    tc_fence_after();
    for (int t = 0; t < 27; ++t) {
      const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;  // offsets + 1
      // B: rows = output channels (SBO 128 B per 8 rows), K halves NT * 16 bytes apart
      const uint64_t bd = smem_desc(Bs + t * (NT * 32), NT * 16, 128);
#pragma unroll
      for (int zz = 0; zz < ZT; ++zz) {
        // A: rows = 16 output lines of plane zz (SBO = one halo row, 10 voxels), K halves HV voxels apart
        const uint64_t ad = smem_desc(As + ((zz + dz) * kPlaneVox + dy * 10 + dx) * 16, HV * 16, 160);
        mma_bf16(tmem + zz * NT, ad, bd, idesc, (kc > 0 || t > 0) ? 1u : 0u);
      }
    }
    mma_commit(&bar[s]);
  };

  const int nk = a.Cin / 16;
  load_stage(0, 0);
  fence_proxy_async();
  __syncthreads();
  bool ok = true;
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc & 1;
    if (tid == 0) issue(kc, s);
    if (kc + 1 < nk) {
      if (kc >= 1) ok = mbar_wait(&bar[s ^ 1], ((kc - 1) >> 1) & 1);  // MMAs of chunk kc-1 read buffer s^1
      ok = __syncthreads_and(ok);
      if (!ok) break;
      load_stage(kc + 1, s ^ 1);
      fence_proxy_async();
    }
    __syncthreads();
  }
  if (ok) ok = mbar_wait(&bar[(nk - 1) & 1], ((nk - 1) >> 1) & 1);
  ok = __syncthreads_and(ok);
  if (ok) {
    tc_fence_after();
    const int ty = tid >> 3, tx = tid & 7;
    const int yy = y0 + ty, xx = x0 + tx;
    const bool valid = yy < a.H && xx < a.W;
    for (int zz = 0; zz < ZT; ++zz) {
      const long long vox =
          b * V + (static_cast<long long>(z0 + zz) * a.H + (valid ? yy : 0)) * a.W + (valid ? xx : 0);
      for (int c0 = 0; c0 < NT; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + zz * NT + c0, v);
        if (!valid) continue;
        const int n = n0 + c0;
        if (a.bias) {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] += a.bias[n + j];
        }
        if (a.relu) {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.0f);
        }
        if (a.mask) {
          const uint4* mp = reinterpret_cast<const uint4*>(a.mask + vox * a.Cout + n);
          for (int h = 0; h < 2; ++h) {
            float mk[8];
            unpack8(mp[h], mk);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[8 * h + j] = mk[j] > 0.0f ? v[8 * h + j] : 0.0f;
          }
        }
        if (a.y32) {
          float4* yp = reinterpret_cast<float4*>(a.y32 + vox * a.Cout + n);
#pragma unroll
          for (int q = 0; q < 4; ++q) yp[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
          uint4* yp = reinterpret_cast<uint4*>(a.y + vox * a.Cout + n);
          for (int h = 0; h < 2; ++h) {
            float f[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) f[j] = v[8 * h + j];
            yp[h] = pack8(f);
          }
        }
      }
    }
  } else if (tid == 0 && a.err) {
    atomicExch(a.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// ------------------------------------------------------------------------------------------------
// tensor-core weight gradient
// ------------------------------------------------------------------------------------------------
struct WgradArgs {
  const bf16* x;   // [B][D][H][W][Cin]
  const bf16* dy;  // [B][D][H][W][Cout]
  float* partial;  // [gridDim.x][27][Cout][Cin]
  int D, H, W, Cin, Cout;
  int n_tiles, tiles_per_cta;
  int* err;
};

constexpr int kWgA = 16 * 128 * 16;   // [line 16][row (output channel) 128][8 x] bf16
constexpr int kWgCopy = 54 * 16 * 16;  // [line (zz, ry) 54][input channel 16][8 x] bf16
constexpr int kWgStage = kWgA + 3 * kWgCopy;
constexpr int kWgSmem = 2 * kWgStage + 32;

__global__ void __launch_bounds__(128, 1) wgrad_tc_kernel(WgradArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * kWgStage);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + 2 * kWgStage + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int kc = blockIdx.y;
  const int t_begin = blockIdx.x * a.tiles_per_cta;
  const int t_end = min(a.n_tiles, t_begin + a.tiles_per_cta);
  const int tiles_x = (a.W + 7) >> 3, tiles_y = (a.H + 15) >> 4;
  const long long V = static_cast<long long>(a.D) * a.H * a.W;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  // rows >= Cout of the A tiles stay zero
  for (int i = tid; i < 2 * kWgStage / 16; i += 128) {
    const int s = i / (kWgStage / 16), r = i % (kWgStage / 16);
    if (r < kWgA / 16) reinterpret_cast<uint4*>(smem + s * kWgStage)[r] = make_uint4(0, 0, 0, 0);
  }
  if (warp == 0) {
    tmem_alloc(slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  // 8 x 8 transpose of bf16: in[x] holds channels 0..7 of voxel x; out[c] holds voxels 0..7 of channel c
  auto transpose8 = [](const uint4 (&in)[8], uint4 (&out)[8]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t w[8] = {(&in[0].x)[k], (&in[1].x)[k], (&in[2].x)[k], (&in[3].x)[k],
                             (&in[4].x)[k], (&in[5].x)[k], (&in[6].x)[k], (&in[7].x)[k]};
      out[2 * k] = make_uint4(__byte_perm(w[0], w[1], 0x5410), __byte_perm(w[2], w[3], 0x5410),
                              __byte_perm(w[4], w[5], 0x5410), __byte_perm(w[6], w[7], 0x5410));
      out[2 * k + 1] = make_uint4(__byte_perm(w[0], w[1], 0x7632), __byte_perm(w[2], w[3], 0x7632),
                                  __byte_perm(w[4], w[5], 0x7632), __byte_perm(w[6], w[7], 0x7632));
    }
  };
  auto load_tile = [&](int tile, int s) {
    uint8_t* As = smem + s * kWgStage;
    uint8_t* Bs = As + kWgA;
    int r = tile;
    const int txi = r % tiles_x;
    r /= tiles_x;
    const int tyi = r % tiles_y;
    r /= tiles_y;
    const int z = r % a.D, b = r / a.D;
    const int x0 = txi * 8, y0 = tyi * 16;
    const int cg8 = a.Cout >> 3;
    // A: per (line ty, 8 output channels) the 8 voxels of the line, transposed to [channel][8 x]
    for (int task = tid; task < 16 * cg8; task += 128) {
      const int ty = task / cg8, cg = task - ty * cg8;
      const int yy = y0 + ty;
      uint4 in[8], out[8];
#pragma unroll
      for (int tx = 0; tx < 8; ++tx) {
        const int xx = x0 + tx;
        in[tx] = make_uint4(0, 0, 0, 0);  // duplicate (wrapped) positions contribute nothing
        if (yy < a.H && xx < a.W)
          in[tx] = *reinterpret_cast<const uint4*>(a.dy + (b * V + (static_cast<long long>(z) * a.H + yy) * a.W + xx) *
                                                   a.Cout + cg * 8);
      }
      transpose8(in, out);
#pragma unroll
      for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4*>(As + ty * 2048 + (cg * 8 + c) * 16) = out[c];
    }
    // B: per (halo line (zz, ry), 8 input channels) the 10 voxels rx = 0..9 of the line; copy c (shift
    // dx = c - 1) holds rx = c .. c + 7, transposed to [channel][8 x]
    const bf16* xb = a.x + b * V * a.Cin + kc * 16;
    for (int task = tid; task < 54 * 2; task += 128) {
      const int line = task >> 1, half = task & 1;
      const int zz = line / 18, ry = line - zz * 18;
      const int zi = wrapi(z + zz - 1, a.D), yi = wrapi(y0 + ry - 1, a.H);
      const bf16* row = xb + (static_cast<long long>(zi) * a.H + yi) * a.W * a.Cin + half * 8;
      uint4 v[10];
#pragma unroll
      for (int rx = 0; rx < 10; ++rx)
        v[rx] = *reinterpret_cast<const uint4*>(row + static_cast<long long>(wrapi(x0 + rx - 1, a.W)) * a.Cin);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        uint4 in[8], out[8];
#pragma unroll
        for (int xp = 0; xp < 8; ++xp) in[xp] = v[xp + c];
        transpose8(in, out);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          *reinterpret_cast<uint4*>(Bs + c * kWgCopy + line * 256 + (half * 8 + j) * 16) = out[j];
      }
    }
  };
  const uint32_t idesc = idesc_bf16(128, 16);
  auto issue = [&](bool first, int s) {
    const uint32_t As = smem_u32(smem + s * kWgStage), Bs = As + kWgA;
    tc_fence_after();
    for (int ks = 0; ks < 8; ++ks) {
      // A: K chunks = output lines 2ks, 2ks+1 (LBO one line = 2048 B), rows = channels (SBO 128 B)
      const uint64_t ad = smem_desc(As + 2 * ks * 2048, 2048, 128);
      for (int t = 0; t < 27; ++t) {
        const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
        // B: halo line (dz, 2ks + dy) of the dx-shifted copy; K chunks one line apart (256 B)
        const uint64_t bd = smem_desc(Bs + dx * kWgCopy + (dz * 18 + 2 * ks + dy) * 256, 256, 128);
        mma_bf16(tmem + t * 16, ad, bd, idesc, (first && ks == 0) ? 0u : 1u);
      }
    }
    mma_commit(&bar[s]);
  };

  bool ok = true;
  const int nt = t_end - t_begin;
  if (nt > 0) {
    load_tile(t_begin, 0);
    fence_proxy_async();
    __syncthreads();
    for (int j = 0; j < nt; ++j) {
      const int s = j & 1;
      if (tid == 0) issue(j == 0, s);
      if (j + 1 < nt) {
        if (j >= 1) ok = mbar_wait(&bar[s ^ 1], ((j - 1) >> 1) & 1);
        ok = __syncthreads_and(ok);
        if (!ok) break;
        load_tile(t_begin + j + 1, s ^ 1);
        fence_proxy_async();
      }
      __syncthreads();
    }
    if (ok) ok = mbar_wait(&bar[(nt - 1) & 1], ((nt - 1) >> 1) & 1);
    ok = __syncthreads_and(ok);
  }
  const int co = tid;
  float* out = a.partial + static_cast<long long>(blockIdx.x) * 27 * a.Cout * a.Cin + kc * 16;
  if (ok && nt > 0) {
    tc_fence_after();
    for (int t = 0; t < 27; ++t) {
      float v[16];
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + t * 16, v);
      if (co < a.Cout) {
        float4* p = reinterpret_cast<float4*>(out + (static_cast<long long>(t) * a.Cout + co) * a.Cin);
#pragma unroll
        for (int q = 0; q < 4; ++q) p[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
    }
  } else {
    if (co < a.Cout)
      for (int t = 0; t < 27; ++t) {
        float4* p = reinterpret_cast<float4*>(out + (static_cast<long long>(t) * a.Cout + co) * a.Cin);
        for (int q = 0; q < 4; ++q) p[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    if (!ok && tid == 0 && a.err) atomicExch(a.err, 2);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// out[i] (+)= sum_p partial[p * len + i], p ascending
__global__ void reduce_partials_kernel(const float* __restrict__ partial, int P, long long len, float* out,
                                       int accumulate) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < len;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    float s = 0.0f;
    for (int p = 0; p < P; ++p) s += partial[p * len + i];
    out[i] = accumulate ? out[i] + s : s;
  }
}

// ------------------------------------------------------------------------------------------------
// CUDA-core kernels
// ------------------------------------------------------------------------------------------------
// First layer (one input channel = per-phase feature): y = relu(b + sum_t W[t][o] f(v + off_t))
__global__ void conv_in_kernel(const uint8_t* __restrict__ ids, const float* __restrict__ feat, int n_phases,
                               const float* __restrict__ w, const float* __restrict__ bias, bf16* __restrict__ y, int D,
                               int H, int W, int Cout, long long total) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= total) return;
  const long long V = static_cast<long long>(D) * H * W;
  const long long b = i / V, v = i % V;
  const int x = static_cast<int>(v % W), yq = static_cast<int>((v / W) % H), z = static_cast<int>(v / (static_cast<long long>(W) * H));
  float f[27];
  for (int t = 0; t < 27; ++t) {
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const long long vv = (static_cast<long long>(wrapi(z + dz, D)) * H + wrapi(yq + dy, H)) * W + wrapi(x + dx, W);
    f[t] = feat[b * n_phases + ids[b * V + vv]];
  }
  for (int c0 = 0; c0 < Cout; c0 += 8) {
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = bias[c0 + j];
    for (int t = 0; t < 27; ++t)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = fmaf(w[t * Cout + c0 + j], f[t], acc[j]);
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = fmaxf(acc[j], 0.0f);
    *reinterpret_cast<uint4*>(y + i * Cout + c0) = pack8(acc);
  }
}

// partial[block][t][o] = sum over the block's (b, z) plane of f(v + off_t) g[v][o]; t = 27: sum of g
__global__ void conv_in_wgrad_kernel(const uint8_t* __restrict__ ids, const float* __restrict__ feat, int n_phases,
                                     const bf16* __restrict__ g, float* partial, int D, int H, int W, int Cout) {
  extern __shared__ float sm[];
  float* fs = sm;            // [9][W]
  float* gs = sm + 9 * W;    // [W][Cout]
  const int b = blockIdx.x / D, z = blockIdx.x % D;
  const long long V = static_cast<long long>(D) * H * W;
  const int tid = threadIdx.x, t = tid / Cout, co = tid % Cout;
  float acc = 0.0f;
  for (int yy = 0; yy < H; ++yy) {
    __syncthreads();
    for (int i = tid; i < 9 * W; i += blockDim.x) {
      const int r = i / W, x = i % W, dz = r / 3 - 1, dy = r % 3 - 1;
      fs[i] = feat[b * n_phases + ids[b * V + (static_cast<long long>(wrapi(z + dz, D)) * H + wrapi(yy + dy, H)) * W + x]];
    }
    const bf16* gr = g + (b * V + (static_cast<long long>(z) * H + yy) * W) * Cout;
    for (int i = tid; i < W * Cout; i += blockDim.x) gs[i] = __bfloat162float(gr[i]);
    __syncthreads();
    if (t < 27) {
      const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3 - 1;
      const float* fr = fs + (dz * 3 + dy) * W;
      for (int x = 0; x < W; ++x) acc = fmaf(fr[wrapi(x + dx, W)], gs[x * Cout + co], acc);
    } else if (t == 27) {
      for (int x = 0; x < W; ++x) acc += gs[x * Cout + co];
    }
  }
  if (t <= 27) partial[static_cast<long long>(blockIdx.x) * 28 * Cout + t * Cout + co] = acc;
}

// partial[block][c] = sum of g[v][c] over the block's voxel range (bias gradient)
__global__ void chansum_kernel(const bf16* __restrict__ g, long long rows, int C, int rows_per_block, float* partial) {
  extern __shared__ float red[];
  const int lanes = blockDim.x / C, tid = threadIdx.x, c = tid % C, vl = tid / C;
  const long long r0 = static_cast<long long>(blockIdx.x) * rows_per_block;
  const long long r1 = min(rows, r0 + rows_per_block);
  float acc = 0.0f;
  if (vl < lanes)
    for (long long r = r0 + vl; r < r1; r += lanes) acc += __bfloat162float(g[r * C + c]);
  red[tid] = acc;
  __syncthreads();
  if (tid < C) {
    float s = 0.0f;
    for (int l = 0; l < lanes; ++l) s += red[l * C + tid];
    partial[static_cast<long long>(blockIdx.x) * C + tid] = s;
  }
}

__device__ __forceinline__ long long child_index(long long u, int Dc, int Hc, int Wc, int a, int bb, int cc) {
  const int ux = static_cast<int>(u % Wc), uy = static_cast<int>((u / Wc) % Hc), uz = static_cast<int>(u / (static_cast<long long>(Wc) * Hc));
  return (static_cast<long long>(2 * uz + a) * (2 * Hc) + (2 * uy + bb)) * (2 * Wc) + (2 * ux + cc);
}
__device__ __forceinline__ long long parent_index(long long v, int D, int H, int W) {
  const int x = static_cast<int>(v % W), y = static_cast<int>((v / W) % H), z = static_cast<int>(v / (static_cast<long long>(W) * H));
  return (static_cast<long long>(z >> 1) * (H >> 1) + (y >> 1)) * (W >> 1) + (x >> 1);
}

// p[b][u][c] = mean of the 8 children of coarse voxel u (fine grid 2Dc x 2Hc x 2Wc)
__global__ void pool_kernel(const bf16* __restrict__ e, bf16* __restrict__ p, int Dc, int Hc, int Wc, int C,
                            long long total) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= total) return;
  const int cgn = C >> 3;
  const int cg = static_cast<int>(i % cgn);
  const long long bu = i / cgn;
  const long long Vc = static_cast<long long>(Dc) * Hc * Wc;
  const long long b = bu / Vc, u = bu % Vc;
  float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < 8; ++k) {
    const long long v = child_index(u, Dc, Hc, Wc, k >> 2, (k >> 1) & 1, k & 1);
    float f[8];
    unpack8(*reinterpret_cast<const uint4*>(e + (b * 8 * Vc + v) * C + cg * 8), f);
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j] += f[j];
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) s[j] *= 0.125f;
  *reinterpret_cast<uint4*>(p + bu * C + cg * 8) = pack8(s);
}

// cat[b][v] = (skip[b][v][0:Cs], src[b][parent(v)][0:Cu])
__global__ void upcat_kernel(const bf16* __restrict__ skip, const bf16* __restrict__ src, bf16* __restrict__ cat,
                             int D, int H, int W, int Cs, int Cu, long long total) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= total) return;
  const int Ct = Cs + Cu, cgn = Ct >> 3;
  const int cg = static_cast<int>(i % cgn);
  const long long bv = i / cgn;
  const long long V = static_cast<long long>(D) * H * W;
  const long long b = bv / V, v = bv % V;
  uint4 val;
  if (cg * 8 < Cs) {
    val = *reinterpret_cast<const uint4*>(skip + bv * Cs + cg * 8);
  } else {
    const long long u = parent_index(v, D, H, W);
    val = *reinterpret_cast<const uint4*>(src + (b * (V >> 3) + u) * Cu + (cg * 8 - Cs));
  }
  *reinterpret_cast<uint4*>(cat + bv * Ct + cg * 8) = val;
}

// g[b][v][c] = (dcat[b][v][c] + dp[b][parent(v)][c] / 8) * (e[b][v][c] > 0), c < C (skip part of dcat)
__global__ void enc_grad_kernel(const bf16* __restrict__ dcat, int Ct, const bf16* __restrict__ dp,
                                const bf16* __restrict__ e, bf16* __restrict__ g, int D, int H, int W, int C,
                                long long total) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= total) return;
  const int cgn = C >> 3;
  const int cg = static_cast<int>(i % cgn);
  const long long bv = i / cgn;
  const long long V = static_cast<long long>(D) * H * W;
  const long long b = bv / V, v = bv % V;
  float a[8], p[8], m[8];
  unpack8(*reinterpret_cast<const uint4*>(dcat + bv * Ct + cg * 8), a);
  unpack8(*reinterpret_cast<const uint4*>(dp + (b * (V >> 3) + parent_index(v, D, H, W)) * C + cg * 8), p);
  unpack8(*reinterpret_cast<const uint4*>(e + bv * C + cg * 8), m);
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = m[j] > 0.0f ? a[j] + 0.125f * p[j] : 0.0f;
  *reinterpret_cast<uint4*>(g + bv * C + cg * 8) = pack8(a);
}

// g[b][u][c] = (sum over the 8 children v of dcat[b][v][Cs + c]) * (src[b][u][c] > 0)
__global__ void up_grad_kernel(const bf16* __restrict__ dcat, int Cs, int Cu, const bf16* __restrict__ src,
                               bf16* __restrict__ g, int Dc, int Hc, int Wc, long long total) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= total) return;
  const int cgn = Cu >> 3, Ct = Cs + Cu;
  const int cg = static_cast<int>(i % cgn);
  const long long bu = i / cgn;
  const long long Vc = static_cast<long long>(Dc) * Hc * Wc;
  const long long b = bu / Vc, u = bu % Vc;
  float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < 8; ++k) {
    const long long v = child_index(u, Dc, Hc, Wc, k >> 2, (k >> 1) & 1, k & 1);
    float f[8];
    unpack8(*reinterpret_cast<const uint4*>(dcat + (b * 8 * Vc + v) * Ct + Cs + cg * 8), f);
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j] += f[j];
  }
  float m[8];
  unpack8(*reinterpret_cast<const uint4*>(src + bu * Cu + cg * 8), m);
#pragma unroll
  for (int j = 0; j < 8; ++j) s[j] = m[j] > 0.0f ? s[j] : 0.0f;
  *reinterpret_cast<uint4*>(g + bu * Cu + cg * 8) = pack8(s);
}

constexpr int kHeadC = 32, kHeadO = 4;

// x0[b][l][v] = scale * (bo[l] + sum_c Wo[l][c] d0[b][v][c])
__global__ void head_predict_kernel(const bf16* __restrict__ d0, const float* __restrict__ wo, const float* __restrict__ bo,
                                    int C, int NO, double scale, double* __restrict__ x0, long long V, long long total) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= total) return;
  const long long b = i / V, v = i % V;
  float f[kHeadC];
  for (int c0 = 0; c0 < C; c0 += 8) {
    float t[8];
    unpack8(*reinterpret_cast<const uint4*>(d0 + i * C + c0), t);
    for (int j = 0; j < 8; ++j) f[c0 + j] = t[j];
  }
  for (int l = 0; l < NO; ++l) {
    float o = bo[l];
    for (int c = 0; c < C; ++c) o = fmaf(wo[l * C + c], f[c], o);
    x0[(b * NO + l) * V + v] = scale * static_cast<double>(o);
  }
}

// Head forward, squared-error loss and head backward.  Per voxel: o = bo + Wo d0, r = o - t / scale,
// g = 2 r / count, dpre[v][c] = (Wo^T g)[c] * (d0 > 0).  Per block: partial sums of g_l d0_c (dWo),
// g_l (dbo) and r^2 (loss), in the head's parameter layout followed by the loss.
// FROM_G: the output gradient g is given (gin[b][l][v], from h1_loss_kernel) instead of formed from
// the target; the loss slot of the partials is then 0.
constexpr int kHeadTile = 256;
template <bool FROM_G>
__global__ void __launch_bounds__(kHeadTile) head_loss_kernel(const bf16* __restrict__ d0, const float* __restrict__ wo,
                                                              const float* __restrict__ bo, const double* __restrict__ target,
                                                              const float* __restrict__ gin, int C, int NO,
                                                              double inv_scale, float inv_count,
                                                              bf16* __restrict__ dpre, float* partial, long long V,
                                                              long long total) {
  __shared__ float ds[kHeadTile][kHeadC + 1];
  __shared__ float gs[kHeadTile][kHeadO + 1];
  const int tid = threadIdx.x;
  const int npair = NO * C;
  float acc = 0.0f;  // thread tid < npair: dWo[l][c]; npair + l: dbo[l]; npair + NO: loss
  for (long long base = static_cast<long long>(blockIdx.x) * kHeadTile; base < total;
       base += static_cast<long long>(gridDim.x) * kHeadTile) {
    const long long i = base + tid;
    float f[kHeadC];
    float g[kHeadO];
    float r2 = 0.0f;
    if (i < total) {
      const long long b = i / V, v = i % V;
      for (int c0 = 0; c0 < C; c0 += 8) {
        float t[8];
        unpack8(*reinterpret_cast<const uint4*>(d0 + i * C + c0), t);
        for (int j = 0; j < 8; ++j) f[c0 + j] = t[j];
      }
      for (int l = 0; l < NO; ++l) {
        if (FROM_G) {
          g[l] = gin[(b * NO + l) * V + v];
        } else {
          float o = bo[l];
          for (int c = 0; c < C; ++c) o = fmaf(wo[l * C + c], f[c], o);
          const float r = o - static_cast<float>(target[(b * NO + l) * V + v] * inv_scale);
          r2 = fmaf(r, r, r2);
          g[l] = 2.0f * r * inv_count;
        }
      }
      for (int c0 = 0; c0 < C; c0 += 8) {
        float d[8];
        for (int j = 0; j < 8; ++j) {
          float s = 0.0f;
          for (int l = 0; l < NO; ++l) s = fmaf(wo[l * C + c0 + j], g[l], s);
          d[j] = f[c0 + j] > 0.0f ? s : 0.0f;
        }
        *reinterpret_cast<uint4*>(dpre + i * C + c0) = pack8(d);
      }
    } else {
      for (int c = 0; c < C; ++c) f[c] = 0.0f;
      for (int l = 0; l < NO; ++l) g[l] = 0.0f;
    }
    __syncthreads();
    for (int c = 0; c < C; ++c) ds[tid][c] = f[c];
    for (int l = 0; l < NO; ++l) gs[tid][l] = g[l];
    gs[tid][kHeadO] = r2 * inv_count;
    __syncthreads();
    if (tid < npair) {
      const int l = tid / C, c = tid % C;
      for (int k = 0; k < kHeadTile; ++k) acc = fmaf(gs[k][l], ds[k][c], acc);
    } else if (tid < npair + NO) {
      for (int k = 0; k < kHeadTile; ++k) acc += gs[k][tid - npair];
    } else if (tid == npair + NO) {
      for (int k = 0; k < kHeadTile; ++k) acc += gs[k][kHeadO];
    }
  }
  if (tid <= npair + NO) partial[static_cast<long long>(blockIdx.x) * (npair + NO + 1) + tid] = acc;
}

// r[b][l][v] = bo[l] + sum_c Wo[l][c] d0[b][v][c] - target[b][l][v] / scale
__global__ void head_residual_kernel(const bf16* __restrict__ d0, const float* __restrict__ wo, const float* __restrict__ bo,
                                     const double* __restrict__ target, int C, int NO, double inv_scale,
                                     float* __restrict__ r, long long V, long long total) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= total) return;
  const long long b = i / V, v = i % V;
  float f[kHeadC];
  for (int c0 = 0; c0 < C; c0 += 8) {
    float t[8];
    unpack8(*reinterpret_cast<const uint4*>(d0 + i * C + c0), t);
    for (int j = 0; j < 8; ++j) f[c0 + j] = t[j];
  }
  for (int l = 0; l < NO; ++l) {
    float o = bo[l];
    for (int c = 0; c < C; ++c) o = fmaf(wo[l * C + c], f[c], o);
    r[(b * NO + l) * V + v] = o - static_cast<float>(target[(b * NO + l) * V + v] * inv_scale);
  }
}

// Discrete H^1 loss of the residual fields r (n^3 periodic, one per (sample, load)): loss = (sum over
// axes of squared forward differences + w2 r^2) / count, gradient g = (2 w2 r + 2 sum over axes of
// (2 r - r(+a) - r(-a))) / count.  Per block: partial sum of the loss.
__global__ void __launch_bounds__(256) h1_loss_kernel(const float* __restrict__ r, float* __restrict__ g, int n,
                                                      long long total, float w2, float inv_count, float* partial) {
  __shared__ float red[256];
  const long long V = static_cast<long long>(n) * n * n;
  float acc = 0.0f;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < total; i += static_cast<long long>(gridDim.x) * 256) {
    const long long f = i / V, v = i % V;
    const int x = static_cast<int>(v % n), y = static_cast<int>((v / n) % n), z = static_cast<int>(v / (static_cast<long long>(n) * n));
    const float* rf = r + f * V;
    const float c = rf[v];
    const float xp = rf[v - x + (x + 1 == n ? 0 : x + 1)], xm = rf[v - x + (x == 0 ? n - 1 : x - 1)];
    const long long row = static_cast<long long>(n);
    const float yp = rf[v + ((y + 1 == n ? 0 : y + 1) - y) * row], ym = rf[v + ((y == 0 ? n - 1 : y - 1) - y) * row];
    const long long pl = row * n;
    const float zp = rf[v + ((z + 1 == n ? 0 : z + 1) - z) * pl], zm = rf[v + ((z == 0 ? n - 1 : z - 1) - z) * pl];
    acc += (xp - c) * (xp - c) + (yp - c) * (yp - c) + (zp - c) * (zp - c) + w2 * c * c;
    g[i] = inv_count * (2.0f * w2 * c + 2.0f * (6.0f * c - xp - xm - yp - ym - zp - zm));
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0] * inv_count;
}

__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float c1, float c2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// BF16 operands of one layer from its FP32 weights W[27][Cout][Cin]:
// wb = W (forward), wt[26 - t][i][o] = W[t][o][i] (input gradient: flipped taps, transposed channels)
__global__ void prep_weights_kernel(const float* __restrict__ w, bf16* __restrict__ wb, bf16* __restrict__ wt, int Cin,
                                    int Cout) {
  const long long n = 27LL * Cin * Cout;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int t = static_cast<int>(i / (static_cast<long long>(Cout) * Cin));
    const int o = static_cast<int>((i / Cin) % Cout), c = static_cast<int>(i % Cin);
    const bf16 h = __float2bfloat16_rn(w[i]);
    wb[i] = h;
    wt[(static_cast<long long>(26 - t) * Cin + c) * Cout + o] = h;
  }
}

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
int blocks_for(long long n, int bs) { return static_cast<int>(std::max<long long>(1, (n + bs - 1) / bs)); }

template <int NT, int ZT>
cudaError_t launch_conv_nt(const ConvArgs& a, int B, cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(conv3_tc_kernel<NT, ZT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                conv_smem_bytes<NT, ZT>());
  });
  if (attr != cudaSuccess) return attr;
  const dim3 grid(((a.W + 7) / 8) * ((a.H + 15) / 16), a.D / ZT, B * (a.Cout / NT));
  conv3_tc_kernel<NT, ZT><<<grid, 128, conv_smem_bytes<NT, ZT>(), s>>>(a);
  return cudaGetLastError();
}

template <int NT>
cudaError_t launch_conv_z(const ConvArgs& a, int B, cudaStream_t s) {
  if (a.D % 4 == 0) return launch_conv_nt<NT, 4>(a, B, s);
  if (a.D % 2 == 0) return launch_conv_nt<NT, 2>(a, B, s);
  return launch_conv_nt<NT, 1>(a, B, s);
}

cudaError_t launch_conv(const ConvArgs& a, int B, cudaStream_t s) {
  if (a.Cout % 64 == 0) return launch_conv_z<64>(a, B, s);
  if (a.Cout % 32 == 0) return launch_conv_z<32>(a, B, s);
  return launch_conv_z<16>(a, B, s);
}

struct WgradPlan {
  int n_tiles, tiles_per_cta, chunks;
};
WgradPlan wgrad_plan(int B, int D, int H, int W, int Cin) {
  WgradPlan p;
  p.n_tiles = B * D * ((H + 15) / 16) * ((W + 7) / 8);
  const int kcs = Cin / 16;
  const int want = std::max(1, std::min(p.n_tiles, 2 * 152 / kcs));
  p.tiles_per_cta = (p.n_tiles + want - 1) / want;
  p.chunks = (p.n_tiles + p.tiles_per_cta - 1) / p.tiles_per_cta;
  return p;
}

cudaError_t launch_wgrad(const bf16* x, const bf16* dy, float* partial, float* out, int accumulate, int B, int D, int H,
                         int W, int Cin, int Cout, int* err, cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
  });
  if (attr != cudaSuccess) return attr;
  const WgradPlan p = wgrad_plan(B, D, H, W, Cin);
  WgradArgs a{x, dy, partial, D, H, W, Cin, Cout, p.n_tiles, p.tiles_per_cta, err};
  wgrad_tc_kernel<<<dim3(p.chunks, Cin / 16), 128, kWgSmem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long len = 27LL * Cout * Cin;
  reduce_partials_kernel<<<blocks_for(len, 256), 256, 0, s>>>(partial, p.chunks, len, out, accumulate);
  return cudaGetLastError();
}

size_t wgrad_partial_floats(int B, int D, int H, int W, int Cin, int Cout) {
  return static_cast<size_t>(wgrad_plan(B, D, H, W, Cin).chunks) * 27 * Cout * Cin;
}

}  // namespace
}  // namespace fehom_unet_impl

// ==================================================================================================
// network object
// ==================================================================================================
using namespace fehom_unet_impl;

struct UnetLayer {
  int cin = 0, cout = 0, level = 0;
  long long w_off = 0, b_off = 0;
  bf16* wb = nullptr;
  bf16* wt = nullptr;
};

struct fehom_unet {
  int n = 0, L = 0, max_batch = 0, n_phases = 0, n_out = 0, dev = 0;
  std::vector<int> w;
  std::vector<UnetLayer> layers;
  long long head_off = 0, n_params = 0;
  float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  int step = 0;
  std::vector<bf16*> EA, E, P, CAT, DA, DD, G0, G1, DC, DP;
  float* partial = nullptr;
  size_t partial_floats = 0;
  float* loss = nullptr;
  int* err = nullptr;
  int loss_kind = 0;     // 0: mean squared error, 1: discrete H^1 seminorm (+ l2_weight * squared error)
  float l2_weight = 0.0f;
  float* rbuf = nullptr;  // [max_batch][n_out][n^3] residual fields (H^1 loss)
  float* gbuf = nullptr;  // [max_batch][n_out][n^3] their gradient
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool weights_dirty = true;
  std::string error;
  std::vector<void*> allocs;

  int idx_e(int l, bool a) const { return 2 * l + (a ? 0 : 1); }
  int idx_d(int l, bool a) const { return 2 * L + 2 * (L - 2 - l) + (a ? 0 : 1); }
  int edge(int l) const { return n >> l; }
  long long vox(int l) const { return static_cast<long long>(edge(l)) * edge(l) * edge(l); }
};

namespace {
std::mutex g_create_mu;
std::string g_create_error;

fehom_status fail(fehom_unet* net, fehom_status st, const std::string& msg) {
  if (net) net->error = msg;
  return st;
}
fehom_status cuda_fail(fehom_unet* net, cudaError_t e, const char* where) {
  return fail(net, FEHOM_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define UCK(call)                                          \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(net, e_, #call); \
  } while (0)

template <class T>
cudaError_t alloc(fehom_unet* net, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e == cudaSuccess) {
    net->allocs.push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
}

fehom_status refresh_weights(fehom_unet* net) {
  if (!net->weights_dirty) return FEHOM_OK;
  for (size_t i = 0; i < net->layers.size(); ++i) {
    const UnetLayer& ly = net->layers[i];
    if (!ly.wb) continue;
    prep_weights_kernel<<<blocks_for(27LL * ly.cin * ly.cout, 256), 256, 0, net->stream>>>(net->theta + ly.w_off, ly.wb,
                                                                                         ly.wt, ly.cin, ly.cout);
    UCK(cudaGetLastError());
  }
  net->weights_dirty = false;
  return FEHOM_OK;
}

// y = relu(conv(x)) at level l with layer ly
fehom_status conv_layer(fehom_unet* net, int batch, const UnetLayer& ly, const bf16* x, bf16* y) {
  const int e = net->edge(ly.level);
  ConvArgs a{x, ly.wb, net->theta + ly.b_off, nullptr, y, nullptr, e, e, e, ly.cin, ly.cout, 1, net->err};
  UCK(launch_conv(a, batch, net->stream));
  return FEHOM_OK;
}

fehom_status forward(fehom_unet* net, int batch, const uint8_t* ids, const float* feat) {
  fehom_status st = refresh_weights(net);
  if (st != FEHOM_OK) return st;
  const int L = net->L;
  const int n = net->n;
  {
    const UnetLayer& ly = net->layers[net->idx_e(0, true)];
    const long long total = batch * net->vox(0);
    conv_in_kernel<<<blocks_for(total, 128), 128, 0, net->stream>>>(ids, feat, net->n_phases, net->theta + ly.w_off,
                                                                  net->theta + ly.b_off, net->EA[0], n, n, n, ly.cout,
                                                                  total);
    UCK(cudaGetLastError());
  }
  if ((st = conv_layer(net, batch, net->layers[net->idx_e(0, false)], net->EA[0], net->E[0])) != FEHOM_OK) return st;
  for (int l = 1; l < L; ++l) {
    const int ec = net->edge(l);
    const long long total = batch * net->vox(l) * (net->w[l - 1] / 8);
    pool_kernel<<<blocks_for(total, 256), 256, 0, net->stream>>>(net->E[l - 1], net->P[l], ec, ec, ec, net->w[l - 1],
                                                               total);
    UCK(cudaGetLastError());
    if ((st = conv_layer(net, batch, net->layers[net->idx_e(l, true)], net->P[l], net->EA[l])) != FEHOM_OK) return st;
    if ((st = conv_layer(net, batch, net->layers[net->idx_e(l, false)], net->EA[l], net->E[l])) != FEHOM_OK) return st;
  }
  const bf16* below = net->E[L - 1];
  for (int l = L - 2; l >= 0; --l) {
    const int e = net->edge(l);
    const int Cs = net->w[l], Cu = net->w[l + 1];
    const long long total = batch * net->vox(l) * ((Cs + Cu) / 8);
    upcat_kernel<<<blocks_for(total, 256), 256, 0, net->stream>>>(net->E[l], below, net->CAT[l], e, e, e, Cs, Cu, total);
    UCK(cudaGetLastError());
    if ((st = conv_layer(net, batch, net->layers[net->idx_d(l, true)], net->CAT[l], net->DA[l])) != FEHOM_OK) return st;
    if ((st = conv_layer(net, batch, net->layers[net->idx_d(l, false)], net->DA[l], net->DD[l])) != FEHOM_OK) return st;
    below = net->DD[l];
  }
  return FEHOM_OK;
}

const bf16* top_output(const fehom_unet* net) { return net->L > 1 ? net->DD[0] : net->E[0]; }

// weight and bias gradients of layer ly from its input x and pre-activation gradient g; then the
// input gradient (times the ReLU mask of the input when mask != null) into dx when dx != null
fehom_status layer_backward(fehom_unet* net, int batch, const UnetLayer& ly, const bf16* x, const bf16* g,
                            const bf16* mask, bf16* dx) {
  const int e = net->edge(ly.level);
  UCK(launch_wgrad(x, g, net->partial, net->grad + ly.w_off, 0, batch, e, e, e, ly.cin, ly.cout, net->err, net->stream));
  const long long rows = batch * net->vox(ly.level);
  const int per = static_cast<int>(std::max<long long>(256, (rows + 2 * 152 - 1) / (2 * 152)));
  const int nblk = blocks_for(rows, per);
  const int bs = ly.cout * std::max(1, 256 / ly.cout);
  chansum_kernel<<<nblk, bs, bs * sizeof(float), net->stream>>>(g, rows, ly.cout, per, net->partial);
  UCK(cudaGetLastError());
  reduce_partials_kernel<<<1, 256, 0, net->stream>>>(net->partial, nblk, ly.cout, net->grad + ly.b_off, 0);
  UCK(cudaGetLastError());
  if (dx) {
    ConvArgs a{g, ly.wt, nullptr, mask, dx, nullptr, e, e, e, ly.cout, ly.cin, 0, net->err};
    UCK(launch_conv(a, batch, net->stream));
  }
  return FEHOM_OK;
}

fehom_status backward(fehom_unet* net, int batch, const uint8_t* ids, const float* feat, const double* target,
                      double out_scale) {
  const int L = net->L;
  fehom_status st;
  // head, loss
  {
    const int C = net->w[0], NO = net->n_out;
    const long long V = net->vox(0), total = batch * V;
    const int nblk = static_cast<int>(std::min<long long>(4 * 152, (total + kHeadTile - 1) / kHeadTile));
    const float inv_count = static_cast<float>(1.0 / (static_cast<double>(total) * NO));
    const float* wo = net->theta + net->head_off;
    const float* bo = wo + NO * C;
    int h1_blocks = 0;
    if (net->loss_kind == 1) {
      head_residual_kernel<<<blocks_for(total, 256), 256, 0, net->stream>>>(top_output(net), wo, bo, target, C, NO,
                                                                           1.0 / out_scale, net->rbuf, V, total);
      UCK(cudaGetLastError());
      h1_blocks = static_cast<int>(std::min<long long>(4 * 152, (total * NO + 255) / 256));
      h1_loss_kernel<<<h1_blocks, 256, 0, net->stream>>>(net->rbuf, net->gbuf, net->n, total * NO, net->l2_weight,
                                                         inv_count, net->partial + net->partial_floats / 2);
      UCK(cudaGetLastError());
      head_loss_kernel<true><<<nblk, kHeadTile, 0, net->stream>>>(top_output(net), wo, bo, target, net->gbuf, C, NO,
                                                                  1.0 / out_scale, inv_count, net->G0[0], net->partial,
                                                                  V, total);
    } else {
      head_loss_kernel<false><<<nblk, kHeadTile, 0, net->stream>>>(top_output(net), wo, bo, target, nullptr, C, NO,
                                                                   1.0 / out_scale, inv_count, net->G0[0], net->partial,
                                                                   V, total);
    }
    UCK(cudaGetLastError());
    const int len = NO * C + NO + 1;
    // parameter gradients of the head; the loss lands in net->loss (one float after them)
    reduce_partials_kernel<<<1, 256, 0, net->stream>>>(net->partial, nblk, len, net->loss - (NO * C + NO), 0);
    UCK(cudaGetLastError());
    if (h1_blocks > 0) {
      reduce_partials_kernel<<<1, 32, 0, net->stream>>>(net->partial + net->partial_floats / 2, h1_blocks, 1, net->loss, 0);
      UCK(cudaGetLastError());
    }
    UCK(cudaMemcpyAsync(net->grad + net->head_off, net->loss - (NO * C + NO), (NO * C + NO) * sizeof(float),
                        cudaMemcpyDeviceToDevice, net->stream));
  }
  for (int l = 0; l <= L - 2; ++l) {
    const int e = net->edge(l + 1);
    if ((st = layer_backward(net, batch, net->layers[net->idx_d(l, false)], net->DA[l], net->G0[l], net->DA[l],
                             net->G1[l])) != FEHOM_OK)
      return st;
    if ((st = layer_backward(net, batch, net->layers[net->idx_d(l, true)], net->CAT[l], net->G1[l], nullptr,
                             net->DC[l])) != FEHOM_OK)
      return st;
    const bf16* src = (l + 1 <= L - 2) ? net->DD[l + 1] : net->E[L - 1];
    const int Cu = net->w[l + 1];
    const long long total = batch * net->vox(l + 1) * (Cu / 8);
    up_grad_kernel<<<blocks_for(total, 256), 256, 0, net->stream>>>(net->DC[l], net->w[l], Cu, src, net->G0[l + 1], e, e,
                                                                  e, total);
    UCK(cudaGetLastError());
  }
  for (int l = L - 1; l >= 0; --l) {
    const int e = net->edge(l);
    if (l < L - 1) {
      const int C = net->w[l];
      const long long total = batch * net->vox(l) * (C / 8);
      enc_grad_kernel<<<blocks_for(total, 256), 256, 0, net->stream>>>(net->DC[l], C + net->w[l + 1], net->DP[l + 1],
                                                                     net->E[l], net->G0[l], e, e, e, C, total);
      UCK(cudaGetLastError());
    }
    if ((st = layer_backward(net, batch, net->layers[net->idx_e(l, false)], net->EA[l], net->G0[l], net->EA[l],
                             net->G1[l])) != FEHOM_OK)
      return st;
    if (l > 0) {
      if ((st = layer_backward(net, batch, net->layers[net->idx_e(l, true)], net->P[l], net->G1[l], nullptr,
                               net->DP[l])) != FEHOM_OK)
        return st;
    } else {
      const UnetLayer& ly = net->layers[net->idx_e(0, true)];
      const int nblk = batch * e;
      const int bs = ((28 * ly.cout + 31) / 32) * 32;
      const size_t sm = (9 * e + e * ly.cout) * sizeof(float);
      if (sm > 48 * 1024)
        UCK(cudaFuncSetAttribute(conv_in_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
      conv_in_wgrad_kernel<<<nblk, bs, sm, net->stream>>>(ids, feat, net->n_phases, net->G1[0], net->partial, e, e, e,
                                                          ly.cout);
      UCK(cudaGetLastError());
      reduce_partials_kernel<<<blocks_for(28 * ly.cout, 256), 256, 0, net->stream>>>(net->partial, nblk, 28 * ly.cout,
                                                                                   net->grad + ly.w_off, 0);
      UCK(cudaGetLastError());
    }
  }
  return FEHOM_OK;
}

fehom_status check_batch(fehom_unet* net, int batch, const void* ids, const void* feat) {
  if (!net) return FEHOM_E_INVALID;
  if (batch < 1 || batch > net->max_batch) return fail(net, FEHOM_E_INVALID, "batch outside 1..max_batch");
  if (!ids || !feat) return fail(net, FEHOM_E_INVALID, "ids and features are required");
  return FEHOM_OK;
}

fehom_status check_err_flag(fehom_unet* net) {
  int h = 0;
  UCK(cudaMemcpyAsync(&h, net->err, sizeof(int), cudaMemcpyDeviceToHost, net->stream));
  UCK(cudaStreamSynchronize(net->stream));
  if (h != 0) return fail(net, FEHOM_E_CUDA, "a tensor-core kernel timed out waiting for its MMAs");
  return FEHOM_OK;
}
}  // namespace

extern "C" {

fehom_status fehom_unet_create(fehom_unet** out, int64_t n, int n_levels, const int* widths, int n_phases, int n_out,
                               int max_batch, void* stream) {
  auto reject = [](const std::string& m) {
    std::lock_guard<std::mutex> g(g_create_mu);
    g_create_error = m;
    return FEHOM_E_INVALID;
  };
  if (!out || !widths) return reject("out and widths are required");
  *out = nullptr;
  if (n_levels < 1 || n_levels > 6) return reject("n_levels outside 1..6");
  const long long stride = 1LL << (n_levels - 1);
  if (n < 1 || n > 512 || n % stride != 0) return reject("n must be a multiple of 2^(n_levels-1), at most 512");
  for (int l = 0; l < n_levels; ++l) {
    if (widths[l] < 16 || widths[l] > 256 || widths[l] % 16 != 0) return reject("widths must be multiples of 16 in 16..256");
    if (l + 1 < n_levels && widths[l] + widths[l + 1] > 256) return reject("w_l + w_{l+1} must be <= 256");
  }
  if (widths[0] > 32) return reject("w_0 must be <= 32");
  if (n_phases < 1 || n_phases > 256) return reject("n_phases outside 1..256");
  if (n_out < 1 || n_out > 4) return reject("n_out outside 1..4");
  if (max_batch < 1) return reject("max_batch must be >= 1");

  fehom_unet* net = new fehom_unet();
  net->n = static_cast<int>(n);
  net->L = n_levels;
  net->max_batch = max_batch;
  net->n_phases = n_phases;
  net->n_out = n_out;
  net->w.assign(widths, widths + n_levels);
  cudaGetDevice(&net->dev);
  auto bail = [&](fehom_status st) {
    {
      std::lock_guard<std::mutex> g(g_create_mu);
      g_create_error = net->error;
    }
    fehom_unet_destroy(net);
    return st;
  };
  if (stream) {
    net->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreate(&net->stream) != cudaSuccess) return bail(fail(net, FEHOM_E_CUDA, "cudaStreamCreate failed"));
    net->own_stream = true;
  }
  // layers in parameter order
  long long off = 0;
  auto add = [&](int cin, int cout, int level) {
    UnetLayer ly;
    ly.cin = cin;
    ly.cout = cout;
    ly.level = level;
    ly.w_off = off;
    off += 27LL * cin * cout;
    ly.b_off = off;
    off += cout;
    net->layers.push_back(ly);
  };
  const int L = n_levels;
  add(1, widths[0], 0);
  add(widths[0], widths[0], 0);
  for (int l = 1; l < L; ++l) {
    add(widths[l - 1], widths[l], l);
    add(widths[l], widths[l], l);
  }
  for (int l = L - 2; l >= 0; --l) {
    add(widths[l] + widths[l + 1], widths[l], l);
    add(widths[l], widths[l], l);
  }
  net->head_off = off;
  off += static_cast<long long>(n_out) * widths[0] + n_out;
  net->n_params = off;

  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t count) {
    if (e == cudaSuccess) e = alloc(net, p, count);
  };
  A(&net->theta, net->n_params);
  A(&net->grad, net->n_params);
  A(&net->m, net->n_params);
  A(&net->v, net->n_params);
  A(&net->err, 1);
  for (size_t i = 1; i < net->layers.size(); ++i) {
    UnetLayer& ly = net->layers[i];
    A(&ly.wb, 27LL * ly.cin * ly.cout);
    A(&ly.wt, 27LL * ly.cin * ly.cout);
  }
  const long long B = max_batch;
  net->EA.assign(L, nullptr);
  net->E.assign(L, nullptr);
  net->P.assign(L, nullptr);
  net->CAT.assign(L, nullptr);
  net->DA.assign(L, nullptr);
  net->DD.assign(L, nullptr);
  net->G0.assign(L, nullptr);
  net->G1.assign(L, nullptr);
  net->DC.assign(L, nullptr);
  net->DP.assign(L, nullptr);
  for (int l = 0; l < L; ++l) {
    const long long V = B * net->vox(l);
    A(&net->EA[l], V * widths[l]);
    A(&net->E[l], V * widths[l]);
    A(&net->G0[l], V * widths[l]);
    A(&net->G1[l], V * widths[l]);
    if (l > 0) {
      A(&net->P[l], V * widths[l - 1]);
      A(&net->DP[l], V * widths[l - 1]);
    }
    if (l + 1 < L) {
      A(&net->CAT[l], V * (widths[l] + widths[l + 1]));
      A(&net->DC[l], V * (widths[l] + widths[l + 1]));
      A(&net->DA[l], V * widths[l]);
      A(&net->DD[l], V * widths[l]);
    }
  }
  // scratch for block partials: weight gradients, bias sums, first layer, head
  size_t pf = 0;
  for (size_t i = 1; i < net->layers.size(); ++i) {
    const UnetLayer& ly = net->layers[i];
    const int ed = net->edge(ly.level);
    pf = std::max(pf, wgrad_partial_floats(max_batch, ed, ed, ed, ly.cin, ly.cout));
    pf = std::max(pf, static_cast<size_t>(2 * 152 + 1) * ly.cout);
  }
  pf = std::max(pf, static_cast<size_t>(B) * net->n * 28 * widths[0]);
  pf = std::max(pf, static_cast<size_t>(4 * 152) * (n_out * widths[0] + n_out + 1));
  pf = 2 * std::max(pf, static_cast<size_t>(4 * 152));  // second half: partials of the H^1 loss
  net->partial_floats = pf;
  A(&net->rbuf, static_cast<size_t>(B) * n_out * net->vox(0));
  A(&net->gbuf, static_cast<size_t>(B) * n_out * net->vox(0));
  A(&net->partial, pf);
  float* headbuf = nullptr;
  A(&headbuf, n_out * widths[0] + n_out + 1);
  if (e != cudaSuccess) return bail(fail(net, FEHOM_E_OOM, std::string("device allocation: ") + cudaGetErrorString(e)));
  net->loss = headbuf + n_out * widths[0] + n_out;
  if (cudaMemsetAsync(net->theta, 0, net->n_params * sizeof(float), net->stream) != cudaSuccess ||
      cudaMemsetAsync(net->m, 0, net->n_params * sizeof(float), net->stream) != cudaSuccess ||
      cudaMemsetAsync(net->v, 0, net->n_params * sizeof(float), net->stream) != cudaSuccess ||
      cudaMemsetAsync(net->err, 0, sizeof(int), net->stream) != cudaSuccess ||
      cudaStreamSynchronize(net->stream) != cudaSuccess)
    return bail(fail(net, FEHOM_E_CUDA, "initialising the network buffers failed"));
  *out = net;
  return FEHOM_OK;
}

void fehom_unet_destroy(fehom_unet* net) {
  if (!net) return;
  if (net->stream) cudaStreamSynchronize(net->stream);
  for (void* p : net->allocs) cudaFree(p);
  if (net->own_stream && net->stream) cudaStreamDestroy(net->stream);
  delete net;
}

const char* fehom_unet_last_error(const fehom_unet* net) {
  if (!net) {
    std::lock_guard<std::mutex> g(g_create_mu);
    return g_create_error.c_str();
  }
  return net->error.c_str();
}

fehom_status fehom_unet_set_loss(fehom_unet* net, int kind, double l2_weight) {
  if (!net) return FEHOM_E_INVALID;
  if ((kind != FEHOM_LOSS_MSE && kind != FEHOM_LOSS_H1) || !(l2_weight >= 0.0))
    return fail(net, FEHOM_E_INVALID, "loss kind must be FEHOM_LOSS_MSE or FEHOM_LOSS_H1, l2_weight >= 0");
  net->loss_kind = kind;
  net->l2_weight = static_cast<float>(l2_weight);
  return FEHOM_OK;
}

fehom_status fehom_unet_param_count(const fehom_unet* net, int64_t* n_params) {
  if (!net || !n_params) return FEHOM_E_INVALID;
  *n_params = net->n_params;
  return FEHOM_OK;
}

fehom_status fehom_unet_set_params(fehom_unet* net, const float* theta) {
  if (!net || !theta) return net ? fail(net, FEHOM_E_INVALID, "theta is required") : FEHOM_E_INVALID;
  UCK(cudaMemcpyAsync(net->theta, theta, net->n_params * sizeof(float), cudaMemcpyHostToDevice, net->stream));
  UCK(cudaMemsetAsync(net->m, 0, net->n_params * sizeof(float), net->stream));
  UCK(cudaMemsetAsync(net->v, 0, net->n_params * sizeof(float), net->stream));
  UCK(cudaStreamSynchronize(net->stream));
  net->step = 0;
  net->weights_dirty = true;
  return FEHOM_OK;
}

fehom_status fehom_unet_get_params(fehom_unet* net, float* theta) {
  if (!net || !theta) return net ? fail(net, FEHOM_E_INVALID, "theta is required") : FEHOM_E_INVALID;
  UCK(cudaMemcpyAsync(theta, net->theta, net->n_params * sizeof(float), cudaMemcpyDeviceToHost, net->stream));
  UCK(cudaStreamSynchronize(net->stream));
  return FEHOM_OK;
}

fehom_status fehom_unet_predict(fehom_unet* net, int batch, const uint8_t* ids, const float* features, double out_scale,
                                double* x0) {
  fehom_status st = check_batch(net, batch, ids, features);
  if (st != FEHOM_OK) return st;
  if (!x0) return fail(net, FEHOM_E_INVALID, "x0 is required");
  if ((st = forward(net, batch, ids, features)) != FEHOM_OK) return st;
  const long long V = net->vox(0), total = batch * V;
  head_predict_kernel<<<blocks_for(total, 256), 256, 0, net->stream>>>(
      top_output(net), net->theta + net->head_off, net->theta + net->head_off + net->n_out * net->w[0], net->w[0],
      net->n_out, out_scale, x0, V, total);
  UCK(cudaGetLastError());
  return FEHOM_OK;
}

fehom_status fehom_unet_loss_grad(fehom_unet* net, int batch, const uint8_t* ids, const float* features,
                                  const double* target, double out_scale, double* loss, float* grad) {
  fehom_status st = check_batch(net, batch, ids, features);
  if (st != FEHOM_OK) return st;
  if (!target || !(out_scale > 0.0)) return fail(net, FEHOM_E_INVALID, "target and out_scale > 0 are required");
  if ((st = forward(net, batch, ids, features)) != FEHOM_OK) return st;
  if ((st = backward(net, batch, ids, features, target, out_scale)) != FEHOM_OK) return st;
  if ((st = check_err_flag(net)) != FEHOM_OK) return st;
  if (loss) {
    float h = 0.0f;
    UCK(cudaMemcpy(&h, net->loss, sizeof(float), cudaMemcpyDeviceToHost));
    *loss = h;
  }
  if (grad) UCK(cudaMemcpy(grad, net->grad, net->n_params * sizeof(float), cudaMemcpyDeviceToHost));
  return FEHOM_OK;
}

fehom_status fehom_unet_train_step(fehom_unet* net, int batch, const uint8_t* ids, const float* features,
                                   const double* target, double out_scale, double lr, double* loss) {
  fehom_status st = check_batch(net, batch, ids, features);
  if (st != FEHOM_OK) return st;
  if (!target || !(out_scale > 0.0) || !(lr > 0.0)) return fail(net, FEHOM_E_INVALID, "target, out_scale > 0, lr > 0 required");
  if ((st = forward(net, batch, ids, features)) != FEHOM_OK) return st;
  if ((st = backward(net, batch, ids, features, target, out_scale)) != FEHOM_OK) return st;
  net->step += 1;
  const double c1 = 1.0 / (1.0 - std::pow(0.9, net->step)), c2 = 1.0 / (1.0 - std::pow(0.999, net->step));
  adam_kernel<<<2 * 152, 256, 0, net->stream>>>(net->theta, net->grad, net->m, net->v, net->n_params,
                                                static_cast<float>(lr), static_cast<float>(c1), static_cast<float>(c2));
  UCK(cudaGetLastError());
  net->weights_dirty = true;
  if (loss) {
    float h = 0.0f;
    UCK(cudaMemcpyAsync(&h, net->loss, sizeof(float), cudaMemcpyDeviceToHost, net->stream));
    if ((st = check_err_flag(net)) != FEHOM_OK) return st;
    *loss = h;
  }
  return FEHOM_OK;
}

fehom_status fehom_conv3_bf16(int B, int D, int H, int W, int Cin, int Cout, const void* x, const void* w,
                              const float* bias, int relu, float* y, void* stream) {
  if (B < 1 || D < 1 || H < 1 || W < 1 || Cin < 16 || Cin % 16 || Cout < 16 || Cout % 16 || Cout > 256 || !x || !w || !y)
    return FEHOM_E_INVALID;
  ConvArgs a{static_cast<const bf16*>(x), static_cast<const bf16*>(w), bias, nullptr, nullptr, y, D, H, W, Cin, Cout,
             relu, nullptr};
  return launch_conv(a, B, static_cast<cudaStream_t>(stream)) == cudaSuccess ? FEHOM_OK : FEHOM_E_CUDA;
}

fehom_status fehom_conv3_wgrad_bf16(int B, int D, int H, int W, int Cin, int Cout, const void* x, const void* dy,
                                    float* dw, void* stream) {
  if (B < 1 || D < 1 || H < 1 || W < 1 || Cin < 16 || Cin % 16 || Cout < 16 || Cout % 16 || Cout > 128 || !x || !dy || !dw)
    return FEHOM_E_INVALID;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* partial = nullptr;
  int* err = nullptr;
  if (cudaMalloc(&partial, wgrad_partial_floats(B, D, H, W, Cin, Cout) * sizeof(float)) != cudaSuccess)
    return FEHOM_E_OOM;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaFree(partial);
    return FEHOM_E_OOM;
  }
  int h = 0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = launch_wgrad(static_cast<const bf16*>(x), static_cast<const bf16*>(dy), partial, dw, 0, B, D, H, W, Cin, Cout,
                     err, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(partial);
  cudaFree(err);
  if (e != cudaSuccess || h != 0) return FEHOM_E_CUDA;
  return FEHOM_OK;
}

}  // extern "C"
