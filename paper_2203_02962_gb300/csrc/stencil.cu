// Matrix-free stiffness apply y = s * D^T W C (D x + e) on the periodic grid (Sec. 5.1; Eq. lin_system).
//
// Voxel-wise constant material C_e = C[phase(e)] is looked up by phase id (Sec. 3.1: the tangent
// is diagonal per quadrature point; here it is constant per voxel as in Sec. 6.1).
//
// Trilinear hexahedron (HEX8_3D), 2x2x2 Gauss points.  The element field is written in the modal
// basis {1, xi, eta, zeta, xi eta, eta zeta, xi zeta, xi eta zeta} on [-1, 1]^3, obtained from the
// 8 nodal values by three butterfly stages (a Hadamard transform).  Its gradient is a sum of the
// seven mutually orthogonal monomials {1, xi, eta, zeta, eta zeta, xi zeta, xi eta}; since 2-point
// Gauss rules integrate their products exactly, the element energy is
//     a_e(u, u) = sum_m mu_m g_m^T Chat g_m,   mu = 1 (m = 1), 1/3 (linear), 1/9 (bilinear),
// where g_m holds the modal coefficients that multiply monomial m in each derivative and
// Chat = V_e S P^T C P S is the material in gradient coordinates (P: gradient -> Mandel strain,
// S: d/dxi -> d/dx scaling, V_e: voxel volume).  This is the same bilinear form as the quadrature
// sum of Eq. global_sum, evaluated with 7 small contractions instead of 8 quadrature points.
// The element forces follow from the transposed butterflies.
//
// 2-D pixels: P1TRI2_2D (two triangles with constant gradients, w = V_p/2 each, Fig. 3 b) and
// Q1_2D (bilinear, modal basis {1, xi, eta, xi eta}, 2x2 Gauss, Fig. 3 a).
//
// Tiling.  A CTA owns BX x BY output nodes of the x-y plane and marches along z through a slab of
// KZ planes.  Per element layer it stages the next node plane (with a periodic halo of one node)
// in shared memory, computes the (BX+1) x (BY+1) elements of the layer once each, writes their
// corner forces to shared memory, and lets each node thread gather the four bottom corners that
// complete its node plane (the four top corners are carried to the next layer in registers).
// No atomics; fixed summation order.
#include "fehom_internal.cuh"
#include "tma.cuh"

#include <algorithm>
#include <cstdio>
#include <type_traits>

namespace fehom {
namespace {

constexpr int BX = 32;
constexpr int PX = BX + 2;  // halo row of the 2-D pixel kernel
constexpr int EX = BX + 1;

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// 4-byte asynchronous global -> shared copies (FP32 stiffness: node planes fetched one layer ahead)
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}

// staged node plane (FP32 kernels): a row holds the nodes i0 - 1 .. i0 + BX at columns RX0 .. RX0 + BX + 1,
// so the tile interior i0 .. i0 + BX - 1 starts on a 16-byte boundary (column 4); row pitch 40 floats
constexpr int RP = BX + 8;
constexpr int RX0 = 3;

// hex8 tiles: BX x BY output nodes per CTA, (BX + 1) x (BY + 1) elements per layer, one element per
// thread; BY = 8 (297 elements, 320 threads) or 16 (561 elements, 576 threads: fewer lanes on halo
// elements, one CTA per SM).  Defaults: FP64 kernels BY = 16 (the FP64 pipe is their bound), FP32
// kernels BY = 8 at three CTAs per SM (more warps to keep the issue slots busy across the per-layer
// barriers).  The PCG apply of either precision takes either height; the stencil tuner of the context
// (api.cu) times both on the solve's buffers and keeps the faster.
template <typename T, int BYT>
struct Hex8Tile {
  static constexpr int BY = BYT;
  static constexpr int EY = BY + 1;
  static constexpr int NE = EX * EY;                 // elements per layer per CTA (297 / 561)
  static constexpr int NT = ((NE + 31) / 32) * 32;   // threads (320 / 576)
  static constexpr int RPLANE = RP * (BY + 2);       // nodes of a staged plane per component
  static constexpr int PER_SM = BY == 16 ? 1 : (sizeof(T) == 8 ? 2 : 3);  // resident CTAs per SM (launch bounds)
};
template <typename T>
constexpr int hex8_default_rows() { return sizeof(T) == 8 ? 16 : 8; }

// Block-wide FP64 sum; every thread gets the result. `sh` holds >= 32 doubles.
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

// Deterministic reduction finalisation: CTA partials -> last-arriving CTA sums them in index order.
// Returns true in the (single) CTA that must finalise; `total` is valid there.
__device__ bool finish_reduction(double part, double* partial, unsigned* counter, int nblk, int bid,
                                 double* sh, double* total) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partial[bid] = part;
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    last = (prev == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc = 0.0;
  // fixed order: thread t sums blocks t, t + NT, ...; then a fixed-shape tree
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += ((volatile double*)partial)[b];
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    *total = t;
    *counter = 0u;  // self-reset for the next launch
  }
  return true;
}

// ------------------------------------------------------------------------------------------------
// element kernels: modal contractions
// ------------------------------------------------------------------------------------------------
// General material: T[j][i] = sum_{l,k active} Ch[(j*3+i)*D + l*3+k] * g[l][k], active dirs = MASK.
template <int MASK, int C, typename T>
__device__ __forceinline__ void contract_gen(const T* __restrict__ Ch, const T (&g)[C][3], T wgt, T (&out)[C][3]) {
  constexpr int D = 3 * C;
#pragma unroll
  for (int j = 0; j < C; ++j)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (!((MASK >> i) & 1)) continue;
      const int kk = (C == 1) ? i : (j * 3 + i);
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < C; ++l)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if (!((MASK >> k) & 1)) continue;
          const int ll = (C == 1) ? k : (l * 3 + k);
          acc = fma(__ldg(Ch + kk * D + ll), g[l][k], acc);
        }
      out[j][i] = acc * wgt;
    }
}

// Hex8 element in face form.  The Hadamard (modal) transform of the 8 nodal values factors into an
// in-plane part per x-y face -- (ss, sd, ds, dd) = the sums / differences along x, then along y, of
// the face's 4 nodes -- and a z part that combines the element's bottom (c = 0) and top (c = 1)
// faces.  Each face is shared by the two element layers next to it, so the kernel forms it once per
// node plane.  In reverse, the element's dual modal forces give per-face partials (the transposed
// z part); a face's two partials are summed before the transposed in-plane part spreads them to
// its 4 corner nodes.
//   bot/top[j][0..3] = (ss, sd, ds, dd) of the bottom / top face of component j
//   pb/pt[j][0..3]   = the element's partials for its bottom / top face
//   t1o              = the monomial-1 dual (Chat g_1 + tau), whose sum over elements is |Y| S P^T <sigma>
// Without a nodal field (HAS_X false: the right-hand side -D^T W C e) only T1 = tau is nonzero.
//
// Modal coefficients q_n[j] of component j (z part below) and the gradient they give per monomial
// (g_m[j][i]: derivative i of component j multiplying monomial m):
//   1: (q1, q2, q3)   xi: (0, q4, q6)   eta: (q4, 0, q5)   zeta: (q6, q5, 0)
//   eta zeta: (q7, 0, 0)   xi zeta: (0, q7, 0)   xi eta: (0, 0, q7)
// The dual Q_n[j] = dE/dq_n[j] sums t_m = Chat g_m over the monomials that q_n enters.
//
// Isotropic material on cubic voxels, t_m = lam' tr(g_m) I + mu' (g_m + g_m^T) weighted 1, 1/3, 1/9:
// the duals reduce to closed forms (35 operations instead of seven contractions):
//   Q1..Q3 = the columns of t_1 (symmetric: Q1[1] = Q2[0], Q1[2] = Q3[0], Q2[2] = Q3[1])
//   Q4 = (L tr_y + mu' q4[0], L tr_x + mu' q4[1], M (q4[2] + s))
//   Q5 = (M (q5[0] + s), L tr_z + mu' q5[1], L tr_y + mu' q5[2])
//   Q6 = (L tr_z + mu' q6[0], M (q6[1] + s), L tr_x + mu' q6[2])
//   Q7 = K7 q7
// with L = lam'/3, M = mu'/3, K7 = (lam' + 4 mu')/9, tr_x = q4[1] + q6[2], tr_y = q4[0] + q5[2],
// tr_z = q6[0] + q5[1] (the traces of the linear monomials' gradients), s = q4[2] + q5[0] + q6[1].
template <typename T, int C, bool ISO, bool HAS_X, bool HAS_E>
__device__ __forceinline__ void hex8_element_faces(const T (&bot)[C][4], const T (&top)[C][4], const T* __restrict__ Ch,
                                                   const T* __restrict__ iso, const double* __restrict__ tau,
                                                   T (&pb)[C][4], T (&pt)[C][4], T (&t1o)[C][3]) {
  T Q1[C], Q2[C], Q3[C], Q4[C], Q5[C], Q6[C], Q7[C];
  if constexpr (!HAS_X) {
#pragma unroll
    for (int j = 0; j < C; ++j) {
      Q1[j] = HAS_E ? T(tau[j * 3 + 0]) : T(0);
      Q2[j] = HAS_E ? T(tau[j * 3 + 1]) : T(0);
      Q3[j] = HAS_E ? T(tau[j * 3 + 2]) : T(0);
      Q4[j] = Q5[j] = Q6[j] = Q7[j] = T(0);
    }
  } else {
    // z part of the modal transform
    T q1[C], q2[C], q3[C], q4[C], q5[C], q6[C], q7[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      q3[j] = top[j][0] - bot[j][0];
      q2[j] = top[j][1] + bot[j][1];
      q5[j] = top[j][1] - bot[j][1];
      q1[j] = top[j][2] + bot[j][2];
      q6[j] = top[j][2] - bot[j][2];
      q4[j] = top[j][3] + bot[j][3];
      q7[j] = top[j][3] - bot[j][3];
    }
    if constexpr (ISO && C == 1) {
      // isotropic conductivity: the duals scale the modal coefficients (iso_entry_scalar)
      T k1, k23, k3;
      if constexpr (sizeof(T) == 4) {
        const float4 c0 = __ldg(reinterpret_cast<const float4*>(iso));
        k1 = c0.x; k23 = c0.y; k3 = c0.z;
      } else {
        const double2 c0 = __ldg(reinterpret_cast<const double2*>(iso));
        k1 = c0.x; k23 = c0.y; k3 = __ldg(iso + 2);
      }
      Q1[0] = k1 * q1[0];
      Q2[0] = k1 * q2[0];
      Q3[0] = k1 * q3[0];
      Q4[0] = k23 * q4[0];
      Q5[0] = k23 * q5[0];
      Q6[0] = k23 * q6[0];
      Q7[0] = k3 * q7[0];
    } else if constexpr (ISO && C == 3) {
      T lam, mu, mu2, L, M, K7;
      if constexpr (sizeof(T) == 4) {  // one entry = 8 floats, 32-byte aligned: two 16-byte loads
        const float4 c0 = __ldg(reinterpret_cast<const float4*>(iso));
        const float4 c1 = __ldg(reinterpret_cast<const float4*>(iso) + 1);
        lam = c0.x; mu = c0.y; mu2 = c0.z; L = c0.w; M = c1.x; K7 = c1.y;
      } else {  // one entry = 8 doubles, 64-byte aligned: three 16-byte loads
        const double2 c0 = __ldg(reinterpret_cast<const double2*>(iso));
        const double2 c1 = __ldg(reinterpret_cast<const double2*>(iso) + 1);
        const double2 c2 = __ldg(reinterpret_cast<const double2*>(iso) + 2);
        lam = c0.x; mu = c0.y; mu2 = c1.x; L = c1.y; M = c2.x; K7 = c2.y;
      }
      const T lt = lam * (q1[0] + q2[1] + q3[2]);
      Q1[0] = fma(mu2, q1[0], lt);
      Q2[1] = fma(mu2, q2[1], lt);
      Q3[2] = fma(mu2, q3[2], lt);
      Q1[1] = Q2[0] = mu * (q1[1] + q2[0]);
      Q1[2] = Q3[0] = mu * (q1[2] + q3[0]);
      Q2[2] = Q3[1] = mu * (q2[2] + q3[1]);
      const T Ltx = L * (q4[1] + q6[2]), Lty = L * (q4[0] + q5[2]), Ltz = L * (q6[0] + q5[1]);
      const T sm = q4[2] + q5[0] + q6[1];
      Q4[0] = fma(mu, q4[0], Lty);
      Q4[1] = fma(mu, q4[1], Ltx);
      Q4[2] = M * (q4[2] + sm);
      Q5[0] = M * (q5[0] + sm);
      Q5[1] = fma(mu, q5[1], Ltz);
      Q5[2] = fma(mu, q5[2], Lty);
      Q6[0] = fma(mu, q6[0], Ltz);
      Q6[1] = M * (q6[1] + sm);
      Q6[2] = fma(mu, q6[2], Ltx);
#pragma unroll
      for (int j = 0; j < 3; ++j) Q7[j] = K7 * q7[j];
    } else {
      // general material: contract each monomial's gradient, then sum the contributions per mode
      T g1[C][3], gx[C][3], gy[C][3], gz[C][3], gyz[C][3], gxz[C][3], gxy[C][3];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        g1[j][0] = q1[j]; g1[j][1] = q2[j]; g1[j][2] = q3[j];
        gx[j][0] = T(0);  gx[j][1] = q4[j]; gx[j][2] = q6[j];
        gy[j][0] = q4[j]; gy[j][1] = T(0);  gy[j][2] = q5[j];
        gz[j][0] = q6[j]; gz[j][1] = q5[j]; gz[j][2] = T(0);
        gyz[j][0] = q7[j]; gyz[j][1] = T(0); gyz[j][2] = T(0);
        gxz[j][0] = T(0); gxz[j][1] = q7[j]; gxz[j][2] = T(0);
        gxy[j][0] = T(0); gxy[j][1] = T(0); gxy[j][2] = q7[j];
      }
      constexpr double third = 1.0 / 3.0, ninth = 1.0 / 9.0;
      T t1[C][3], tx[C][3], ty[C][3], tz[C][3], tyz[C][3], txz[C][3], txy[C][3];
      contract_gen<7>(Ch, g1, T(1), t1);
      contract_gen<6>(Ch, gx, T(third), tx);
      contract_gen<5>(Ch, gy, T(third), ty);
      contract_gen<3>(Ch, gz, T(third), tz);
      contract_gen<1>(Ch, gyz, T(ninth), tyz);
      contract_gen<2>(Ch, gxz, T(ninth), txz);
      contract_gen<4>(Ch, gxy, T(ninth), txy);
#pragma unroll
      for (int j = 0; j < C; ++j) {
        Q1[j] = t1[j][0]; Q2[j] = t1[j][1]; Q3[j] = t1[j][2];
        Q4[j] = tx[j][1] + ty[j][0];
        Q5[j] = ty[j][2] + tz[j][1];
        Q6[j] = tx[j][2] + tz[j][0];
        Q7[j] = tyz[j][0] + txz[j][1] + txy[j][2];
      }
    }
    if constexpr (HAS_E) {
#pragma unroll
      for (int j = 0; j < C; ++j) {
        Q1[j] += T(tau[j * 3 + 0]);
        Q2[j] += T(tau[j * 3 + 1]);
        Q3[j] += T(tau[j * 3 + 2]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < C; ++j) {
    t1o[j][0] = Q1[j]; t1o[j][1] = Q2[j]; t1o[j][2] = Q3[j];
    // the transposed z part
    pb[j][0] = -Q3[j];         pt[j][0] = Q3[j];
    pb[j][1] = Q2[j] - Q5[j];  pt[j][1] = Q2[j] + Q5[j];
    pb[j][2] = Q1[j] - Q6[j];  pt[j][2] = Q1[j] + Q6[j];
    pb[j][3] = Q4[j] - Q7[j];  pt[j][3] = Q4[j] + Q7[j];
  }
}

// ------------------------------------------------------------------------------------------------
// reductions fused into the stiffness apply
//   RED_NONE  y only
//   RED_PCG   <x, y> -> pAp and alpha = rz / pAp in the load's PCG state (last CTA, fixed order)
//   RED_STATS per CTA: sum y^2 over its nodes and the sum of the monomial-1 duals over its elements
//             (partials [load][cta][1 + D], reduced on the host in index order)
// ------------------------------------------------------------------------------------------------
//   RED_SUMS  the RED_STATS sums without storing y (y may be NULL)
enum { RED_NONE = 0, RED_PCG = 1, RED_STATS = 2, RED_SUMS = 3 };

__device__ void pcg_alpha_update(PcgState& s, double total, double* hist) {
  s.pAp = total;
  if (!(total > 0.0) || !isfinite(total)) {
    s.state = ST_BREAK;
    s.alpha = 0.0;
  } else {
    s.alpha = s.rz / total;
  }
  if (hist != nullptr && s.iter < kHist) hist[s.iter] = s.alpha;
}

// ------------------------------------------------------------------------------------------------
// 3-D hex8 kernel
//
// Per element layer k (between node planes k and k + 1):
//   A. face threads read the 4 nodes of their x-y face of plane k + 1 (periodic offsets computed
//      once; neighbouring faces share nodes through L1) and store its in-plane butterflies (one
//      thread per face: the butterflies are private to it);
//   B. element threads combine the faces of planes k and k + 1, contract with the material, add
//      the bottom partials to the top partials carried from layer k - 1 (registers) and spread the
//      face total to its 4 corners of plane k (corner buffer k mod 2);
//   (barrier)
//   C. node threads gather the 4 faces around their node of plane k and write y.
// One barrier per layer: the corner buffers alternate, so the gather of layer k - 1 and the writes
// of layer k + 1 to the same buffer are ordered by the barrier of layer k.
// ------------------------------------------------------------------------------------------------
// RAW (FP32 kernels with a field): instead of step A, the raw node planes (tile + halo) are fetched
// with cp.async one layer ahead into a ring of three plane buffers, made visible by a second
// barrier per layer (which also orders the single corner buffer), and each element forms the
// butterflies of its top face itself, the bottom face being the previous layer's top (FP32 adds are
// cheap; the FP64 kernels keep the per-plane butterflies, which save FP64 operations).  The x
// values of the <x, y> dot come from the same staged plane.
template <typename T, int C, bool HAS_X>
__host__ __device__ constexpr bool hex8_raw() { return HAS_X && sizeof(T) == 4; }
constexpr int kRing = 5;  // RAW: staged node planes k .. k + 4
// RAW elasticity packs the corner forces of an element as one float4 per corner (3 components + pad)
template <typename T, int C, bool HAS_X>
__host__ __device__ constexpr bool hex8_pack() { return hex8_raw<T, C, HAS_X>() && C == 3; }
// staging of the RAW kernels' node planes: STG_CP4 4-byte cp.async copies of every entry (any grid),
// STG_CP16 16-byte cp.async row copies (every x tile full), STG_TMA one tensor-memory-accelerator box per
// plane issued by one thread, completion on an mbarrier per ring slot (every x tile full)
enum { STG_CP4 = 0, STG_CP16 = 1, STG_TMA = 2 };
// ring slot stride in elements: TMA destinations sit on 128-byte boundaries
template <typename T, int C, int BYT, int STG>
__host__ __device__ constexpr int hex8_slot_elems() {
  constexpr int e = C * Hex8Tile<T, BYT>::RPLANE;
  return STG == STG_TMA ? (int)((e * sizeof(T) + 127) / 128 * 128 / sizeof(T)) : e;
}
constexpr int kTmaHdr = 128;  // bytes before the TMA ring: one mbarrier per slot
template <typename T, int C, bool HAS_X, int BYT, int STG = STG_CP4>
__host__ __device__ constexpr size_t hex8_smem_elems() {
  using TL = Hex8Tile<T, BYT>;
  return hex8_raw<T, C, HAS_X>()
             ? (size_t)kRing * hex8_slot_elems<T, C, BYT, STG>() +
                   2 * 4 * (hex8_pack<T, C, HAS_X>() ? 4 : C) * TL::NE +
                   (STG == STG_TMA ? (kTmaHdr + 128) / sizeof(T) : 0)
             : (size_t)2 * 4 * C * TL::NE + 2 * 4 * C * TL::NE;
}

template <typename T, int C, bool ISO, bool HAS_X, bool HAS_E, int RED, int BYT, int STG = STG_CP4>
__global__ void __launch_bounds__(Hex8Tile<T, BYT>::NT, Hex8Tile<T, BYT>::PER_SM)
    hex8_apply_kernel(const __grid_constant__ CUtensorMap tmap, StencilArgs a, int kz_per_cta) {
  constexpr bool RAW = hex8_raw<T, C, HAS_X>();
  constexpr bool PACK = hex8_pack<T, C, HAS_X>();
  constexpr bool WIDE = STG != STG_CP4;
  constexpr bool TMA = RAW && STG == STG_TMA;
  constexpr int BY = BYT, NE = Hex8Tile<T, BYT>::NE, NT = Hex8Tile<T, BYT>::NT;
  constexpr int RPLANE = Hex8Tile<T, BYT>::RPLANE;
  constexpr int SLOTE = hex8_slot_elems<T, C, BYT, STG>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // TMA: a 128-byte aligned base (the launch adds 128 bytes of slack), one mbarrier per ring slot first
  unsigned char* smem_base =
      TMA ? smem_raw + ((128u - (tma::smem_u32(smem_raw) & 127u)) & 127u) : smem_raw;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_base);
  T* FB = reinterpret_cast<T*>(smem_base);  // [2 planes][4][C][NE] face butterflies (not RAW)
  T* RW = reinterpret_cast<T*>(smem_base + (TMA ? kTmaHdr : 0));  // [kRing slots][C][BY + 2][RP] staged planes (RAW)
  // [4 corners][C][NE] face contributions to plane k; without RAW two of them, by the parity of k
  T* FC0 = RAW ? RW + kRing * SLOTE : FB + 2 * 4 * C * NE;
  __shared__ double red_sh[32];

  const Dims d = a.d;
  const int load = blockIdx.z;
  if (RED == RED_PCG && a.st != nullptr && a.st[load].state != ST_RUN) return;

  const int tiles_x = (d.nx + BX - 1) / BX;
  const int i0 = (blockIdx.x % tiles_x) * BX;
  const int j0 = (blockIdx.x / tiles_x) * BY;
  const int k0 = blockIdx.y * kz_per_cta;
  const int k1 = min(k0 + kz_per_cta, d.nz);
  const int tid = threadIdx.x;

  const T* x = HAS_X ? reinterpret_cast<const T*>(a.x) + (long long)load * a.load_stride : nullptr;
  T* y = reinterpret_cast<T*>(a.y) + (long long)load * a.load_stride;
  const T* mats = reinterpret_cast<const T*>(a.mats);
  const T* isot = reinterpret_cast<const T*>(a.iso);
  const double* tau = HAS_E ? a.tau + (long long)load * a.n_phases * (3 * C) : nullptr;
  const long long plane = (long long)d.nx * d.ny;
  const T ysc = T(a.y_scale);

  // face / element thread (ei, ej): face (ei, ej) of a plane = the x-y square whose corners are the
  // nodes (i0 - 1 + ei + a, j0 - 1 + ej + b); element (ei, ej) of a layer sits on that face
  const int ei = tid % EX, ej = tid / EX;
  const bool face_thread = tid < NE;
  const int fi0 = wrap(i0 - 1 + ei, d.nx), fi1 = wrap(i0 + ei, d.nx);
  const int fj0 = wrap(j0 - 1 + ej, d.ny), fj1 = wrap(j0 + ej, d.ny);
  const int off00 = fj0 * d.nx + fi0, off10 = fj0 * d.nx + fi1, off01 = fj1 * d.nx + fi0, off11 = fj1 * d.nx + fi1;
  const bool owner = face_thread && ei >= 1 && ej >= 1 && i0 + ei - 1 < d.nx && j0 + ej - 1 < d.ny;

  // node thread (ni, nj): node (i0 + ni, j0 + nj)
  const int ni = tid % BX, nj = tid / BX;
  const bool node_thread = tid < BX * BY && (i0 + ni) < d.nx && (j0 + nj) < d.ny;
  const long long node_off = (long long)(j0 + nj) * d.nx + i0 + ni;

  T carry[C][4];  // top partials of the previous layer for this thread's face
#pragma unroll
  for (int j = 0; j < C; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) carry[j][q] = T(0);
  DotAcc<T> acc_p;                     // RED_PCG: <x, y>
  double acc_y = 0.0;                  // RED_STATS / RED_SUMS: sum y^2 (FP64 kernels only)
  double acc_t[3 * C];                 // RED_STATS / RED_SUMS: sum of the monomial-1 duals of owned elements
#pragma unroll
  for (int i = 0; i < 3 * C; ++i) acc_t[i] = 0.0;

  auto next = [&](int z) { return z + 1 == d.nz ? 0 : z + 1; };
  // A: in-plane butterflies of the faces of node plane kz into slot SLOT
  auto faces = [&](auto slot_c, int kz) {
    if constexpr (HAS_X) {
      constexpr int SLOT = decltype(slot_c)::value;
      if (face_thread) {
        const T* xk = x + (long long)kz * plane;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const T* xj = xk + (long long)j * d.N;
          const T v00 = __ldg(xj + off00), v10 = __ldg(xj + off10), v01 = __ldg(xj + off01), v11 = __ldg(xj + off11);
          const T s0 = v10 + v00, d0 = v10 - v00, s1 = v11 + v01, d1 = v11 - v01;
          T* fb = FB + ((SLOT * 4) * C + j) * NE + tid;
          fb[0 * C * NE] = s1 + s0;  // ss
          fb[1 * C * NE] = s1 - s0;  // sd
          fb[2 * C * NE] = d1 + d0;  // ds
          fb[3 * C * NE] = d1 - d0;  // dd
        }
      }
    }
  };

  // RAW: stage node plane kz (tile nodes i0 - 1 .. i0 + BX, j0 - 1 .. j0 + BY) into ring slot `slot`.
  // WIDE (every tile lies inside the grid along x; nx, the load stride and the field base 16-byte
  // aligned; chosen by the host): each (component, row) is one 4-byte copy per halo node and eight
  // 16-byte copies of the interior, one task per thread.  Otherwise every staged entry is a 4-byte copy
  // with periodic wrap (this thread: entries tid + q NT of the padded plane; pad columns skipped).
  // Source offsets are fixed per CTA.
  // TMA: one box (x = i0 - 4 .. i0 + 35, rows j0 - 1 .. j0 + BY, the C components of the load) per plane,
  // issued by thread 0; the box reads zeros outside the grid, so at the periodic seams the halo entries
  // the wrap needs are patched by one load per thread (fetched a plane ahead) after the box has landed.
  // A plane is read only after a CTA barrier that follows thread 0's wait (acquire) on its mbarrier.
  constexpr int NROW = C * (BY + 2);  // staged rows per plane
  constexpr int NSTAGE = (WIDE || TMA) ? 1 : (C * RPLANE + NT - 1) / NT;
  int soff[NSTAGE], doff = 0;
  bool w16 = false;
#pragma unroll
  for (int q = 0; q < NSTAGE; ++q) soff[q] = -1;
  // TMA: per slot, the parity of its next phase and whether it was ever used (thread 0 keeps them in
  // shared memory: they are only needed to drain the ring after a failed wait)
  [[maybe_unused]] unsigned* tma_book = reinterpret_cast<unsigned*>(full + kRing);
  // TMA seam patch of this thread (staged entry and source offset from x), or dst < 0; recomputed where it
  // is used instead of held in registers across the layer loop
  [[maybe_unused]] auto seam_entry = [&](int& dst, unsigned& off) {
    const bool ls = i0 == 0, rs = i0 + BX == d.nx, ts = j0 == 0;
    const int rb = d.ny - j0 + 1;  // staged row of y = ny
    const bool bs = rb <= BY + 1;
    const int nl = ls ? C * (BY + 2) : 0, nr = rs ? C * (BY + 2) : 0;
    const int nt = ts ? C * (BX + 2) : 0, nb = bs ? C * (BX + 2) : 0;
    int e = tid, r = -1, j = 0, col = 0;  // col: staged column relative to RX0 (0 = x i0 - 1)
    if (e < nl) {
      r = e / C; j = e % C; col = 0;
    } else if ((e -= nl) < nr) {
      r = e / C; j = e % C; col = BX + 1;
    } else if ((e -= nr) < nt) {
      r = 0; j = e / (BX + 2); col = e % (BX + 2);
    } else if ((e -= nt) < nb) {
      r = rb; j = e / (BX + 2); col = e % (BX + 2);
    }
    dst = -1;
    if (r >= 0) {
      dst = j * RPLANE + r * RP + RX0 + col;
      off = (unsigned)((long long)j * d.N + (long long)wrap(j0 - 1 + r, d.ny) * d.nx + wrap(i0 - 1 + col, d.nx));
    }
  };
  // the CTA touches a periodic seam (then some of its threads patch entries after each box lands)
  [[maybe_unused]] const bool seam_cta = i0 == 0 || i0 + BX == d.nx || j0 == 0 || d.ny - j0 + 1 <= BY + 1;
  if constexpr (RAW && WIDE && !TMA) {
    if (tid < NROW * 10) {
      const int row = tid / 10, q = tid - row * 10, j = row / (BY + 2), r = row - j * (BY + 2);
      const int col = q == 0 ? 0 : (q == 9 ? BX + 1 : 1 + 4 * (q - 1));  // column relative to RX0
      doff = j * RPLANE + r * RP + RX0 + col;
      soff[0] = j * (int)d.N + wrap(j0 - 1 + r, d.ny) * d.nx + wrap(i0 - 1 + col, d.nx);
      w16 = q != 0 && q != 9;
    }
  } else if constexpr (RAW) {
#pragma unroll
    for (int q = 0; q < NSTAGE; ++q) {
      const int idx = tid + q * NT;
      if (idx < C * RPLANE) {
        const int j = idx / RPLANE, rem = idx - j * RPLANE, r = rem / RP, c = rem - r * RP - RX0;
        if (c >= 0 && c < BX + 2) soff[q] = j * (int)d.N + wrap(j0 - 1 + r, d.ny) * d.nx + wrap(i0 - 1 + c, d.nx);
      }
    }
  }
  auto stage_plane = [&](int slot, int kz, [[maybe_unused]] long long kzoff) {
    if constexpr (TMA) {
      if (tid == 0) {
        tma::fence_proxy_async();
        tma::mbar_expect_tx(&full[slot], (unsigned)(sizeof(T) * C * RPLANE));
        tma::load_4d(RW + slot * SLOTE, &tmap, i0 - 4, j0 - 1, load * C, kz, &full[slot]);
        tma_book[0] ^= 1u << slot;
        tma_book[1] |= 1u << slot;
      }
      return;
    } else if constexpr (RAW) {
      const T* xk = x + kzoff;  // kzoff = kz * plane
      T* dst = RW + slot * C * RPLANE;
      if constexpr (WIDE) {
        if (soff[0] >= 0) {
          if (w16) cp_async16(dst + doff, xk + soff[0]);
          else cp_async4(dst + doff, xk + soff[0]);
        }
      } else {
#pragma unroll
        for (int q = 0; q < NSTAGE; ++q)
          if (soff[q] >= 0) cp_async4(dst + tid + q * NT, xk + soff[q]);
      }
    }
    cp_async_commit();
  };
  // RAW: butterflies (ss, sd, ds, dd) of this thread's face in staged slot `slot`
  auto raw_face = [&](int slot, T (&f)[C][4]) {
    const T* src = RW + slot * SLOTE + ej * RP + RX0 + ei;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const T* sj = src + j * RPLANE;
      const T v00 = sj[0], v10 = sj[1], v01 = sj[RP], v11 = sj[RP + 1];
      const T s0 = v10 + v00, d0 = v10 - v00, s1 = v11 + v01, d1 = v11 - v01;
      f[j][0] = s1 + s0;
      f[j][1] = s1 - s0;
      f[j][2] = d1 + d0;
      f[j][3] = d1 - d0;
    }
  };
  T fprev[C][4];  // RAW: butterflies of the top face of the previous layer (this layer's bottom face)

  // B + C for element layer k (planes k: slot CUR, k + 1: slot CUR ^ 1); kzc = wrap(k).  RAW: plane k
  // sits in ring slot s0 = (k - k0 + 1) mod kRing and plane k + 4 (kz4 = wrap(k + 4)) goes to the slot
  // before it; both are carried from layer to layer instead of recomputed (no integer division)
  // TMA: a wait that gave up (about a second) ends the launch for the whole CTA at the next barrier
  [[maybe_unused]] bool timeout = false;
  [[maybe_unused]] T fv = T(0);                      // seam patch of the next plane to patch
  // the seam patch of plane p for this thread (0 when it has none)
  [[maybe_unused]] auto fetch = [&](int p) -> T {
    if constexpr (TMA) {
      if (!seam_cta) return T(0);
      int dst;
      unsigned off = 0u;
      seam_entry(dst, off);
      return dst >= 0 ? __ldg(x + off + (long long)wrap(p, d.nz) * plane) : T(0);
    } else {
      return T(0);
    }
  };

  // offsets kz * plane of the layer's plane and of the plane staged four ahead, carried from layer to
  // layer (no 64-bit multiplies in the loop)
  long long pc = (long long)wrap(k0 - 1, d.nz) * plane, p4 = RAW ? (long long)wrap(k0 + 3, d.nz) * plane : 0;
  // phase id of this face thread's element in the next layer (the first layer is k0 - 1, plane wrap(k0 - 1))
  int ph_n = (face_thread && a.ids != nullptr) ? a.ids[(long long)wrap(k0 - 1, d.nz) * plane + off00] : 0;
  auto layer = [&](auto cur_c, int k, int kzc, [[maybe_unused]] int s0, [[maybe_unused]] int kz4) -> bool {
    [[maybe_unused]] constexpr int CUR = decltype(cur_c)::value;
    [[maybe_unused]] const int s1 = s0 == kRing - 1 ? 0 : s0 + 1;
    // the face butterflies are private to their thread, and the corner buffer FC alternates with
    // the parity of the layer (the barrier of layer k - 1 orders the gather of layer k - 2 before
    // the writes below), so no barrier is needed before the element step
    if constexpr (!RAW) faces(std::integral_constant<int, CUR ^ 1>{}, next(kzc));
    T* FC = FC0 + CUR * 4 * (PACK ? 4 : C) * NE;
    if (face_thread) {
      T bot[C][4], top[C][4];
      if constexpr (RAW) {
        if (k == k0 - 1) {
          raw_face(s0, bot);
        } else {
#pragma unroll
          for (int j = 0; j < C; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) bot[j][q] = fprev[j][q];
        }
        raw_face(s1, top);
#pragma unroll
        for (int j = 0; j < C; ++j)
#pragma unroll
          for (int q = 0; q < 4; ++q) fprev[j][q] = top[j][q];
      } else {
#pragma unroll
        for (int j = 0; j < C; ++j)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            bot[j][q] = HAS_X ? FB[((CUR * 4 + q) * C + j) * NE + tid] : T(0);
            top[j][q] = HAS_X ? FB[(((CUR ^ 1) * 4 + q) * C + j) * NE + tid] : T(0);
          }
      }
      // this layer's phase id was read a layer ahead; the next layer's read is issued before the
      // element arithmetic so that its latency hides behind this layer
      const int ph = ph_n;
      if (a.ids != nullptr && k + 1 < k1) ph_n = a.ids[(kzc + 1 == d.nz ? 0 : pc + plane) + off00];
      T pb[C][4], pt[C][4], t1[C][3];
      hex8_element_faces<T, C, ISO, HAS_X, HAS_E>(bot, top, mats + (long long)ph * (9 * C * C), isot + kIsoStride * ph,
                                                  HAS_E ? tau + ph * (3 * C) : nullptr, pb, pt, t1);
      T cv[4][C];  // corner forces: (0, 0), (1, 0), (0, 1), (1, 1)
#pragma unroll
      for (int j = 0; j < C; ++j) {
        // face total of plane k, then the transposed in-plane part: corners (a, b) of the face
        const T ss = pb[j][0] + carry[j][0], sd = pb[j][1] + carry[j][1];
        const T ds = pb[j][2] + carry[j][2], dd = pb[j][3] + carry[j][3];
        const T s0 = ss - sd, s1 = ss + sd, d0 = ds - dd, d1 = ds + dd;
        cv[0][j] = s0 - d0;
        cv[1][j] = s0 + d0;
        cv[2][j] = s1 - d1;
        cv[3][j] = s1 + d1;
#pragma unroll
        for (int q = 0; q < 4; ++q) carry[j][q] = pt[j][q];
      }
      if constexpr (PACK) {
        float4* F4 = reinterpret_cast<float4*>(FC);
#pragma unroll
        for (int cn = 0; cn < 4; ++cn) F4[cn * NE + tid] = make_float4(cv[cn][0], cv[cn][1], cv[cn][2], 0.0f);
      } else {
#pragma unroll
        for (int cn = 0; cn < 4; ++cn)
#pragma unroll
          for (int j = 0; j < C; ++j) FC[(cn * C + j) * NE + tid] = cv[cn][j];
      }
      if ((RED == RED_STATS || RED == RED_SUMS) && owner && k >= k0) {
#pragma unroll
        for (int j = 0; j < C; ++j)
#pragma unroll
          for (int i = 0; i < 3; ++i) acc_t[j * 3 + i] += (double)t1[j][i];
      }
    }
    // RAW: this thread's copies of plane k + 2 (issued three layers ago) have landed; the barrier
    // makes them visible for element layer k + 1 and frees the slot of plane k - 1.  TMA: thread 0 waits
    // for the box of plane k + 2 and the seam entries are patched before the barrier
    if constexpr (TMA) {
      // plane k + 2 sits in slot s0 + 2 (mod kRing), in that slot's phase number (k - k0 + 3) / kRing
      const int s_fix = s0 + 2 >= kRing ? s0 + 2 - kRing : s0 + 2;
      const unsigned par_fix = (unsigned)((k - k0 + 3) / kRing) & 1u;
      if (k + 2 <= k1) {
        if (tid == 0 && !tma::mbar_wait(&full[s_fix], par_fix)) timeout = true;
        if (seam_cta) {
          int dst;
          unsigned off = 0u;
          seam_entry(dst, off);
          if (dst >= 0) {
            if (!tma::mbar_wait(&full[s_fix], par_fix)) timeout = true;
            RW[s_fix * SLOTE + dst] = fv;
            fv = k + 3 <= k1 ? __ldg(x + off + (long long)wrap(k + 3, d.nz) * plane) : T(0);
          }
        }
      }
      if (__syncthreads_or(timeout)) return false;
      if (k + 4 <= k1) stage_plane(s0 == 0 ? kRing - 1 : s0 - 1, kz4, p4);
    } else {
      if constexpr (RAW) cp_async_wait_group<1>();
      __syncthreads();
      if constexpr (RAW) {
        if (k + 4 <= k1) stage_plane(s0 == 0 ? kRing - 1 : s0 - 1, kz4, p4);
        else cp_async_commit();  // an empty group keeps one group per layer
      }
    }
    if (node_thread && k >= k0) {
      // node (i, j) of plane k is corner (1,1) of face (i-1, j-1), (0,1) of (i, j-1),
      // (1,0) of (i-1, j) and (0,0) of (i, j)
      const int e00 = nj * EX + ni;
      T gv[C];
      if constexpr (PACK) {
        const float4* F4 = reinterpret_cast<const float4*>(FC);
        const float4 a3 = F4[3 * NE + e00], a2 = F4[2 * NE + e00 + 1], a1 = F4[1 * NE + e00 + EX],
                     a0 = F4[0 * NE + e00 + EX + 1];
        gv[0] = a3.x + a2.x + a1.x + a0.x;
        gv[1] = a3.y + a2.y + a1.y + a0.y;
        gv[2] = a3.z + a2.z + a1.z + a0.z;
      } else {
#pragma unroll
        for (int j = 0; j < C; ++j)
          gv[j] = FC[(3 * C + j) * NE + e00] + FC[(2 * C + j) * NE + e00 + 1] + FC[(1 * C + j) * NE + e00 + EX] +
                  FC[(0 * C + j) * NE + e00 + EX + 1];
      }
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const T v = gv[j];
        const T val = ysc * v;
        const long long gidx = (long long)j * d.N + pc + node_off;
        if (RED != RED_SUMS) y[gidx] = val;
        if constexpr (RED == RED_PCG) {
          if constexpr (RAW) acc_p.add(val, RW[s0 * SLOTE + j * RPLANE + (nj + 1) * RP + RX0 + ni + 1]);
          else acc_p.add(val, __ldg(x + gidx));
        }
        if (RED == RED_STATS || RED == RED_SUMS) acc_y += (double)val * (double)val;
      }
    }
    // the next layer writes the other corner buffer; plane k's slot is refilled after the barrier
    // of layer k + 1
    return true;
  };

  int kz = wrap(k0 - 1, d.nz);
  bool ok = true;
  if constexpr (TMA) {  // planes k0 - 1 .. k0 + 2 issued; k0 - 1 and k0 landed, patched and visible to all
    if (tid == 0) {
      for (int sl = 0; sl < kRing; ++sl) tma::mbar_init(&full[sl], 1);
      tma_book[0] = tma_book[1] = 0u;
      tma::fence_mbar_init();
    }
    __syncthreads();
    for (int p = 0; p < 4; ++p)
      if (k0 - 1 + p <= k1) stage_plane(p, wrap(k0 - 1 + p, d.nz), (long long)wrap(k0 - 1 + p, d.nz) * plane);
    const T fa = fetch(k0 - 1), fb = fetch(k0);
    int dst = -1;
    unsigned off = 0u;
    if (seam_cta) seam_entry(dst, off);
    if (tid == 0 || dst >= 0)
      if (!tma::mbar_wait(&full[0], 0) || !tma::mbar_wait(&full[1], 0)) timeout = true;
    if (dst >= 0) {
      RW[dst] = fa;
      RW[SLOTE + dst] = fb;
    }
    fv = k0 + 1 <= k1 ? fetch(k0 + 1) : T(0);
    ok = !__syncthreads_or(timeout);
  } else if constexpr (RAW) {  // planes k0 - 1 .. k0 + 2, one group each; the first two visible to all
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (k0 - 1 + p <= k1) stage_plane(p, wrap(k0 - 1 + p, d.nz), (long long)wrap(k0 - 1 + p, d.nz) * plane);
      else cp_async_commit();
    }
    cp_async_wait_group<2>();
    __syncthreads();
  } else {
    faces(std::integral_constant<int, 0>{}, kz);
  }
  int k = k0 - 1;
  int s0 = 0, kz4 = RAW ? wrap(k0 + 3, d.nz) : 0;
  auto advance = [&] {
    kz = next(kz);
    pc = kz == 0 ? 0 : pc + plane;
    if constexpr (RAW) {
      kz4 = next(kz4);
      p4 = kz4 == 0 ? 0 : p4 + plane;
      s0 = s0 == kRing - 1 ? 0 : s0 + 1;
    }
    ++k;
  };
  while (ok && k < k1) {
    if (!(ok = layer(std::integral_constant<int, 0>{}, k, kz, s0, kz4))) break;
    advance();
    if (k >= k1) break;
    if (!(ok = layer(std::integral_constant<int, 1>{}, k, kz, s0, kz4))) break;
    advance();
  }
  if constexpr (TMA) {
    if (!ok) {  // a wait gave up: let the boxes in flight land (bounded), mark the load and leave
      if (tid == 0) {
        for (int sl = 0; sl < kRing; ++sl)
          if ((tma_book[1] >> sl) & 1u) tma::mbar_wait(&full[sl], ((tma_book[0] >> sl) & 1u) ^ 1u);
        if (a.st != nullptr) {
          a.st[load].err = 1;
          a.st[load].state = ST_BREAK;
        }
      }
      return;
    }
  }

  if (RED == RED_PCG) {
    const double part = block_sum(acc_p.value(), red_sh);
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    double total;
    if (finish_reduction(part, a.red.partial + (long long)load * a.red.max_blocks, a.red.count + load, nblk,
                         bid, red_sh, &total)) {
      if (threadIdx.x == 0)
        pcg_alpha_update(a.st[load], total, a.red.hist ? a.red.hist + (long long)load * 2 * kHist : nullptr);
    }
  }
  if (RED == RED_STATS || RED == RED_SUMS) {
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    double* out = a.stats + ((long long)load * nblk + bid) * (1 + 3 * C);
    const double ty = block_sum(acc_y, red_sh);
    if (threadIdx.x == 0) out[0] = ty;
#pragma unroll
    for (int i = 0; i < 3 * C; ++i) {
      const double t = block_sum(acc_t[i], red_sh);
      if (threadIdx.x == 0) out[1 + i] = t;
    }
  }
}

// ------------------------------------------------------------------------------------------------
// 2-D pixel kernels (P1 triangles, Q1)
// ------------------------------------------------------------------------------------------------
// t1o receives the sum of the quadrature-point duals that carry the constant strain (both triangles
// for P1, the monomial-1 dual for Q1): their sum over elements is |Y| S P^T <sigma>.
template <typename T, int C, int ELEM, bool HAS_E>
__device__ __forceinline__ void pixel_element(const T (&u)[C][4], const T* __restrict__ Ch,
                                              const double* __restrict__ tau, T (&f)[C][4], T (&t1o)[C][2]) {
  constexpr int D = 2 * C;
  // corners: 0 = (0,0), 1 = (1,0), 2 = (0,1), 3 = (1,1); g[j][dir] = raw difference / modal coefficient
  auto contract = [&](const T (&g)[C][2], T w, T (&out)[C][2], int mask) {
#pragma unroll
    for (int j = 0; j < C; ++j)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        T acc = T(0);
#pragma unroll
        for (int l = 0; l < C; ++l)
#pragma unroll
          for (int k = 0; k < 2; ++k)
            if ((mask >> k) & 1) acc = fma(__ldg(Ch + (j * 2 + i) * D + l * 2 + k), g[l][k], acc);
        out[j][i] = acc * w;
      }
  };
  if constexpr (ELEM == P1TRI2_2D) {
    // triangle A (0,0),(1,0),(1,1): gx = u1 - u0, gy = u3 - u1; triangle B (0,0),(1,1),(0,1): gx = u3 - u2, gy = u2 - u0
    T gA[C][2], gB[C][2], tA[C][2], tB[C][2];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      gA[j][0] = u[j][1] - u[j][0];
      gA[j][1] = u[j][3] - u[j][1];
      gB[j][0] = u[j][3] - u[j][2];
      gB[j][1] = u[j][2] - u[j][0];
    }
    contract(gA, T(1), tA, 3);
    contract(gB, T(1), tB, 3);
    if constexpr (HAS_E) {
#pragma unroll
      for (int j = 0; j < C; ++j)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          tA[j][i] += T(tau[j * 2 + i]);
          tB[j][i] += T(tau[j * 2 + i]);
        }
    }
#pragma unroll
    for (int j = 0; j < C; ++j)
#pragma unroll
      for (int i = 0; i < 2; ++i) t1o[j][i] = tA[j][i] + tB[j][i];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      f[j][0] = -tA[j][0] - tB[j][1];
      f[j][1] = tA[j][0] - tA[j][1];
      f[j][2] = tB[j][1] - tB[j][0];
      f[j][3] = tA[j][1] + tB[j][0];
    }
  } else {
    // Q1: modal q1 (xi), q2 (eta), q3 (xi eta); monomials 1: (q1, q2), xi: (0, q3), eta: (q3, 0)
    T g1[C][2], gx[C][2], gy[C][2], t1[C][2], tx[C][2], ty[C][2];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const T s0 = u[j][1] + u[j][0], d0 = u[j][1] - u[j][0];
      const T s1 = u[j][3] + u[j][2], d1 = u[j][3] - u[j][2];
      const T q1 = d1 + d0, q2 = s1 - s0, q3 = d1 - d0;
      g1[j][0] = q1; g1[j][1] = q2;
      gx[j][0] = T(0); gx[j][1] = q3;
      gy[j][0] = q3; gy[j][1] = T(0);
    }
    constexpr double third = 1.0 / 3.0;
    contract(g1, T(1), t1, 3);
    contract(gx, T(third), tx, 2);
    contract(gy, T(third), ty, 1);
    if constexpr (HAS_E) {
#pragma unroll
      for (int j = 0; j < C; ++j)
#pragma unroll
        for (int i = 0; i < 2; ++i) t1[j][i] += T(tau[j * 2 + i]);
    }
#pragma unroll
    for (int j = 0; j < C; ++j)
#pragma unroll
      for (int i = 0; i < 2; ++i) t1o[j][i] = t1[j][i];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const T Q1 = t1[j][0], Q2 = t1[j][1], Q3 = tx[j][1] + ty[j][0];
      // transposed: d0 = Q1 - Q3, d1 = Q1 + Q3, s0 = -Q2, s1 = Q2
      const T d0 = Q1 - Q3, d1 = Q1 + Q3, s0 = -Q2, s1 = Q2;
      f[j][0] = s0 - d0;
      f[j][1] = s0 + d0;
      f[j][2] = s1 - d1;
      f[j][3] = s1 + d1;
    }
  }
}

constexpr int BY2 = 8;  // 2-D tile: BX x BY2 nodes
constexpr int PY2 = BY2 + 2, EY2 = BY2 + 1, NE2 = EX * EY2, NT2 = ((NE2 + 31) / 32) * 32;

template <typename T, int C, int ELEM, bool HAS_X, bool HAS_E, int RED>
__global__ void __launch_bounds__(NT2) pixel_apply_kernel(StencilArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* pl = reinterpret_cast<T*>(smem_raw);  // [C][PY2][PX]
  T* F = pl + C * PY2 * PX;                // [4][C][EY2][EX]
  __shared__ double red_sh[32];
  const Dims d = a.d;
  const int load = blockIdx.z;
  if (RED == RED_PCG && a.st != nullptr && a.st[load].state != ST_RUN) return;
  const int tiles_x = (d.nx + BX - 1) / BX;
  const int i0 = (blockIdx.x % tiles_x) * BX;
  const int j0 = (blockIdx.x / tiles_x) * BY2;
  const int tid = threadIdx.x;
  const T* x = HAS_X ? reinterpret_cast<const T*>(a.x) + (long long)load * a.load_stride : nullptr;
  T* y = reinterpret_cast<T*>(a.y) + (long long)load * a.load_stride;
  const T* mats = reinterpret_cast<const T*>(a.mats);
  const double* tau = HAS_E ? a.tau + (long long)load * a.n_phases * (2 * C) : nullptr;
  if (HAS_X) {
    for (int idx = tid; idx < C * PY2 * PX; idx += NT2) {
      const int px = idx % PX, py = (idx / PX) % PY2, j = idx / (PX * PY2);
      pl[idx] = x[(long long)j * d.N + (long long)wrap(j0 - 1 + py, d.ny) * d.nx + wrap(i0 - 1 + px, d.nx)];
    }
  }
  __syncthreads();
  const int ei = tid % EX, ej = tid / EX;
  double acc_t[2 * C];
#pragma unroll
  for (int i = 0; i < 2 * C; ++i) acc_t[i] = 0.0;
  if (tid < NE2) {
    T u[C][4];
#pragma unroll
    for (int j = 0; j < C; ++j)
#pragma unroll
      for (int cn = 0; cn < 4; ++cn)
        u[j][cn] = HAS_X ? pl[(j * PY2 + ej + (cn >> 1)) * PX + ei + (cn & 1)] : T(0);
    const int ph = a.ids ? a.ids[(long long)wrap(j0 - 1 + ej, d.ny) * d.nx + wrap(i0 - 1 + ei, d.nx)] : 0;
    T f[C][4], t1[C][2];
    pixel_element<T, C, ELEM, HAS_E>(u, mats + (long long)ph * (4 * C * C), HAS_E ? tau + ph * (2 * C) : nullptr, f, t1);
#pragma unroll
    for (int j = 0; j < C; ++j)
#pragma unroll
      for (int cn = 0; cn < 4; ++cn) F[((cn * C + j) * EY2 + ej) * EX + ei] = f[j][cn];
    if ((RED == RED_STATS || RED == RED_SUMS) && ei >= 1 && ej >= 1 && i0 + ei - 1 < d.nx && j0 + ej - 1 < d.ny) {
#pragma unroll
      for (int j = 0; j < C; ++j)
#pragma unroll
        for (int i = 0; i < 2; ++i) acc_t[j * 2 + i] += (double)t1[j][i];
    }
  }
  __syncthreads();
  DotAcc<T> acc_p;
  double acc_y = 0.0;
  const int ni = tid % BX, nj = tid / BX;
  if (tid < BX * BY2 && i0 + ni < d.nx && j0 + nj < d.ny) {
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const T v = F[((3 * C + j) * EY2 + nj) * EX + ni] + F[((2 * C + j) * EY2 + nj) * EX + ni + 1] +
                  F[((1 * C + j) * EY2 + nj + 1) * EX + ni] + F[((0 * C + j) * EY2 + nj + 1) * EX + ni + 1];
      const T val = T(a.y_scale) * v;
      if (RED != RED_SUMS) y[(long long)j * d.N + (long long)(j0 + nj) * d.nx + i0 + ni] = val;
      if (RED == RED_PCG) acc_p.add(val, pl[(j * PY2 + nj + 1) * PX + ni + 1]);
      if ((RED == RED_STATS || RED == RED_SUMS)) acc_y += (double)val * (double)val;
    }
  }
  if (RED == RED_PCG) {
    const double part = block_sum(acc_p.value(), red_sh);
    double total;
    if (finish_reduction(part, a.red.partial + (long long)load * a.red.max_blocks, a.red.count + load,
                         gridDim.x, blockIdx.x, red_sh, &total)) {
      if (threadIdx.x == 0)
        pcg_alpha_update(a.st[load], total, a.red.hist ? a.red.hist + (long long)load * 2 * kHist : nullptr);
    }
  }
  if ((RED == RED_STATS || RED == RED_SUMS)) {
    double* out = a.stats + ((long long)load * gridDim.x + blockIdx.x) * (1 + 2 * C);
    const double ty = block_sum(acc_y, red_sh);
    if (threadIdx.x == 0) out[0] = ty;
#pragma unroll
    for (int i = 0; i < 2 * C; ++i) {
      const double t = block_sum(acc_t[i], red_sh);
      if (threadIdx.x == 0) out[1 + i] = t;
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Two-node stencil (Fig. 3 c, P1TRI4_2D, scalar): per pixel a corner node (type 0, field block 0)
// and a centre node (type 1, block 1), four P1 triangles (edge, centre) with w = V_p / 4 each.
// Scaled gradients G = (h_x g_x, h_y g_y) of the bottom, right, top and left triangles:
//   b: (u10 - u00, 2 uO - u00 - u10)   r: (u10 + u11 - 2 uO, u11 - u10)
//   t: (u11 - u01, u01 + u11 - 2 uO)   l: (2 uO - u00 - u01, u01 - u00)
// dual t_T = Chat G_T + tau (Chat = w S C S, S = diag(1 / h)), forces f_a = sum_T (dG_T / du_a) . t_T.
// ------------------------------------------------------------------------------------------------
template <typename T, bool HAS_E>
__device__ __forceinline__ void pixel4_element(const T (&u)[4], T uO, const T* __restrict__ Ch,
                                               const double* __restrict__ tau, T (&f)[4], T& fO, T (&t1o)[2]) {
  const T G[4][2] = {{u[1] - u[0], T(2) * uO - u[0] - u[1]},
                     {u[1] + u[3] - T(2) * uO, u[3] - u[1]},
                     {u[3] - u[2], u[2] + u[3] - T(2) * uO},
                     {T(2) * uO - u[0] - u[2], u[2] - u[0]}};
  const T c00 = __ldg(Ch + 0), c01 = __ldg(Ch + 1), c10 = __ldg(Ch + 2), c11 = __ldg(Ch + 3);
  T t[4][2];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    t[q][0] = fma(c00, G[q][0], c01 * G[q][1]);
    t[q][1] = fma(c10, G[q][0], c11 * G[q][1]);
    if constexpr (HAS_E) {
      t[q][0] += T(tau[0]);
      t[q][1] += T(tau[1]);
    }
  }
  t1o[0] = t[0][0] + t[1][0] + t[2][0] + t[3][0];
  t1o[1] = t[0][1] + t[1][1] + t[2][1] + t[3][1];
  // corners 0 = (0,0), 1 = (1,0), 2 = (0,1), 3 = (1,1)
  f[0] = -t[0][0] - t[0][1] - t[3][0] - t[3][1];
  f[1] = t[0][0] - t[0][1] + t[1][0] - t[1][1];
  f[3] = t[1][0] + t[1][1] + t[2][0] + t[2][1];
  f[2] = -t[2][0] + t[2][1] - t[3][0] + t[3][1];
  fO = T(2) * (t[0][1] - t[1][0] - t[2][1] + t[3][0]);
}

template <typename T, bool HAS_X, bool HAS_E, int RED>
__global__ void __launch_bounds__(NT2) pixel4_apply_kernel(StencilArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* pl = reinterpret_cast<T*>(smem_raw);  // [2 types][PY2][PX]: corner nodes, pixel centres
  T* F = pl + 2 * PY2 * PX;                // [5][EY2][EX]: forces on the 4 corners and the centre
  __shared__ double red_sh[32];
  const Dims d = a.d;
  const int load = blockIdx.z;
  if (RED == RED_PCG && a.st != nullptr && a.st[load].state != ST_RUN) return;
  const int tiles_x = (d.nx + BX - 1) / BX;
  const int i0 = (blockIdx.x % tiles_x) * BX;
  const int j0 = (blockIdx.x / tiles_x) * BY2;
  const int tid = threadIdx.x;
  const T* x = HAS_X ? reinterpret_cast<const T*>(a.x) + (long long)load * a.load_stride : nullptr;
  T* y = reinterpret_cast<T*>(a.y) + (long long)load * a.load_stride;
  const T* mats = reinterpret_cast<const T*>(a.mats);
  const double* tau = HAS_E ? a.tau + (long long)load * a.n_phases * 2 : nullptr;
  if (HAS_X) {
    for (int idx = tid; idx < 2 * PY2 * PX; idx += NT2) {
      const int px = idx % PX, py = (idx / PX) % PY2, j = idx / (PX * PY2);
      pl[idx] = x[(long long)j * d.N + (long long)wrap(j0 - 1 + py, d.ny) * d.nx + wrap(i0 - 1 + px, d.nx)];
    }
  }
  __syncthreads();
  const int ei = tid % EX, ej = tid / EX;
  double acc_t[2] = {0.0, 0.0};
  if (tid < NE2) {
    // element (ei, ej) = pixel (i0 - 1 + ei, j0 - 1 + ej): corners (ei + a, ej + b), centre (ei, ej) of the tile
    T u[4], uO = T(0);
#pragma unroll
    for (int cn = 0; cn < 4; ++cn) u[cn] = HAS_X ? pl[(ej + (cn >> 1)) * PX + ei + (cn & 1)] : T(0);
    if (HAS_X) uO = pl[(PY2 + ej) * PX + ei];
    const int ph = a.ids ? a.ids[(long long)wrap(j0 - 1 + ej, d.ny) * d.nx + wrap(i0 - 1 + ei, d.nx)] : 0;
    T f[4], fO, t1[2];
    pixel4_element<T, HAS_E>(u, uO, mats + (long long)ph * 4, HAS_E ? tau + ph * 2 : nullptr, f, fO, t1);
#pragma unroll
    for (int cn = 0; cn < 4; ++cn) F[(cn * EY2 + ej) * EX + ei] = f[cn];
    F[(4 * EY2 + ej) * EX + ei] = fO;
    if ((RED == RED_STATS || RED == RED_SUMS) && ei >= 1 && ej >= 1 && i0 + ei - 1 < d.nx && j0 + ej - 1 < d.ny) {
      acc_t[0] += (double)t1[0];
      acc_t[1] += (double)t1[1];
    }
  }
  __syncthreads();
  DotAcc<T> acc_p;
  double acc_y = 0.0;
  const int ni = tid % BX, nj = tid / BX;
  if (tid < BX * BY2 && i0 + ni < d.nx && j0 + nj < d.ny) {
    // corner node (i0 + ni, j0 + nj): the four pixels around it; centre of pixel (i0 + ni, j0 + nj): element (ni + 1, nj + 1)
    const T v0 = F[(3 * EY2 + nj) * EX + ni] + F[(2 * EY2 + nj) * EX + ni + 1] + F[(1 * EY2 + nj + 1) * EX + ni] +
                 F[(0 * EY2 + nj + 1) * EX + ni + 1];
    const T v1 = F[(4 * EY2 + nj + 1) * EX + ni + 1];
    const T val0 = T(a.y_scale) * v0, val1 = T(a.y_scale) * v1;
    const long long g = (long long)(j0 + nj) * d.nx + i0 + ni;
    if (RED != RED_SUMS) {
      y[g] = val0;
      y[d.N + g] = val1;
    }
    if (RED == RED_PCG) {
      acc_p.add(val0, pl[(nj + 1) * PX + ni + 1]);
      acc_p.add(val1, pl[(PY2 + nj + 1) * PX + ni + 1]);
    }
    if ((RED == RED_STATS || RED == RED_SUMS)) acc_y += (double)val0 * (double)val0 + (double)val1 * (double)val1;
  }
  if (RED == RED_PCG) {
    const double part = block_sum(acc_p.value(), red_sh);
    double total;
    if (finish_reduction(part, a.red.partial + (long long)load * a.red.max_blocks, a.red.count + load,
                         gridDim.x, blockIdx.x, red_sh, &total)) {
      if (threadIdx.x == 0)
        pcg_alpha_update(a.st[load], total, a.red.hist ? a.red.hist + (long long)load * 2 * kHist : nullptr);
    }
  }
  if ((RED == RED_STATS || RED == RED_SUMS)) {
    double* out = a.stats + ((long long)load * gridDim.x + blockIdx.x) * 3;
    const double ty = block_sum(acc_y, red_sh);
    if (threadIdx.x == 0) out[0] = ty;
    for (int i = 0; i < 2; ++i) {
      const double t = block_sum(acc_t[i], red_sh);
      if (threadIdx.x == 0) out[1 + i] = t;
    }
  }
}

template <typename K>
cudaError_t set_smem(K kern, size_t bytes) {
  if (bytes > 32 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

// hex8 grid: x-y tiles times z slabs times loads.  Each slab recomputes one element layer below it,
// and the CTAs run in waves over the 152 SMs, a CTA's layer time growing with the CTAs sharing its
// SM; the slab depth kz (at least 4 planes) minimises waves x (kz + 1), waves = ceil(CTAs / 152).
template <int BYT>
void hex8_grid(const Dims& d, int n_loads, int* tiles, int* slabs, int* kz) {
  *tiles = ((d.nx + BX - 1) / BX) * ((d.ny + BYT - 1) / BYT);
  const long long cols = (long long)*tiles * max(n_loads, 1);
  long long best = -1;
  int bkz = d.nz;
  for (int sl = 1; sl <= max(1, d.nz / 4); ++sl) {
    const int k = (d.nz + sl - 1) / sl;
    const long long ctas = cols * ((d.nz + k - 1) / k);
    const long long cost = ((ctas + 151) / 152) * (k + 1);
    if (best < 0 || cost < best) {
      best = cost;
      bkz = k;
    }
  }
  *kz = bkz;
  *slabs = (d.nz + bkz - 1) / bkz;
}

// modes: PCG (x, <x, y>), STATS (residual / right-hand side with sums), plain (x and/or e)
// every x tile full and 16-byte aligned rows: the FP32 PCG apply stages node planes with 16-byte copies
bool hex8_wide(const StencilArgs& a) {
  return a.d.nx % BX == 0 && a.d.nx % 4 == 0 && a.load_stride % 4 == 0 &&
         (reinterpret_cast<unsigned long long>(a.x) & 15) == 0;
}

template <typename T, int C, bool ISO, bool HAS_X, bool HAS_E, int RED, int BYT = hex8_default_rows<T>(),
          int STG = STG_CP4>
cudaError_t launch_hex8_t(const StencilArgs& a, int* ctas, cudaStream_t s) {
  const Dims& d = a.d;
  int tiles, slabs, kz;
  hex8_grid<BYT>(d, a.n_loads, &tiles, &slabs, &kz);
  if (ctas) *ctas = tiles * slabs;
  if (RED == RED_PCG && tiles * slabs > a.red.max_blocks) return cudaErrorInvalidConfiguration;
  CUtensorMap map{};
  if constexpr (STG == STG_TMA) {
    // the field of every load as (x, y, component, z): a box lands as [component][row][x], the staged layout
    const unsigned long long dims[4] = {(unsigned long long)d.nx, (unsigned long long)d.ny,
                                        (unsigned long long)C * a.n_loads, (unsigned long long)d.nz};
    const unsigned long long strides[3] = {(unsigned long long)d.nx * sizeof(T), (unsigned long long)d.N * sizeof(T),
                                           (unsigned long long)d.nx * d.ny * sizeof(T)};
    const unsigned box[4] = {RP, BYT + 2, C, 1};
    if (!hex8_wide(a) || !encode_f32_map(&map, a.x, dims, strides, box)) return cudaErrorInvalidValue;
  }
  const size_t smem = sizeof(T) * hex8_smem_elems<T, C, HAS_X, BYT, STG>();
  auto kern = hex8_apply_kernel<T, C, ISO, HAS_X, HAS_E, RED, BYT, STG>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(tiles, slabs, a.n_loads);
  kern<<<grid, Hex8Tile<T, BYT>::NT, smem, s>>>(map, a, kz);
  return cudaGetLastError();
}

template <typename T, bool HAS_X, bool HAS_E, int RED>
cudaError_t launch_pixel4_t(const StencilArgs& a, int* ctas, cudaStream_t s) {
  const Dims& d = a.d;
  const int tiles = ((d.nx + BX - 1) / BX) * ((d.ny + BY2 - 1) / BY2);
  if (ctas) *ctas = tiles;
  if (RED == RED_PCG && tiles > a.red.max_blocks) return cudaErrorInvalidConfiguration;
  const size_t smem = sizeof(T) * (2 * PY2 * PX + 5 * EY2 * EX);
  auto kern = pixel4_apply_kernel<T, HAS_X, HAS_E, RED>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(tiles, 1, a.n_loads);
  kern<<<grid, NT2, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int C, int ELEM, bool HAS_X, bool HAS_E, int RED>
cudaError_t launch_pixel_t(const StencilArgs& a, int* ctas, cudaStream_t s) {
  const Dims& d = a.d;
  const int tiles = ((d.nx + BX - 1) / BX) * ((d.ny + BY2 - 1) / BY2);
  if (ctas) *ctas = tiles;
  if (RED == RED_PCG && tiles > a.red.max_blocks) return cudaErrorInvalidConfiguration;
  const size_t smem = sizeof(T) * (C * PY2 * PX + 4 * C * EY2 * EX);
  auto kern = pixel_apply_kernel<T, C, ELEM, HAS_X, HAS_E, RED>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(tiles, 1, a.n_loads);
  kern<<<grid, NT2, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int C, bool ISO>
cudaError_t dispatch_hex8(const StencilArgs& a, int* ctas, cudaStream_t s) {
  const bool hx = a.x != nullptr, he = a.tau != nullptr;
  if (a.st != nullptr) {
    if (!hx || he) return cudaErrorInvalidValue;
    constexpr int R0 = hex8_default_rows<T>(), R1 = 24 - hex8_default_rows<T>();
    const bool alt = a.tile_rows != 0 && a.tile_rows != R0;
    constexpr bool raw = hex8_raw<T, C, true>();
    const bool wide = raw && hex8_wide(a);
    if ((a.staging == 2 || a.staging == 3) && !wide) return cudaErrorInvalidValue;
    if constexpr (raw) {
      if (wide && a.staging == 3)  // FP32: TMA plane staging
        return alt ? launch_hex8_t<T, C, ISO, true, false, RED_PCG, R1, STG_TMA>(a, ctas, s)
                   : launch_hex8_t<T, C, ISO, true, false, RED_PCG, R0, STG_TMA>(a, ctas, s);
      if (wide && (a.staging == 0 || a.staging == 2))  // FP32: 16-byte cp.async plane staging
        return alt ? launch_hex8_t<T, C, ISO, true, false, RED_PCG, R1, STG_CP16>(a, ctas, s)
                   : launch_hex8_t<T, C, ISO, true, false, RED_PCG, R0, STG_CP16>(a, ctas, s);
    }
    return alt ? launch_hex8_t<T, C, ISO, true, false, RED_PCG, R1>(a, ctas, s)
               : launch_hex8_t<T, C, ISO, true, false, RED_PCG, R0>(a, ctas, s);
  }
  if (a.stats != nullptr && a.y == nullptr) {
    if (hx && he) return launch_hex8_t<T, C, ISO, true, true, RED_SUMS>(a, ctas, s);
    return cudaErrorInvalidValue;
  }
  if (a.stats != nullptr) {
    if (hx && he) return launch_hex8_t<T, C, ISO, true, true, RED_STATS>(a, ctas, s);
    if (he) return launch_hex8_t<T, C, ISO, false, true, RED_STATS>(a, ctas, s);
    return cudaErrorInvalidValue;
  }
  if (hx && he) return launch_hex8_t<T, C, ISO, true, true, RED_NONE>(a, ctas, s);
  if (hx) return launch_hex8_t<T, C, ISO, true, false, RED_NONE>(a, ctas, s);
  if (he) return launch_hex8_t<T, C, ISO, false, true, RED_NONE>(a, ctas, s);
  return cudaErrorInvalidValue;
}

template <typename T, int C, int ELEM>
cudaError_t dispatch_pixel(const StencilArgs& a, int* ctas, cudaStream_t s) {
  const bool hx = a.x != nullptr, he = a.tau != nullptr;
  if (a.st != nullptr) {
    if (!hx || he) return cudaErrorInvalidValue;
    return launch_pixel_t<T, C, ELEM, true, false, RED_PCG>(a, ctas, s);
  }
  if (a.stats != nullptr && a.y == nullptr) {
    if (hx && he) return launch_pixel_t<T, C, ELEM, true, true, RED_SUMS>(a, ctas, s);
    return cudaErrorInvalidValue;
  }
  if (a.stats != nullptr) {
    if (hx && he) return launch_pixel_t<T, C, ELEM, true, true, RED_STATS>(a, ctas, s);
    if (he) return launch_pixel_t<T, C, ELEM, false, true, RED_STATS>(a, ctas, s);
    return cudaErrorInvalidValue;
  }
  if (hx && he) return launch_pixel_t<T, C, ELEM, true, true, RED_NONE>(a, ctas, s);
  if (hx) return launch_pixel_t<T, C, ELEM, true, false, RED_NONE>(a, ctas, s);
  if (he) return launch_pixel_t<T, C, ELEM, false, true, RED_NONE>(a, ctas, s);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t dispatch_pixel4(const StencilArgs& a, int* ctas, cudaStream_t s) {
  const bool hx = a.x != nullptr, he = a.tau != nullptr;
  if (a.st != nullptr) {
    if (!hx || he) return cudaErrorInvalidValue;
    return launch_pixel4_t<T, true, false, RED_PCG>(a, ctas, s);
  }
  if (a.stats != nullptr && a.y == nullptr) {
    if (hx && he) return launch_pixel4_t<T, true, true, RED_SUMS>(a, ctas, s);
    return cudaErrorInvalidValue;
  }
  if (a.stats != nullptr) {
    if (hx && he) return launch_pixel4_t<T, true, true, RED_STATS>(a, ctas, s);
    if (he) return launch_pixel4_t<T, false, true, RED_STATS>(a, ctas, s);
    return cudaErrorInvalidValue;
  }
  if (hx && he) return launch_pixel4_t<T, true, true, RED_NONE>(a, ctas, s);
  if (hx) return launch_pixel4_t<T, true, false, RED_NONE>(a, ctas, s);
  if (he) return launch_pixel4_t<T, false, true, RED_NONE>(a, ctas, s);
  return cudaErrorInvalidValue;
}


// ------------------------------------------------------------------------------------------------
// Refinement residual in double-float arithmetic (hex8 elasticity, isotropic phases, cubic voxels):
//   r_out = r_in - K d,   K d = D^T W C D d  for an FP32 correction field d,
// the element evaluated as in hex8_element_faces (face form, closed-form isotropic duals) on
// double-float values: a value is hi + lo in two floats (about 48 significant bits), so the FP64-
// accurate residual runs on the FP32 pipe, which on GB300 issues 64 times the FP64 rate.  The first
// butterfly stage of the FP32 inputs is exact (TwoSum); later sums and products round once in
// double-float, with an error of order 2^-44 of the operands' magnitudes.  r_in and r_out are FP64
// (r_out may alias r_in); r_out = r_in - (hi + lo) is formed in FP64.  Fused statistics per load and
// CTA: sum r_out^2 and the sums of the monomial-1 duals of d over the CTA's elements (the change of
// |Y| S P^T <sigma>), [load][cta][1 + 9] doubles.  Tiles as the FP32 kernel (32 x 8), one CTA per SM.
// RHS = true: the right-hand side b = -D^T W C e instead (no field; the monomial-1 duals are the
// per-phase prestress tau of the load, given as float pairs [load][phase][9][2]; r_in is not read):
// r_out = b, with sum b^2 and the dual sums (|Y| S P^T <sigma> at zero fluctuation).
// ------------------------------------------------------------------------------------------------
struct __align__(8) DF {
  float h, l;
};
// Knuth's TwoSum: a + b = s + e exactly
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
// Dekker's FastTwoSum (|s| >= |e|): renormalises (s, e)
__device__ __forceinline__ DF df_norm(float s, float e) {
  const float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ DF operator+(DF a, DF b) {
  const DF s = df_two_sum(a.h, b.h);
  return df_norm(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ DF operator-(DF a, DF b) {
  const DF s = df_two_sum(a.h, -b.h);
  return df_norm(s.h, s.l + (a.l - b.l));
}
__device__ __forceinline__ DF operator*(DF a, DF c) {  // the lo x lo term (2^-48) is dropped
  const float p = a.h * c.h;
  float e = fmaf(a.h, c.h, -p);
  e = fmaf(a.h, c.l, e);
  e = fmaf(a.l, c.h, e);
  return df_norm(p, e);
}
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.h + (double)a.l; }

template <bool RHS>
__global__ void __launch_bounds__(Hex8Tile<float, 8>::NT, 2)
    hex8_residual_df_kernel(StencilArgs a, const double* __restrict__ r_in, const float* __restrict__ taudf,
                            int kz_per_cta) {
  constexpr int C = 3, BY = 8, NE = Hex8Tile<float, 8>::NE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DF* FB = reinterpret_cast<DF*>(smem_raw);  // [2 planes][4][C][NE] face butterflies (thread-private)
  DF* FC0 = FB + 2 * 4 * C * NE;             // [2 layers][4 corners][C][NE] face contributions
  __shared__ double red_sh[32];

  const Dims d = a.d;
  const int load = blockIdx.z;
  const int tiles_x = (d.nx + BX - 1) / BX;
  const int i0 = (blockIdx.x % tiles_x) * BX;
  const int j0 = (blockIdx.x / tiles_x) * BY;
  const int k0 = blockIdx.y * kz_per_cta;
  const int k1 = min(k0 + kz_per_cta, d.nz);
  const int tid = threadIdx.x;
  const float* dx = RHS ? nullptr : reinterpret_cast<const float*>(a.x) + (long long)load * a.load_stride;
  const double* rin = RHS ? nullptr : r_in + (long long)load * a.load_stride;
  const float* tload = RHS ? taudf + (long long)load * a.n_phases * 18 : nullptr;
  double* rout = reinterpret_cast<double*>(a.y) + (long long)load * a.load_stride;
  const float* isodf = reinterpret_cast<const float*>(a.iso);  // [phase][16]: 6 constants as (hi, lo)
  const long long plane = (long long)d.nx * d.ny;

  const int ei = tid % EX, ej = tid / EX;
  const bool face_thread = tid < NE;
  const int fi0 = wrap(i0 - 1 + ei, d.nx), fi1 = wrap(i0 + ei, d.nx);
  const int fj0 = wrap(j0 - 1 + ej, d.ny), fj1 = wrap(j0 + ej, d.ny);
  const int off00 = fj0 * d.nx + fi0, off10 = fj0 * d.nx + fi1, off01 = fj1 * d.nx + fi0, off11 = fj1 * d.nx + fi1;
  const bool owner = face_thread && ei >= 1 && ej >= 1 && i0 + ei - 1 < d.nx && j0 + ej - 1 < d.ny;
  const int ni = tid % BX, nj = tid / BX;
  const bool node_thread = tid < BX * BY && (i0 + ni) < d.nx && (j0 + nj) < d.ny;
  const long long node_off = (long long)(j0 + nj) * d.nx + i0 + ni;

  DF carry[C][4];
#pragma unroll
  for (int j = 0; j < C; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) carry[j][q] = {0.0f, 0.0f};
  DF acc_t[3 * C];
#pragma unroll
  for (int i = 0; i < 3 * C; ++i) acc_t[i] = {0.0f, 0.0f};
  double acc_y = 0.0;

  auto next = [&](int z) { return z + 1 == d.nz ? 0 : z + 1; };
  auto faces = [&](int slot, int kz) {  // in-plane butterflies of plane kz (exact first stage)
    if (!RHS && face_thread) {
      const float* xk = dx + (long long)kz * plane;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const float* xj = xk + (long long)j * d.N;
        const float v00 = __ldg(xj + off00), v10 = __ldg(xj + off10), v01 = __ldg(xj + off01), v11 = __ldg(xj + off11);
        const DF s0 = df_two_sum(v10, v00), d0 = df_two_sum(v10, -v00);
        const DF s1 = df_two_sum(v11, v01), d1 = df_two_sum(v11, -v01);
        DF* fb = FB + ((slot * 4) * C + j) * NE + tid;
        fb[0 * C * NE] = s1 + s0;
        fb[1 * C * NE] = s1 - s0;
        fb[2 * C * NE] = d1 + d0;
        fb[3 * C * NE] = d1 - d0;
      }
    }
  };

  // element layer k (planes k: slot cur, k + 1: slot cur ^ 1), then the gather of plane k
  auto layer = [&](int cur, int k, int kzc) {
    faces(cur ^ 1, next(kzc));
    DF* FC = FC0 + cur * 4 * C * NE;
    if (face_thread && RHS) {  // only the prestress: Q1..Q3 = tau of the element's phase, Q4..Q7 = 0
      const int ph = a.ids ? a.ids[(long long)kzc * plane + off00] : 0;
      const float* tp = tload + ph * 18;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const DF Q1 = {tp[6 * j + 0], tp[6 * j + 1]}, Q2 = {tp[6 * j + 2], tp[6 * j + 3]},
                 Q3 = {tp[6 * j + 4], tp[6 * j + 5]};
        const DF ss = carry[j][0] - Q3, sd = Q2 + carry[j][1], ds = Q1 + carry[j][2], dd = carry[j][3];
        carry[j][0] = Q3;
        carry[j][1] = Q2;
        carry[j][2] = Q1;
        carry[j][3] = {0.0f, 0.0f};
        const DF s0 = ss - sd, s1 = ss + sd, d0 = ds - dd, d1 = ds + dd;
        FC[(0 * C + j) * NE + tid] = s0 - d0;
        FC[(1 * C + j) * NE + tid] = s0 + d0;
        FC[(2 * C + j) * NE + tid] = s1 - d1;
        FC[(3 * C + j) * NE + tid] = s1 + d1;
        if (owner && k >= k0) {
          acc_t[j * 3 + 0] = acc_t[j * 3 + 0] + Q1;
          acc_t[j * 3 + 1] = acc_t[j * 3 + 1] + Q2;
          acc_t[j * 3 + 2] = acc_t[j * 3 + 2] + Q3;
        }
      }
    } else if (face_thread) {
      DF q1[C], q2[C], q3[C], q4[C], q5[C], q6[C], q7[C];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const DF b0 = FB[((cur * 4 + 0) * C + j) * NE + tid], t0 = FB[(((cur ^ 1) * 4 + 0) * C + j) * NE + tid];
        const DF b1 = FB[((cur * 4 + 1) * C + j) * NE + tid], t1 = FB[(((cur ^ 1) * 4 + 1) * C + j) * NE + tid];
        const DF b2 = FB[((cur * 4 + 2) * C + j) * NE + tid], t2 = FB[(((cur ^ 1) * 4 + 2) * C + j) * NE + tid];
        const DF b3 = FB[((cur * 4 + 3) * C + j) * NE + tid], t3 = FB[(((cur ^ 1) * 4 + 3) * C + j) * NE + tid];
        q3[j] = t0 - b0;
        q2[j] = t1 + b1;
        q5[j] = t1 - b1;
        q1[j] = t2 + b2;
        q6[j] = t2 - b2;
        q4[j] = t3 + b3;
        q7[j] = t3 - b3;
      }
      const int ph = a.ids ? a.ids[(long long)kzc * plane + off00] : 0;
      const float4 c0 = __ldg(reinterpret_cast<const float4*>(isodf + 16 * ph));
      const float4 c1 = __ldg(reinterpret_cast<const float4*>(isodf + 16 * ph) + 1);
      const float4 c2 = __ldg(reinterpret_cast<const float4*>(isodf + 16 * ph) + 2);
      const DF lam = {c0.x, c0.y}, mu = {c0.z, c0.w}, mu2 = {c1.x, c1.y}, L = {c1.z, c1.w}, M = {c2.x, c2.y},
               K7 = {c2.z, c2.w};
      DF Q1[C], Q2[C], Q3[C], Q4[C], Q5[C], Q6[C], Q7[C];
      const DF lt = lam * ((q1[0] + q2[1]) + q3[2]);
      Q1[0] = mu2 * q1[0] + lt;
      Q2[1] = mu2 * q2[1] + lt;
      Q3[2] = mu2 * q3[2] + lt;
      Q1[1] = Q2[0] = mu * (q1[1] + q2[0]);
      Q1[2] = Q3[0] = mu * (q1[2] + q3[0]);
      Q2[2] = Q3[1] = mu * (q2[2] + q3[1]);
      const DF Ltx = L * (q4[1] + q6[2]), Lty = L * (q4[0] + q5[2]), Ltz = L * (q6[0] + q5[1]);
      const DF sm = (q4[2] + q5[0]) + q6[1];
      Q4[0] = mu * q4[0] + Lty;
      Q4[1] = mu * q4[1] + Ltx;
      Q4[2] = M * (q4[2] + sm);
      Q5[0] = M * (q5[0] + sm);
      Q5[1] = mu * q5[1] + Ltz;
      Q5[2] = mu * q5[2] + Lty;
      Q6[0] = mu * q6[0] + Ltz;
      Q6[1] = M * (q6[1] + sm);
      Q6[2] = mu * q6[2] + Ltx;
#pragma unroll
      for (int j = 0; j < C; ++j) Q7[j] = K7 * q7[j];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        // transposed z part, face total of plane k, transposed in-plane part
        const DF ss = carry[j][0] - Q3[j], sd = (Q2[j] - Q5[j]) + carry[j][1];
        const DF ds = (Q1[j] - Q6[j]) + carry[j][2], dd = (Q4[j] - Q7[j]) + carry[j][3];
        carry[j][0] = Q3[j];
        carry[j][1] = Q2[j] + Q5[j];
        carry[j][2] = Q1[j] + Q6[j];
        carry[j][3] = Q4[j] + Q7[j];
        const DF s0 = ss - sd, s1 = ss + sd, d0 = ds - dd, d1 = ds + dd;
        FC[(0 * C + j) * NE + tid] = s0 - d0;
        FC[(1 * C + j) * NE + tid] = s0 + d0;
        FC[(2 * C + j) * NE + tid] = s1 - d1;
        FC[(3 * C + j) * NE + tid] = s1 + d1;
      }
      if (owner && k >= k0) {
#pragma unroll
        for (int j = 0; j < C; ++j) {
          acc_t[j * 3 + 0] = acc_t[j * 3 + 0] + Q1[j];
          acc_t[j * 3 + 1] = acc_t[j * 3 + 1] + Q2[j];
          acc_t[j * 3 + 2] = acc_t[j * 3 + 2] + Q3[j];
        }
      }
    }
    __syncthreads();
    if (node_thread && k >= k0) {
      const int e00 = nj * EX + ni;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const DF v = ((FC[(3 * C + j) * NE + e00] + FC[(2 * C + j) * NE + e00 + 1]) + FC[(1 * C + j) * NE + e00 + EX]) +
                     FC[(0 * C + j) * NE + e00 + EX + 1];
        const long long gidx = (long long)j * d.N + (long long)kzc * plane + node_off;
        const double rv = (RHS ? 0.0 : rin[gidx]) - df_to_double(v);
        rout[gidx] = rv;
        acc_y = fma(rv, rv, acc_y);
      }
    }
  };

  int kz = wrap(k0 - 1, d.nz);
  faces(0, kz);
  int cur = 0;
  (void)tload;
  for (int k = k0 - 1; k < k1; ++k) {
    layer(cur, k, kz);
    kz = next(kz);
    cur ^= 1;
  }

  const int nblk = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  double* out = a.stats + ((long long)load * nblk + bid) * (1 + 3 * C);
  const double ty = block_sum(acc_y, red_sh);
  if (threadIdx.x == 0) out[0] = ty;
#pragma unroll
  for (int i = 0; i < 3 * C; ++i) {
    const double t = block_sum(df_to_double(acc_t[i]), red_sh);
    if (threadIdx.x == 0) out[1 + i] = t;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_stiffness(const StencilArgs& a, cudaStream_t s, int* ctas) {
  const Dims& d = a.d;
  if (d.elem == HEX8_3D) {
    if (d.c == 1) return a.iso ? dispatch_hex8<T, 1, true>(a, ctas, s) : dispatch_hex8<T, 1, false>(a, ctas, s);
    if (a.iso) return dispatch_hex8<T, 3, true>(a, ctas, s);
    return dispatch_hex8<T, 3, false>(a, ctas, s);
  }
  if (d.elem == P1TRI2_2D)
    return d.c == 1 ? dispatch_pixel<T, 1, P1TRI2_2D>(a, ctas, s) : dispatch_pixel<T, 2, P1TRI2_2D>(a, ctas, s);
  if (d.elem == Q1_2D) return d.c == 1 ? dispatch_pixel<T, 1, Q1_2D>(a, ctas, s) : dispatch_pixel<T, 2, Q1_2D>(a, ctas, s);
  if (d.elem == P1TRI4_2D) return dispatch_pixel4<T>(a, ctas, s);
  return cudaErrorInvalidValue;
}

int stiffness_ctas(const Dims& d, int n_loads) {
  if (d.elem == HEX8_3D) {
    int tiles, slabs, kz;
    hex8_grid<hex8_default_rows<double>()>(d, n_loads, &tiles, &slabs, &kz);
    return tiles * slabs;
  }
  return ((d.nx + BX - 1) / BX) * ((d.ny + BY2 - 1) / BY2);
}

cudaError_t launch_residual_df(const StencilArgs& a, const double* r_in, const float* taudf, cudaStream_t s,
                               int* ctas) {
  const Dims& d = a.d;
  if (d.elem != HEX8_3D || d.c != 3 || a.stats == nullptr) return cudaErrorInvalidValue;
  const bool rhs = taudf != nullptr;
  if (rhs ? false : (a.iso == nullptr || r_in == nullptr || a.x == nullptr)) return cudaErrorInvalidValue;
  int tiles, slabs, kz;
  hex8_grid<8>(d, a.n_loads, &tiles, &slabs, &kz);
  if (ctas) *ctas = tiles * slabs;
  const size_t smem = sizeof(DF) * (size_t)(2 + 2) * 4 * 3 * Hex8Tile<float, 8>::NE;
  auto kern = rhs ? hex8_residual_df_kernel<true> : hex8_residual_df_kernel<false>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(tiles, slabs, a.n_loads), Hex8Tile<float, 8>::NT, smem, s>>>(a, r_in, taudf, kz);
  return cudaGetLastError();
}

int residual_df_ctas(const Dims& d, int n_loads) {
  int tiles, slabs, kz;
  hex8_grid<8>(d, n_loads, &tiles, &slabs, &kz);
  return tiles * slabs;
}

template cudaError_t launch_stiffness<double>(const StencilArgs&, cudaStream_t, int*);
template cudaError_t launch_stiffness<float>(const StencilArgs&, cudaStream_t, int*);

namespace {
__global__ void eig_bounds_kernel(Dims d, const uint8_t* __restrict__ ids, const double* __restrict__ lo,
                                  const double* __restrict__ hi, unsigned long long* hist_lo,
                                  unsigned long long* hist_hi) {
  __shared__ unsigned int hl[256], hh[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hl[i] = hh[i] = 0u;
  __syncthreads();
  const long long plane = (long long)d.nx * d.ny;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < d.N; v += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(v % d.nx), j = (int)((v / d.nx) % d.ny), k = (int)(v / plane);
    int pmin = -1, pmax = -1;
    const int ncorner = d.dim == 3 ? 8 : 4;
    for (int cn = 0; cn < ncorner; ++cn) {
      // the voxel that has this node as its corner (a, b, c)
      const int ii = wrap(i - (cn & 1), d.nx), jj = wrap(j - ((cn >> 1) & 1), d.ny);
      const int kk = d.dim == 3 ? wrap(k - (cn >> 2), d.nz) : 0;
      const int p = ids ? ids[(long long)kk * plane + (long long)jj * d.nx + ii] : 0;
      if (pmin < 0 || lo[p] < lo[pmin]) pmin = p;
      if (pmax < 0 || hi[p] > hi[pmax]) pmax = p;
    }
    atomicAdd(&hl[pmin], 1u);
    atomicAdd(&hh[pmax], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    if (hl[i]) atomicAdd(&hist_lo[i], (unsigned long long)hl[i]);
    if (hh[i]) atomicAdd(&hist_hi[i], (unsigned long long)hh[i]);
  }
}

__global__ void phase_hist_kernel(const uint8_t* ids, long long N, unsigned long long* hist) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x)
    atomicAdd(&h[ids[v]], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}
}  // namespace

cudaError_t launch_eig_bounds(const Dims& d, const uint8_t* ids, const double* lo, const double* hi,
                              unsigned long long* hist_lo, unsigned long long* hist_hi, cudaStream_t s) {
  const int blocks = (int)std::min<long long>(2 * 152, (d.N + 255) / 256);
  eig_bounds_kernel<<<blocks, 256, 0, s>>>(d, ids, lo, hi, hist_lo, hist_hi);
  return cudaGetLastError();
}

cudaError_t launch_phase_histogram(const uint8_t* ids, long long N, unsigned long long* hist, cudaStream_t s) {
  const int blocks = (int)std::min<long long>(2 * 152, (N + 255) / 256);
  phase_hist_kernel<<<blocks, 256, 0, s>>>(ids, N, hist);
  return cudaGetLastError();
}

}  // namespace fehom
