// Host side of the Tensor Memory Accelerator helpers (tma.cuh): cuTensorMapEncodeTiled is looked up from
// the driver once, so the library does not link against libcuda.
#include "tma.cuh"

#include <cudaTypedefs.h>

#include <mutex>

namespace fehom {
namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}
}  // namespace

bool tma_available() { return encode_fn() != nullptr; }

bool encode_f32_map(CUtensorMap* map, const void* base, const unsigned long long dims[4],
                    const unsigned long long strides[3], const unsigned box[4]) {
  auto fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  cuuint64_t gd[4], gs[3];
  cuuint32_t bx[4];
  const cuuint32_t es[4] = {1, 1, 1, 1};
  for (int i = 0; i < 4; ++i) {
    gd[i] = dims[i];
    bx[i] = box[i];
  }
  for (int i = 0; i < 3; ++i) {
    if (strides[i] % 16 != 0) return false;
    gs[i] = strides[i];
  }
  if ((box[0] * 4) % 16 != 0) return false;
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), gd, gs, bx, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace fehom
