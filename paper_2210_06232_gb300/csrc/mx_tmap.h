// Host side of the tensor-copy (TMA) paths: cuTensorMapEncodeTiled from the
// driver, looked up once through the runtime (no link against libcuda).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mx {

inline PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      (void)cudaGetLastError();
  }
  return fn;
}

// Tensor map of rank R over scalars of size es (4: FP32, 8: FP64); dim[0] innermost.
// False when the driver entry is missing or the layout breaks a tensor-copy rule
// (16-byte aligned base and strides; inner box of a multiple of 16 bytes).
inline bool tensor_map(CUtensorMap* m, int es, int R, const void* base, const cuuint64_t* dim, const cuuint32_t* box) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
  if (!enc || R < 1 || R > 5) return false;
  cuuint64_t stride[4];
  cuuint64_t st = (cuuint64_t)es;
  for (int r = 0; r + 1 < R; ++r) {
    st *= dim[r];
    if (st & 15u) return false;
    stride[r] = st;
  }
  if ((((uintptr_t)base) & 15u) || ((box[0] * (cuuint64_t)es) & 15u)) return false;
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  return enc(m, dt, (cuuint32_t)R, const_cast<void*>(base), dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace mx
