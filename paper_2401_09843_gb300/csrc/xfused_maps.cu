// TMA descriptors for the fused x pass (host code).  cuTensorMapEncodeTiled
// is a driver entry point; it is looked up once through the runtime so the
// library needs no link against the driver library.
#include <cudaTypedefs.h>

#include "ns3d_launch.h"

namespace ns3d {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// FP32 complex array [rows][ncols] viewed as floats [rows][2 ncols]; boxes of
// box_rows rows x kXfusedW complex (the kernel's tile width: its staged slots
// and expected byte counts follow from the same constant)
bool rows_map(CUtensorMap* map, const void* base, long long rows, long long ncols, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc || box_rows < 1 || box_rows > 256) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * ncols), (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ncols * 8)};
  static_assert((2 * kXfusedW * sizeof(float)) % 16 == 0, "TMA box rows: multiples of 16 bytes");
  const cuuint32_t box[2] = {(cuuint32_t)(2 * kXfusedW), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool xfused_make_maps(XFusedMaps* maps, const Geom& g, int B, const void* dq, const void* u0,
                      const void* us) {
  const long long ncols = (long long)g.N * g.h;
  const int H = g.N / 2;
  return rows_map(&maps->dq, dq, (long long)B * 6 * g.P, ncols, H) &&
         rows_map(&maps->u0, u0, (long long)B * 3 * g.N, ncols, H) &&
         rows_map(&maps->us, us, (long long)B * 3 * g.N, ncols, H);
}

}  // namespace ns3d
