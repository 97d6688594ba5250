// step_fold_s16.cu -- instances of the folded D3Q19 step for BF16 and FP16
// storage (FP32 arithmetic), in their own translation unit so they compile in
// parallel with the FP32 ones.

#include "step_fold.cuh"

namespace maclab {

namespace {

template <typename S>
cudaError_t dispatch_t(const FoldShape& s, const TiledArgs& ta, const void* in, void* out, cudaStream_t st,
                       dim3 grid, int* resident) {
  switch (s.bxc * 100 + s.ty) {
    case 3208: return launch_fold_shape<S, 32, 8>(ta, in, out, st, grid, resident);
    case 3204: return launch_fold_shape<S, 32, 4>(ta, in, out, st, grid, resident);
    case 6404: return launch_fold_shape<S, 64, 4>(ta, in, out, st, grid, resident);
    case 12804: return launch_fold_shape<S, 128, 4>(ta, in, out, st, grid, resident);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t fold_dispatch_s16(int precision, const FoldShape& s, const TiledArgs& ta, const void* in,
                              void* out, cudaStream_t st, dim3 grid, int* resident) {
  if (precision == MACLAB_BF16_STORE) return dispatch_t<__nv_bfloat16>(s, ta, in, out, st, grid, resident);
  if (precision == MACLAB_F16_STORE) return dispatch_t<__half>(s, ta, in, out, st, grid, resident);
  return cudaErrorInvalidValue;
}

}  // namespace maclab
