// step_rows2_s16.cu -- the two-rows-per-thread D3Q19 step for BF16 and FP16
// storage (FP32 arithmetic); a translation unit of its own so the build
// compiles it in parallel with the FP32 instances.

#include "step_rows2.cuh"

namespace maclab {

template <typename S>
cudaError_t rows2_dispatch(int bxc, int tyt, const TiledArgs& ta, const void* in, void* out,
                           const CUtensorMap& tm_own, const CUtensorMap& tm_halo, cudaStream_t st, dim3 grid,
                           int* resident) {
  switch (bxc * 100 + tyt) {
    case 1604: return launch_rows2_shape<S, 16, 4>(ta, in, out, tm_own, tm_halo, st, grid, resident);
    case 3204: return launch_rows2_shape<S, 32, 4>(ta, in, out, tm_own, tm_halo, st, grid, resident);
  }
  return cudaErrorInvalidValue;
}
template cudaError_t rows2_dispatch<__nv_bfloat16>(int, int, const TiledArgs&, const void*, void*,
                                                  const CUtensorMap&, const CUtensorMap&, cudaStream_t, dim3, int*);
template cudaError_t rows2_dispatch<__half>(int, int, const TiledArgs&, const void*, void*, const CUtensorMap&,
                                           const CUtensorMap&, cudaStream_t, dim3, int*);


}  // namespace maclab
