// step_rows2_nu.cu -- the two-rows-per-thread D3Q19 kernel in its viscosity-term
// mode (FP32 storage); a translation unit of its own so the build compiles it
// in parallel with the step instances.

#include "step_rows2.cuh"

namespace maclab {

cudaError_t rows2_nu_dispatch(int bxc, int tyt, const TiledArgs& ta, const void* in, const void* out,
                              const CUtensorMap& tm_own, const CUtensorMap& tm_halo, cudaStream_t st, dim3 grid,
                              int* resident) {
  void* o = const_cast<void*>(out);  // read only in this mode
  switch (bxc * 100 + tyt) {
    case 1604: return launch_rows2_shape<float, 16, 4, true>(ta, in, o, tm_own, tm_halo, st, grid, resident);
    case 3202: return launch_rows2_shape<float, 32, 2, true>(ta, in, o, tm_own, tm_halo, st, grid, resident);
    case 3204: return launch_rows2_shape<float, 32, 4, true>(ta, in, o, tm_own, tm_halo, st, grid, resident);
  }
  return cudaErrorInvalidValue;
}

}  // namespace maclab
