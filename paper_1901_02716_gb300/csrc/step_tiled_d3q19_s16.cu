// Instances of the tiled step kernel: D3Q19, BF16 and FP16 storage (FP32 math).
#include "step_tiled.cuh"

namespace maclab {
MACLAB_TILED_LAUNCH_DEF
MACLAB_TILED_INST(kD3Q19, __nv_bfloat16, 32, 6)
MACLAB_TILED_INST(kD3Q19, __nv_bfloat16, 64, 6)
MACLAB_TILED_INST(kD3Q19, __half, 32, 6)
MACLAB_TILED_INST(kD3Q19, __half, 64, 6)
}  // namespace maclab
