// Instances of the tiled step kernel: D3Q19, FP32 storage (the main path).
#include "step_tiled.cuh"

namespace maclab {
MACLAB_TILED_LAUNCH_DEF
MACLAB_TILED_INST(kD3Q19, float, 32, 6)
MACLAB_TILED_INST(kD3Q19, float, 32, 10)
}  // namespace maclab
