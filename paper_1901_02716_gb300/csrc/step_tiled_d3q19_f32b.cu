// Instances of the tiled step kernel: D3Q19, FP32 storage, other widths.
#include "step_tiled.cuh"

namespace maclab {
MACLAB_TILED_LAUNCH_DEF
MACLAB_TILED_INST(kD3Q19, float, 16, 10)
MACLAB_TILED_INST(kD3Q19, float, 64, 6)
MACLAB_TILED_INST(kD3Q19, float, 128, 4)
}  // namespace maclab
