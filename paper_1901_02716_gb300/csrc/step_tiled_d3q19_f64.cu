// Instances of the tiled step kernel: D3Q19, FP64 storage.
#include "step_tiled.cuh"

namespace maclab {
MACLAB_TILED_LAUNCH_DEF
MACLAB_TILED_INST(kD3Q19, double, 16, 10)
MACLAB_TILED_INST(kD3Q19, double, 32, 6)
}  // namespace maclab
