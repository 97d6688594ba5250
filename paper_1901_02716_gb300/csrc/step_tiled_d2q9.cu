// Instances of the tiled step kernel: D2Q9, every storage type.
#include "step_tiled.cuh"

namespace maclab {
MACLAB_TILED_LAUNCH_DEF
#define D2_ALL(S)                       \
  MACLAB_TILED_INST(kD2Q9, S, 16, 1)    \
  MACLAB_TILED_INST(kD2Q9, S, 32, 1)    \
  MACLAB_TILED_INST(kD2Q9, S, 64, 1)    \
  MACLAB_TILED_INST(kD2Q9, S, 128, 1)   \
  MACLAB_TILED_INST(kD2Q9, S, 256, 1)
D2_ALL(double)
D2_ALL(float)
D2_ALL(__nv_bfloat16)
D2_ALL(__half)
}  // namespace maclab
