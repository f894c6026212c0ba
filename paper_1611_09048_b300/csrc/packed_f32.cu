// packed_f32.cu -- packed-path kernels for f32 storage.
#include <algorithm>
#define ISAAC_DT ISAAC_F32
#define ISAAC_TABLE k_packed_f32
#include "packed_inst.cuh"
