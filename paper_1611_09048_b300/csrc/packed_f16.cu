// packed_f16.cu -- packed-path kernels for f16 storage.
#include <algorithm>
#define ISAAC_DT ISAAC_F16
#define ISAAC_TABLE k_packed_f16
#include "packed_inst.cuh"
