// packed_e4m3.cu -- packed-path kernels for e4m3 storage.
#include <algorithm>
#define ISAAC_DT ISAAC_E4M3
#define ISAAC_TABLE k_packed_e4m3
#include "packed_inst.cuh"
