// packed_bf16.cu -- packed-path kernels for bf16 storage.
#include <algorithm>
#define ISAAC_DT ISAAC_BF16
#define ISAAC_TABLE k_packed_bf16
#include "packed_inst.cuh"
