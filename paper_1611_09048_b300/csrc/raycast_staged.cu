// raycast_staged.cu -- instantiations of the staged zero-copy march and its
// kernel table (looked up by find_zc for kModeStaged).
#include "common.h"
#include "kernel_table.h"
#include "raycast_staged.cuh"

namespace isaac {

static_assert(kModeStaged > MODE_ISO, "the staged mode follows the march modes");

// kStageWarps warps per block, kStageBlocksPerSM blocks per SM; the LUTs and
// the warps' buffers in dynamic shared memory (52 KB per block).
template <int NACT, unsigned SIG>
static void launch_staged(const KParams &p, dim3 grid, cudaStream_t st)
{
    constexpr int smem = NACT * 256 * (int)sizeof(float4) + kStageWarps * kStageBytes;
    cudaFuncSetAttribute(k_raycast_staged<NACT, SIG, int>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const unsigned want = (grid.x * kMarchThreads + kStageWarps * 32 - 1) / (kStageWarps * 32);
    const unsigned blocks = std::max(1u, std::min(want, (unsigned)(sm_count() * kStageBlocksPerSM)));
    k_raycast_staged<NACT, SIG, int><<<blocks, kStageWarps * 32, smem, st>>>(p);
}

// {nact, sig, interp, rl, wide, mode, launcher}: trilinear, 32-bit offsets,
// one thread per ray; one scalar, and E, B, rho in AoS and component planes.
static const ZcEntry k_entries[] = {
    {1, 0x9u, 1, 1, false, kModeStaged, launch_staged<1, 0x9u>},
    {3, 0x9BBu, 1, 1, false, kModeStaged, launch_staged<3, 0x9BBu>},
    {3, 0x933u, 1, 1, false, kModeStaged, launch_staged<3, 0x933u>},
};

extern const ZcEntry *const k_staged_entries = k_entries;
extern const int k_n_staged_entries = (int)(sizeof(k_entries) / sizeof(k_entries[0]));

}  // namespace isaac
