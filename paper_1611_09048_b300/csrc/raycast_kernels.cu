// raycast_kernels.cu -- instantiations of the zero-copy frame kernel and the
// table the host dispatches from.
#include "common.h"
#include "kernel_table.h"
#include "raycast.cuh"

namespace isaac {

template <int NACT, unsigned SIG, int INTERP, typename Idx, int RL, int MODE>
static void launch_zc(const KParams &p, dim3 grid, cudaStream_t st)
{
    k_raycast<NACT, SIG, INTERP, Idx, RL, MODE><<<grid, kMarchThreads, 0, st>>>(p);
}

// {nact, sig, interp, rl, wide, mode, launcher}
#define ISAAC_Z(N, S, I, R, W, M) \
    {N, S, I, R, W, M, launch_zc<N, S, I, std::conditional_t<W, long long, int>, R, M>}
#define ISAAC_Z2(N, S, R, W, M) ISAAC_Z(N, S, 0, R, W, M), ISAAC_Z(N, S, 1, R, W, M)
// Precompiled source signatures (Sec. 3.2 compiles the source loop for the
// application's source list): one scalar; E, B, rho in AoS and in component
// planes.  Anything else runs the generic kernel with run-time f_dim.
static const ZcEntry k_entries[] = {
    ISAAC_Z2(1, 0x9u, 1, false, MODE_PLAIN), ISAAC_Z2(1, 0x9u, 2, false, MODE_PLAIN),
    ISAAC_Z2(1, 0x9u, 4, false, MODE_PLAIN), ISAAC_Z2(1, 0x9u, 8, false, MODE_PLAIN),
    ISAAC_Z2(1, 0x9u, 16, false, MODE_PLAIN),
    ISAAC_Z2(3, 0x9BBu, 1, false, MODE_PLAIN), ISAAC_Z2(3, 0x9BBu, 2, false, MODE_PLAIN),
    ISAAC_Z2(3, 0x9BBu, 4, false, MODE_PLAIN), ISAAC_Z2(3, 0x9BBu, 8, false, MODE_PLAIN),
    ISAAC_Z2(3, 0x9BBu, 16, false, MODE_PLAIN),
    ISAAC_Z2(3, 0x933u, 4, false, MODE_PLAIN),
    ISAAC_Z2(1, 0u, 4, false, MODE_PLAIN), ISAAC_Z2(2, 0u, 4, false, MODE_PLAIN),
    ISAAC_Z2(3, 0u, 4, false, MODE_PLAIN), ISAAC_Z2(4, 0u, 4, false, MODE_PLAIN),
    ISAAC_Z2(1, 0u, 4, true, MODE_PLAIN), ISAAC_Z2(2, 0u, 4, true, MODE_PLAIN),
    ISAAC_Z2(3, 0u, 4, true, MODE_PLAIN), ISAAC_Z2(4, 0u, 4, true, MODE_PLAIN),
    ISAAC_Z2(1, 0u, 1, false, MODE_TOUCH), ISAAC_Z2(2, 0u, 1, false, MODE_TOUCH),
    ISAAC_Z2(3, 0u, 1, false, MODE_TOUCH), ISAAC_Z2(4, 0u, 1, false, MODE_TOUCH),
    ISAAC_Z2(1, 0u, 4, false, MODE_LABEL), ISAAC_Z2(2, 0u, 4, false, MODE_LABEL),
    ISAAC_Z2(3, 0u, 4, false, MODE_LABEL), ISAAC_Z2(4, 0u, 4, false, MODE_LABEL),
    // iso surfaces
    ISAAC_Z2(1, 0x9u, 4, false, MODE_ISO), ISAAC_Z2(3, 0x9BBu, 4, false, MODE_ISO),
    ISAAC_Z2(1, 0u, 4, false, MODE_ISO), ISAAC_Z2(2, 0u, 4, false, MODE_ISO),
    ISAAC_Z2(3, 0u, 4, false, MODE_ISO), ISAAC_Z2(4, 0u, 4, false, MODE_ISO),
    // marches with empty-space skipping
    ISAAC_Z2(1, 0x9u, 4, false, MODE_SKIP), ISAAC_Z2(3, 0x9BBu, 8, false, MODE_SKIP),
    ISAAC_Z2(1, 0u, 4, false, MODE_SKIP), ISAAC_Z2(2, 0u, 4, false, MODE_SKIP),
    ISAAC_Z2(3, 0u, 4, false, MODE_SKIP), ISAAC_Z2(4, 0u, 4, false, MODE_SKIP),
    // long-ray marches (after an interval proposal): a warp per ray
    ISAAC_Z2(1, 0x9u, 32, false, MODE_LONG), ISAAC_Z2(3, 0x9BBu, 32, false, MODE_LONG),
    ISAAC_Z2(3, 0x933u, 32, false, MODE_LONG),
    ISAAC_Z2(1, 0u, 32, false, MODE_LONG), ISAAC_Z2(2, 0u, 32, false, MODE_LONG),
    ISAAC_Z2(3, 0u, 32, false, MODE_LONG), ISAAC_Z2(4, 0u, 32, false, MODE_LONG),
    ISAAC_Z2(1, 0u, 32, true, MODE_LONG), ISAAC_Z2(2, 0u, 32, true, MODE_LONG),
    ISAAC_Z2(3, 0u, 32, true, MODE_LONG), ISAAC_Z2(4, 0u, 32, true, MODE_LONG),
};
#undef ISAAC_Z2
#undef ISAAC_Z

extern const ZcEntry *const k_zc_entries = k_entries;
extern const int k_n_zc_entries = (int)(sizeof(k_entries) / sizeof(k_entries[0]));

// The setup, background and copy kernels are launched from this translation unit.
// Two fill blocks per SM leave room for the setup blocks that start beside them.
void launch_fill(const KParams &p, cudaStream_t st)
{
    const int blocks = std::max(1, std::min(p.H, sm_count() * 2));
    k_fill_background<<<blocks, 256, 0, st>>>(p);
}

// The setup is a programmatic dependent launch of the fill before it in the
// stream: its blocks may start once every fill block has started, and wait in
// the kernel (griddepcontrol.wait) for the fill's completion before they write.
void launch_setup(const KParams &p, cudaStream_t st)
{
    const int tiles = ((p.rx1 - p.rx0 + 15) / 16) * ((p.ry1 - p.ry0 + 7) / 8);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)tiles);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_setup_rays, p);
}

void launch_copy_rays(const KParams &p, RayRec *out, long long cap, int *count, cudaStream_t st)
{
    const long long blocks = std::max(1LL, std::min<long long>((cap + 255) / 256, 148LL * 4));
    k_copy_rays<<<(unsigned)blocks, 256, 0, st>>>(p, out, cap, count);
}

}  // namespace isaac
