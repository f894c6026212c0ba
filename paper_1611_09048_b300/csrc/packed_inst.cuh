// packed_inst.cuh -- kernel table of the packed path for one storage format.
// Included by packed_<format>.cu with ISAAC_DT and ISAAC_TABLE defined, so
// the formats compile as separate translation units.
#include "common.h"
#include "packed.cuh"

namespace isaac {

template <int NACT, unsigned SIG, int DT, int PAD, int INTERP, int RL, bool LONG>
static void launch_packed(const KParams &p, dim3 grid, cudaStream_t st)
{
    k_raycast_packed<NACT, SIG, DT, PAD, INTERP, RL, LONG><<<grid, kMarchThreads, 0, st>>>(p);
}

template <int DT, int PAD>
static void launch_pack(const KPack &p, cudaStream_t st)
{
    if constexpr (DT == ISAAC_E4M3) {
        const long long gx = (p.bx + kPackBricksX - 1) / kPackBricksX;
        k_pack_e4m3<PAD><<<(unsigned)(gx * p.by * p.bz), 256, 0, st>>>(p);
    } else {
        const long long rows = (long long)p.py * p.pz;   // a warp per row, 8 per block
        const long long blocks = std::min<long long>((rows + 7) / 8, (long long)sm_count() * 16);
        k_pack<DT, PAD><<<(unsigned)blocks, 256, 0, st>>>(p);
    }
}

// {nact, sig, pad, interp, rl, long, launcher}; pad of a specialised signature
// is next_pow2(component total), the generic kernels use pad 8.  The long-ray
// marches (a warp per ray) exist for every layout a proposal can meet.
#define ISAAC_E(N, S, P, I, R) {N, S, P, I, R, false, launch_packed<N, S, ISAAC_DT, P, I, R, false>}
#define ISAAC_E2(N, S, P, R) ISAAC_E(N, S, P, 0, R), ISAAC_E(N, S, P, 1, R)
#define ISAAC_L(N, S, P, I) {N, S, P, I, 32, true, launch_packed<N, S, ISAAC_DT, P, I, 32, true>}
#define ISAAC_L2(N, S, P) ISAAC_L(N, S, P, 0), ISAAC_L(N, S, P, 1)
static const PackedEntry k_entries[] = {
    ISAAC_E2(1, 0x1u, 1, 1), ISAAC_E2(1, 0x1u, 1, 2), ISAAC_E2(1, 0x1u, 1, 4),
    ISAAC_E2(1, 0x1u, 1, 8), ISAAC_E2(1, 0x1u, 1, 16),
    ISAAC_E2(1, 0x3u, 4, 2), ISAAC_E2(2, 0x11u, 2, 2), ISAAC_E2(2, 0x31u, 4, 2),
    ISAAC_E2(2, 0x33u, 8, 2),
    ISAAC_E2(3, 0x133u, 8, 1), ISAAC_E2(3, 0x133u, 8, 2), ISAAC_E2(3, 0x133u, 8, 4),
    ISAAC_E2(3, 0x133u, 8, 8), ISAAC_E2(3, 0x133u, 8, 16),
    ISAAC_E2(1, 0u, 8, 2), ISAAC_E2(2, 0u, 8, 2), ISAAC_E2(3, 0u, 8, 2), ISAAC_E2(4, 0u, 8, 2),
    ISAAC_L2(1, 0x1u, 1), ISAAC_L2(1, 0x3u, 4), ISAAC_L2(2, 0x11u, 2), ISAAC_L2(2, 0x31u, 4),
    ISAAC_L2(2, 0x33u, 8), ISAAC_L2(3, 0x133u, 8),
    ISAAC_L2(1, 0u, 8), ISAAC_L2(2, 0u, 8), ISAAC_L2(3, 0u, 8), ISAAC_L2(4, 0u, 8),
};
#undef ISAAC_L2
#undef ISAAC_L
#undef ISAAC_E2
#undef ISAAC_E

extern const PackedTable ISAAC_TABLE = {
    k_entries, (int)(sizeof(k_entries) / sizeof(k_entries[0])),
    {launch_pack<ISAAC_DT, 1>, launch_pack<ISAAC_DT, 2>, launch_pack<ISAAC_DT, 4>,
     launch_pack<ISAAC_DT, 8>},
};

}  // namespace isaac
