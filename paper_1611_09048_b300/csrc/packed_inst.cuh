// packed_inst.cuh -- kernel table of the packed path for one storage format.
// Included by packed_<format>.cu with ISAAC_DT and ISAAC_TABLE defined, so
// the formats compile as separate translation units.
#include "packed.cuh"

namespace isaac {

template <int NACT, unsigned SIG, int DT, int PAD, int INTERP>
static void launch_packed(const KParams &p, dim3 grid, cudaStream_t st)
{
    k_raycast_packed<NACT, SIG, DT, PAD, INTERP><<<grid, 128, 0, st>>>(p);
}

template <int DT, int PAD>
static void launch_pack(const KPack &p, cudaStream_t st)
{
    if constexpr (DT == ISAAC_E4M3) {
        k_pack_e4m3<PAD><<<(unsigned)(p.bx * p.by * p.bz), 512, 0, st>>>(p);
    } else {
        const long long total = (long long)p.px * p.py * p.pz;
        const long long blocks = std::min<long long>((total + 255) / 256, 148LL * 16);
        k_pack<DT, PAD><<<(unsigned)blocks, 256, 0, st>>>(p);
    }
}

#define ISAAC_S(N, S, P) {launch_packed<N, S, ISAAC_DT, P, 0>, launch_packed<N, S, ISAAC_DT, P, 1>}
#define ISAAC_G(N)                                                                          \
    {{launch_packed<N, 0u, ISAAC_DT, 1, 0>, launch_packed<N, 0u, ISAAC_DT, 1, 1>},           \
     {launch_packed<N, 0u, ISAAC_DT, 2, 0>, launch_packed<N, 0u, ISAAC_DT, 2, 1>},           \
     {launch_packed<N, 0u, ISAAC_DT, 4, 0>, launch_packed<N, 0u, ISAAC_DT, 4, 1>},           \
     {launch_packed<N, 0u, ISAAC_DT, 8, 0>, launch_packed<N, 0u, ISAAC_DT, 8, 1>}}

extern const PackedTable ISAAC_TABLE = {
    // order of k_packed_sigs: {1}, {3}, {1,1}, {3,1}, {3,3}, {3,3,1}; pad = next_pow2(ncomp)
    {ISAAC_S(1, 0x1u, 1), ISAAC_S(1, 0x3u, 4), ISAAC_S(2, 0x11u, 2), ISAAC_S(2, 0x31u, 4),
     ISAAC_S(2, 0x33u, 8), ISAAC_S(3, 0x133u, 8)},
    {ISAAC_G(1), ISAAC_G(2), ISAAC_G(3), ISAAC_G(4)},
    {launch_pack<ISAAC_DT, 1>, launch_pack<ISAAC_DT, 2>, launch_pack<ISAAC_DT, 4>,
     launch_pack<ISAAC_DT, 8>},
};

#undef ISAAC_S
#undef ISAAC_G

}  // namespace isaac
