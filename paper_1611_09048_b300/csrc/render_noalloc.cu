// render_noalloc.cu -- isaac_render_noalloc: the frame of isaac_render for
// callers that must not allocate device memory.
//
// isaac_render keeps a per-stream workspace (the frame's compact ray list)
// that it allocates with cudaMalloc on first use and grows on demand.  Some
// in-situ hosts cannot allow that: a simulation such as a particle-in-cell
// code typically reserves almost all device memory for itself at start-up and
// serves every later request from its own pool, so a library-side cudaMalloc
// either fails or fragments memory the simulation counts on; and a host that
// renders from inside its time-step loop may forbid allocation there because
// cudaMalloc can synchronise the whole device.  This entry point runs the very
// same kernels with the ray list in a fixed array compiled into the library
// (static device memory, present on every GPU that loads the library until the
// process exits), so it never allocates or frees anything.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "common.h"
#include "raycast.cuh"

namespace isaac {

// At most this many ray records: the screen rectangle a frame can cover (the
// pixels whose rays may reach the local box) must not exceed it.
constexpr long long kNoAllocMaxRays = 1LL << 18;   // 262,144 records = 12 MiB
constexpr size_t kNoAllocBytes = (size_t)kWsHeader + (size_t)kNoAllocMaxRays * sizeof(RayRec);

// The scratch array: counters (reset by the background kernel of every call)
// followed by the ray list.  Every call shares it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the array's name only stands in for the symbol; kernels need this
// address instead.
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64];
static int g_noalloc_sms[64];

static int noalloc_setup(void **addr, int *sms)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return check_cuda("cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(ISAAC_ENOTSUP, "device ordinal %d beyond 63", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return fail(ISAAC_ECUDA, "cudaGetSymbolAddress of the render scratch failed: %s",
                        cudaGetErrorString(e));
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = 148;
        }
        g_noalloc_sms[dev] = n;
        g_noalloc_addr[dev] = ptr;
    }
    *addr = g_noalloc_addr[dev];
    *sms = g_noalloc_sms[dev];
    return ISAAC_OK;
}

}  // namespace isaac

using namespace isaac;

extern "C" int isaac_render_noalloc(const isaac_source *sources, const isaac_chain *chains,
                                    int32_t n_sources, const float *luts, const float *weights,
                                    const isaac_camera *camera, const isaac_plane *clip,
                                    int32_t n_clip, const isaac_render_opts *opts,
                                    const isaac_framebuffer *fb, void *stream)
{
    clear_error();
    KParams p;
    memset(&p, 0, sizeof p);
    int rc = prepare_frame(camera, clip, n_clip, opts, p);
    if (rc) return rc;
    if (opts->flags & ISAAC_LUTS_HOST)
        return fail(ISAAC_EINVAL, "isaac_render_noalloc reads device LUTs only (host LUTs need "
                                  "the pinned staging isaac_render allocates)");
    int nact = 0;
    unsigned sig = 0;
    bool wide = false;
    rc = prepare_sources(sources, chains, n_sources, luts, weights, opts, p, &nact, &sig, &wide);
    if (rc) return rc;
    rc = prepare_fb(fb, p);
    if (rc) return rc;
    if (p.touched) return fail(ISAAC_ENOTSUP, "the footprint output is not offered here");
    const long long rect = (long long)(p.rx1 - p.rx0) * (long long)(p.ry1 - p.ry0);
    const cudaStream_t st = (cudaStream_t)stream;
    if (nact == 0 || rect == 0) {   // nothing to ray cast: background only, no scratch needed
        p.rx0 = p.rx1 = p.ry0 = p.ry1 = 0;
        p.ctr = nullptr;
        launch_fill(p, st);
        return check_cuda("isaac_render_noalloc launch");
    }
    if (rect > kNoAllocMaxRays)
        return fail(ISAAC_ENOMEM,
                    "the box covers a %dx%d-pixel screen rectangle (%lld pixels); "
                    "isaac_render_noalloc holds at most %lld rays -- use isaac_render or a "
                    "smaller image", p.rx1 - p.rx0, p.ry1 - p.ry0, rect, kNoAllocMaxRays);
    int rl = 1;
    FrameLaunch fn = find_zc(nact, sig, opts->interp, wide, MODE_PLAIN,
                             choose_lanes(rect, opts->lanes_per_ray, zc_corner_bytes(p, nact)), &rl);
    if (!fn) return fail(ISAAC_ENOTSUP, "no kernel for %d sources", nact);
    void *scratch = nullptr;
    int sms = 0;
    rc = noalloc_setup(&scratch, &sms);
    if (rc) return rc;
    p.ctr = static_cast<WsCounters *>(scratch);
    p.rays = reinterpret_cast<RayRec *>(static_cast<char *>(scratch) + kWsHeader);
    p.grab = march_grab();
    launch_fill(p, st);     // also resets the counters left by the previous call
    launch_setup(p, st);
    const long long want = (rect * rl + kMarchThreads - 1) / kMarchThreads;
    fn(p, dim3((unsigned)std::max(1LL, std::min(want, (long long)sms * kMarchBlocksPerSM))), st);
    return check_cuda("isaac_render_noalloc launch");
}
