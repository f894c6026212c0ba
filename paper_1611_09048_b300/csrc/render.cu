// render.cu -- isaac_render: source validation, kernel selection by source
// signature and lanes per ray, the per-stream workspace and the three-kernel
// frame launch.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.h"
#include "raycast.cuh"

namespace isaac {

// ------------------------------------------------------------ workspace

// One workspace per (device, stream): counters + one ray record per pixel of
// the largest screen rectangle seen on that stream.  Frames on one stream are
// ordered, so they can share it; different streams never do.
struct Workspace {
    int device;
    cudaStream_t stream;
    void *ptr;
    size_t bytes;
};
static std::mutex g_ws_mu;
static std::vector<Workspace> g_ws;

// Device copies of host LUTs (ISAAC_LUTS_HOST) sit at the end of the workspace.
constexpr size_t kWsLutBytes = (size_t)ISAAC_MAX_ACTIVE * 256 * sizeof(float4);

// Host LUTs go through a ring of pinned slots per (device, stream): the call
// copies them into the next slot on the host, then the slot to the workspace
// on the stream; an event per slot tells when the slot may be refilled.
constexpr int kLutSlots = 8;
struct LutStage {
    int device;
    cudaStream_t stream;
    float4 *host;                 // kLutSlots * ISAAC_MAX_ACTIVE * 256 pinned entries
    cudaEvent_t done[kLutSlots];
    bool used[kLutSlots];
    int next;
};
static std::vector<LutStage> g_lut_stage;   // guarded by g_ws_mu

static int stage_host_luts(KParams &p, float4 *dev_luts, int nact, int dev, cudaStream_t st)
{
    LutStage *g = nullptr;
    for (LutStage &e : g_lut_stage)
        if (e.device == dev && e.stream == st) g = &e;
    if (!g) {
        LutStage e{};
        e.device = dev;
        e.stream = st;
        if (cudaHostAlloc(reinterpret_cast<void **>(&e.host), kLutSlots * kWsLutBytes,
                          cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return fail(ISAAC_ENOMEM, "cannot allocate pinned LUT staging (%zu bytes)",
                        kLutSlots * kWsLutBytes);
        }
        for (int i = 0; i < kLutSlots; ++i) {
            if (cudaEventCreateWithFlags(&e.done[i], cudaEventDisableTiming) != cudaSuccess)
                return check_cuda("LUT staging event");
        }
        g_lut_stage.push_back(e);
        g = &g_lut_stage.back();
    }
    const int slot = g->next;
    g->next = (g->next + 1) % kLutSlots;
    if (g->used[slot] && cudaEventSynchronize(g->done[slot]) != cudaSuccess)
        return check_cuda("LUT staging slot wait");
    float4 *h = g->host + (size_t)slot * ISAAC_MAX_ACTIVE * 256;
    for (int a = 0; a < nact; ++a) memcpy(h + (size_t)a * 256, p.lut[a], 256 * sizeof(float4));
    if (cudaMemcpyAsync(dev_luts, h, (size_t)nact * 256 * sizeof(float4), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
        return check_cuda("LUT upload");
    if (cudaEventRecord(g->done[slot], st) != cudaSuccess) return check_cuda("LUT staging event");
    g->used[slot] = true;
    for (int a = 0; a < nact; ++a) p.lut[a] = dev_luts + (size_t)a * 256;
    p.luts_host = 2;
    return ISAAC_OK;
}

int bind_workspace(KParams &p, cudaStream_t st, size_t extra, void **extra_ptr)
{
    const long long rect = (long long)(p.rx1 - p.rx0) * (long long)(p.ry1 - p.ry0);
    const size_t lists = (size_t)kWsHeader + (size_t)std::max(1LL, rect) * (sizeof(RayRec) + sizeof(unsigned));
    const size_t need = lists + ((extra + 15) & ~(size_t)15) + kWsLutBytes + 256;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return check_cuda("cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_ws_mu);
    Workspace *w = nullptr;
    for (Workspace &e : g_ws)
        if (e.device == dev && e.stream == st) w = &e;
    if (!w) {
        g_ws.push_back({dev, st, nullptr, 0});
        w = &g_ws.back();
    }
    if (w->bytes < need) {
        if (w->ptr) {
            // frames still in flight on this stream may use the old buffer
            if (cudaStreamSynchronize(st) != cudaSuccess) return check_cuda("workspace sync");
            cudaFree(w->ptr);
            w->ptr = nullptr;
            w->bytes = 0;
        }
        const size_t bytes = need + need / 4;
        if (cudaMalloc(&w->ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(ISAAC_ENOMEM, "cannot allocate a %zu-byte render workspace", bytes);
        }
        w->bytes = bytes;
    }
    p.ctr = static_cast<WsCounters *>(w->ptr);
    p.rays = reinterpret_cast<RayRec *>(static_cast<char *>(w->ptr) + kWsHeader);
    p.longs = reinterpret_cast<unsigned *>(p.rays + std::max(1LL, rect));
    if (extra_ptr) *extra_ptr = static_cast<char *>(w->ptr) + lists;
    if (p.luts_host == 1) {
        // the last kWsLutBytes of the block, 256-byte aligned (need reserves the slack)
        const uintptr_t end = reinterpret_cast<uintptr_t>(w->ptr) + w->bytes - kWsLutBytes;
        float4 *dev_luts = reinterpret_cast<float4 *>(end & ~uintptr_t(255));
        int nact = 0;
        while (nact < ISAAC_MAX_ACTIVE && p.lut[nact]) ++nact;
        return stage_host_luts(p, dev_luts, nact, dev, st);
    }
    return ISAAC_OK;
}

int sm_count()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = 148;
        }
        cached[dev] = n;
    }
    return cached[dev];
}

int choose_lanes(long long rect_pixels, int hint, int corner_bytes)
{
    (void)rect_pixels;
    if (hint) return hint;
    // Measured on B300 at 1080p over 512^3: with E, B, rho in FP32 (28 bytes
    // per corner) 1, 2, 4, 8 and 16 lanes per ray give 5.4, 10.0, 13.4, 15.0
    // and 13.7 G samples/s; with 16-bit records (16 bytes) and with one FP32
    // scalar 4 lanes are fastest.  More lanes per ray put more of a warp's
    // gathers on one ray's neighbouring cells, fewer leave more rays in flight.
    return corner_bytes >= 24 ? 8 : 4;
}

int zc_corner_bytes(const KParams &p, int nact)
{
    int b = 0;
    for (int a = 0; a < nact; ++a) b += 4 * p.src[a].fdim;
    return b;
}

bool staging_allowed(const KParams &p, int nact, const isaac_render_opts *opts, bool wide)
{
    if (!(opts->flags & ISAAC_MARCH_STAGED) || opts->interp != 1 || wide || p.touched) return false;
    for (int a = 1; a < nact; ++a)   // one staged box serves every source
        if (p.src[a].lo != p.src[0].lo || p.src[a].hi_pad != p.src[0].hi_pad) return false;
    return true;
}

int march_grab()
{
    static const int env = [] {
        const char *e = getenv("ISAAC_MARCH_GRAB");
        return e ? atoi(e) : 0;
    }();
    return env >= 1 && env <= 64 ? env : 16;
}

// Events recorded around the march kernel of this thread's frames (isaac_time_march).
static thread_local cudaEvent_t t_march_start = nullptr, t_march_stop = nullptr;

int launch_frame_with(KParams &p, FrameLaunch fn, int rl, cudaStream_t st, const FrameHook *hook,
                      FrameLaunch fn_long)
{
    const bool any = fn && p.rx1 > p.rx0 && p.ry1 > p.ry0;
    if (!any) {   // nothing to ray cast: the background covers every pixel
        p.rx0 = p.rx1 = p.ry0 = p.ry1 = 0;
        p.ctr = nullptr;
        launch_fill(p, st);
        return check_cuda("render launch");
    }
    int rc = bind_workspace(p, st);
    if (rc) return rc;
    if (!hook || !fn_long) p.longs = nullptr;   // only a proposal fills the long-ray list
    p.grab = march_grab();
    launch_fill(p, st);
    launch_setup(p, st);
    if (hook) {
        rc = hook->fn(p, hook->arg, st);
        if (rc) return rc;
    }
    const long long rect = (long long)(p.rx1 - p.rx0) * (long long)(p.ry1 - p.ry0);
    const long long want = (rect * rl + kMarchThreads - 1) / kMarchThreads;
    const long long cap = (long long)sm_count() * kMarchBlocksPerSM;
    if (t_march_start) cudaEventRecord(t_march_start, st);
    if (p.longs) fn_long(p, dim3((unsigned)std::max(1LL, std::min(want, cap))), st);
    fn(p, dim3((unsigned)std::max(1LL, std::min(want, cap))), st);
    if (t_march_stop) cudaEventRecord(t_march_stop, st);
    return check_cuda("render launch");
}

// --------------------------------------------------------------- dispatch

FrameLaunch find_zc(int nact, unsigned sig, int interp, bool wide, int mode, int rl,
                    int *rl_used)
{
    const ZcEntry *best = nullptr;
    const bool staged = mode == kModeStaged;
    const ZcEntry *table = staged ? k_staged_entries : k_zc_entries;
    const int n_table = staged ? k_n_staged_entries : k_n_zc_entries;
    for (int pass = 0; pass < 2 && !best; ++pass) {
        const unsigned want = pass == 0 ? sig : 0u;
        for (int i = 0; i < n_table; ++i) {
            const ZcEntry &e = table[i];
            if (e.nact != nact || e.sig != want || e.interp != interp || e.wide != wide ||
                e.mode != mode)
                continue;
            if (!best || (e.rl == rl) || (best->rl != rl && std::abs(e.rl - rl) < std::abs(best->rl - rl)))
                best = &e;
        }
    }
    if (!best) return nullptr;
    *rl_used = best->rl;
    return best->fn;
}

int prepare_sources(const isaac_source *sources, const isaac_chain *chains, int32_t n_sources,
                    const float *luts, const float *weights, const isaac_render_opts *opts,
                    KParams &p, int *nact_out, unsigned *sig_out, bool *wide_out, int reach)
{
    if (!sources || !chains || !weights)
        return fail(ISAAC_EINVAL, "sources, chains and weights are required");
    if (n_sources < 1 || n_sources > ISAAC_MAX_SOURCES)
        return fail(ISAAC_EINVAL, "n_sources %d outside 1..%d", n_sources, ISAAC_MAX_SOURCES);
    if (opts->active_mask >> n_sources)
        return fail(ISAAC_EINVAL, "active_mask 0x%x has bits beyond n_sources %d",
                    opts->active_mask, n_sources);
    int nact = 0;
    unsigned sig = 0;
    bool wide = false;
    for (int s = 0; s < n_sources; ++s) {
        if (!((opts->active_mask >> s) & 1u)) continue;
        if (nact == ISAAC_MAX_ACTIVE)
            return fail(ISAAC_ENOTSUP, "more than %d active sources", ISAAC_MAX_ACTIVE);
        if (!std::isfinite(weights[s])) return fail(ISAAC_EINVAL, "weight %d is not finite", s);
        unsigned nib = 0;
        bool w = false;
        int rc = prepare_source(sources[s], s, opts->n, opts->interp, weights[s], 4, p.src[nact],
                                &nib, &w, reach);
        if (rc) return rc;
        rc = compile_chain(chains[s], sources[s].f_dim, s, p.ch[nact]);
        if (rc) return rc;
        if (!luts) return fail(ISAAC_EINVAL, "luts is NULL");
        if (!(opts->flags & ISAAC_LUTS_HOST) && ((uintptr_t)luts) % 16)
            return fail(ISAAC_EINVAL, "luts must be 16-byte aligned");
        p.lut[nact] = reinterpret_cast<const float4 *>(luts) + (size_t)s * 256;
        sig |= nib << (4 * nact);
        wide |= w;
        ++nact;
    }
    if (opts->flags & ISAAC_LUTS_HOST) p.luts_host = 1;   // staged when the workspace is bound
    *nact_out = nact;
    *sig_out = sig;
    *wide_out = wide;
    return ISAAC_OK;
}

}  // namespace isaac

using namespace isaac;

extern "C" int isaac_render(const isaac_source *sources, const isaac_chain *chains,
                            int32_t n_sources, const float *luts, const float *weights,
                            const isaac_camera *camera, const isaac_plane *clip, int32_t n_clip,
                            const isaac_render_opts *opts, const isaac_framebuffer *fb,
                            void *stream)
{
    clear_error();
    KParams p;
    memset(&p, 0, sizeof p);
    int rc = prepare_frame(camera, clip, n_clip, opts, p);
    if (rc) return rc;
    int nact = 0;
    unsigned sig = 0;
    bool wide = false;
    update_sources(n_sources, opts->active_mask);
    rc = prepare_sources(sources, chains, n_sources, luts, weights, opts, p, &nact, &sig, &wide);
    if (rc) return rc;
    rc = prepare_fb(fb, p);
    if (rc) return rc;
    FrameLaunch fn = nullptr;
    int rl = 1;
    if (nact > 0) {
        const long long rect = (long long)(p.rx1 - p.rx0) * (long long)(p.ry1 - p.ry0);
        if (staging_allowed(p, nact, opts, wide)) fn = find_zc(nact, sig, 1, false, kModeStaged, 1, &rl);
        if (!fn) {
            const int want = p.touched ? 1 : choose_lanes(rect, opts->lanes_per_ray, zc_corner_bytes(p, nact));
            fn = find_zc(nact, sig, opts->interp, wide, p.touched ? MODE_TOUCH : MODE_PLAIN, want, &rl);
        }
        if (!fn)
            return fail(ISAAC_ENOTSUP, "no kernel for %d sources (footprint with 64-bit offsets?)",
                        nact);
    }
    return launch_frame_with(p, fn, rl, (cudaStream_t)stream, nullptr);
}

// The frame of isaac_render in one of the march modes, with an optional hook
// between ray setup and march (the interval proposal).
static int render_mode(const isaac_source *sources, const isaac_chain *chains, int32_t n_sources,
                       const float *luts, const float *weights, const isaac_camera *camera,
                       const isaac_plane *clip, int32_t n_clip, const isaac_render_opts *opts,
                       const isaac_framebuffer *fb, cudaStream_t st, int mode,
                       const FrameHook *hook, KParams &p)
{
    memset(&p, 0, sizeof p);
    int rc = prepare_frame(camera, clip, n_clip, opts, p);
    if (rc) return rc;
    int nact = 0;
    unsigned sig = 0;
    bool wide = false;
    update_sources(n_sources, opts->active_mask);
    rc = prepare_sources(sources, chains, n_sources, luts, weights, opts, p, &nact, &sig, &wide);
    if (rc) return rc;
    rc = prepare_fb(fb, p);
    if (rc) return rc;
    if (p.touched) return fail(ISAAC_ENOTSUP, "the footprint output is not offered here");
    FrameLaunch fn = nullptr, fn_long = nullptr;
    int rl = 1;
    if (nact > 0) {
        const long long rect = (long long)(p.rx1 - p.rx0) * (long long)(p.ry1 - p.ry0);
        fn = find_zc(nact, sig, opts->interp, wide, mode,
                     choose_lanes(rect, opts->lanes_per_ray, zc_corner_bytes(p, nact)), &rl);
        if (!fn) return fail(ISAAC_ENOTSUP, "no kernel for %d sources in this mode", nact);
        if (hook && mode == MODE_PLAIN) {
            int rl_long = 0;
            fn_long = find_zc(nact, sig, opts->interp, wide, MODE_LONG, kLongRayLanes, &rl_long);
        }
    }
    return launch_frame_with(p, fn, rl, st, hook, fn_long);
}

extern "C" int isaac_trace(const isaac_source *sources, const isaac_chain *chains,
                           int32_t n_sources, const float *luts, const float *weights,
                           const isaac_camera *camera, const isaac_plane *clip, int32_t n_clip,
                           const isaac_render_opts *opts, const isaac_framebuffer *fb,
                           const isaac_proposal *proposal, isaac_ray *rays, int64_t capacity,
                           int32_t *count, void *stream)
{
    clear_error();
    if (!rays || capacity < 0 || !count) return fail(ISAAC_EINVAL, "rays, capacity and count are required");
    if (((uintptr_t)rays) % 16 || ((uintptr_t)count) % 4)
        return fail(ISAAC_EINVAL, "rays must be 16-byte aligned, count 4-byte aligned");
    FrameHook hook;
    int rc = proposal_hook(proposal, opts, &hook);
    if (rc) return rc;
    KParams p;
    const cudaStream_t st = (cudaStream_t)stream;
    rc = render_mode(sources, chains, n_sources, luts, weights, camera, clip, n_clip, opts, fb, st,
                     MODE_LABEL, proposal ? &hook : nullptr, p);
    if (rc) return rc;
    if (!p.ctr) {   // nothing was cast: no rays
        if (cudaMemsetAsync(count, 0, sizeof(int32_t), st) != cudaSuccess) return check_cuda("isaac_trace");
        return ISAAC_OK;
    }
    launch_copy_rays(p, reinterpret_cast<RayRec *>(rays), capacity, count, st);
    return check_cuda("isaac_trace copy");
}

extern "C" int isaac_render_learned(const isaac_source *sources, const isaac_chain *chains,
                                    int32_t n_sources, const float *luts, const float *weights,
                                    const isaac_camera *camera, const isaac_plane *clip,
                                    int32_t n_clip, const isaac_render_opts *opts,
                                    const isaac_framebuffer *fb, const isaac_proposal *proposal,
                                    void *stream)
{
    clear_error();
    if (!proposal) return fail(ISAAC_EINVAL, "proposal is required");
    FrameHook hook;
    int rc = proposal_hook(proposal, opts, &hook);
    if (rc) return rc;
    KParams p;
    return render_mode(sources, chains, n_sources, luts, weights, camera, clip, n_clip, opts, fb,
                       (cudaStream_t)stream, MODE_PLAIN, &hook, p);
}

extern "C" int isaac_render_skip(const isaac_source *sources, const isaac_chain *chains,
                                 int32_t n_sources, const float *luts, const float *weights,
                                 const isaac_camera *camera, const isaac_plane *clip,
                                 int32_t n_clip, const isaac_render_opts *opts,
                                 const isaac_framebuffer *fb, const float *ranges,
                                 int64_t ranges_len, int32_t cell, void *stream)
{
    clear_error();
    KParams p;
    memset(&p, 0, sizeof p);
    int rc = prepare_frame(camera, clip, n_clip, opts, p);
    if (rc) return rc;
    int nact = 0;
    unsigned sig = 0;
    bool wide = false;
    update_sources(n_sources, opts->active_mask);
    rc = prepare_sources(sources, chains, n_sources, luts, weights, opts, p, &nact, &sig, &wide);
    if (rc) return rc;
    rc = prepare_fb(fb, p);
    if (rc) return rc;
    if (p.touched) return fail(ISAAC_ENOTSUP, "the footprint output is not offered here");
    if (!ranges || ((uintptr_t)ranges) % 8) return fail(ISAAC_EINVAL, "ranges must be 8-byte aligned device memory");
    if (cell < 2 || cell > 1024) return fail(ISAAC_EINVAL, "cell %d outside 2..1024", cell);
    p.skip_cell = cell;
    p.sgx = (p.nx + cell - 1) / cell;
    p.sgy = (p.ny + cell - 1) / cell;
    p.sgz = (p.nz + cell - 1) / cell;
    const long long cells = (long long)p.sgx * p.sgy * p.sgz;
    int slots = 0;
    for (int a = 0; a < nact; ++a) slots += p.src[a].fdim;
    if (ranges_len < cells * slots * 2)
        return fail(ISAAC_EINVAL, "ranges holds %lld floats; the active sources need %lld (same n, "
                    "cell and active_mask as isaac_range_grid)", (long long)ranges_len, cells * slots * 2);
    const cudaStream_t st = (cudaStream_t)stream;
    FrameLaunch fn = nullptr;
    int rl = 1;
    if (nact > 0 && p.rx1 > p.rx0 && p.ry1 > p.ry0) {
        const long long rect = (long long)(p.rx1 - p.rx0) * (long long)(p.ry1 - p.ry0);
        fn = find_zc(nact, sig, opts->interp, wide, MODE_SKIP,
                     choose_lanes(rect, opts->lanes_per_ray, zc_corner_bytes(p, nact)), &rl);
        if (!fn) return fail(ISAAC_ENOTSUP, "no empty-space-skipping kernel for %d sources", nact);
        void *flags = nullptr;
        rc = bind_workspace(p, st, (size_t)((cells + 31) / 32) * 4 + 16, &flags);
        if (rc) return rc;
        unsigned *bits = reinterpret_cast<unsigned *>((reinterpret_cast<uintptr_t>(flags) + 15) & ~uintptr_t(15));
        p.empty = bits;
        rc = launch_empty_flags(p, nact, ranges, slots, cells, bits, st);
        if (rc) return rc;
    }
    return launch_frame_with(p, fn, rl, st, nullptr);
}

extern "C" int isaac_render_iso(const isaac_source *sources, const isaac_chain *chains,
                                int32_t n_sources, const float *luts, const float *iso_values,
                                const isaac_camera *camera, const isaac_plane *clip, int32_t n_clip,
                                const isaac_render_opts *opts, const isaac_framebuffer *fb,
                                void *stream)
{
    clear_error();
    if (!iso_values) return fail(ISAAC_EINVAL, "iso_values is required");
    if (n_sources < 1 || n_sources > ISAAC_MAX_SOURCES)
        return fail(ISAAC_EINVAL, "n_sources %d outside 1..%d", n_sources, ISAAC_MAX_SOURCES);
    float ones[ISAAC_MAX_SOURCES];
    for (int s = 0; s < ISAAC_MAX_SOURCES; ++s) ones[s] = 1.0f;
    KParams p;
    memset(&p, 0, sizeof p);
    int rc = prepare_frame(camera, clip, n_clip, opts, p);
    if (rc) return rc;
    int nact = 0;
    unsigned sig = 0;
    bool wide = false;
    update_sources(n_sources, opts->active_mask);
    // two guard layers where the sources have them: the gradient stencil of a
    // hit reaches one voxel beyond the box
    rc = prepare_sources(sources, chains, n_sources, luts, ones, opts, p, &nact, &sig, &wide, 2);
    if (rc) return rc;
    rc = prepare_fb(fb, p);
    if (rc) return rc;
    if (p.touched) return fail(ISAAC_ENOTSUP, "the footprint output is not offered here");
    int a = 0;
    for (int s = 0; s < n_sources; ++s) {
        if (!((opts->active_mask >> s) & 1u)) continue;
        if (!std::isfinite(iso_values[s])) return fail(ISAAC_EINVAL, "iso value %d is not finite", s);
        p.iso[a++] = iso_values[s];
    }
    FrameLaunch fn = nullptr;
    int rl = 1;
    if (nact > 0) {
        fn = find_zc(nact, sig, opts->interp, wide, MODE_ISO, 4, &rl);
        if (!fn) return fail(ISAAC_ENOTSUP, "no iso-surface kernel for %d sources (64-bit offsets?)", nact);
    }
    return launch_frame_with(p, fn, rl, (cudaStream_t)stream, nullptr);
}

extern "C" int isaac_release_workspaces(void)
{
    clear_error();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return check_cuda("cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_ws_mu);
    if (cudaDeviceSynchronize() != cudaSuccess) return check_cuda("cudaDeviceSynchronize");
    std::vector<Workspace> keep;
    for (Workspace &w : g_ws) {
        if (w.device == dev) {
            if (w.ptr) cudaFree(w.ptr);
        } else {
            keep.push_back(w);
        }
    }
    g_ws.swap(keep);
    std::vector<LutStage> keep_stage;
    for (LutStage &e : g_lut_stage) {
        if (e.device == dev) {
            for (int i = 0; i < kLutSlots; ++i) cudaEventDestroy(e.done[i]);
            cudaFreeHost(e.host);
        } else {
            keep_stage.push_back(e);
        }
    }
    g_lut_stage.swap(keep_stage);
    return check_cuda("isaac_release_workspaces");
}

extern "C" const char *isaac_last_error(void) { return last_error(); }

extern "C" int isaac_abi_version(void) { return ISAAC_ABI_VERSION; }

extern "C" int isaac_time_march(void *start_event, void *stop_event)
{
    clear_error();
    if ((start_event == nullptr) != (stop_event == nullptr))
        return fail(ISAAC_EINVAL, "give both events or neither");
    t_march_start = static_cast<cudaEvent_t>(start_event);
    t_march_stop = static_cast<cudaEvent_t>(stop_event);
    return ISAAC_OK;
}

// Measurement aid: stream `bytes` of device memory `passes` times through
// 16-byte loads (an L2 bandwidth probe when the buffer fits in L2).
static __global__ void k_probe_read(const uint4 *__restrict__ buf, long long n, int passes,
                                    unsigned *sink)
{
    unsigned acc = 0;
    for (int r = 0; r < passes; ++r)
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x9e3779b9u) sink[blockIdx.x & 1023] = acc;   // keeps the loads alive
}

extern "C" int isaac_probe_read(const void *buf, int64_t bytes, int32_t passes, uint32_t *sink,
                                void *stream)
{
    clear_error();
    if (!buf || !sink || bytes < 16 || passes < 1 || ((uintptr_t)buf) % 16)
        return fail(ISAAC_EINVAL, "a 16-byte aligned buffer of >= 16 bytes, passes >= 1 and a sink are required");
    const long long n = bytes / 16;
    const int blocks = sm_count() * 8;
    k_probe_read<<<blocks, 256, 0, (cudaStream_t)stream>>>(static_cast<const uint4 *>(buf), n, passes,
                                                          sink);
    return check_cuda("isaac_probe_read launch");
}
