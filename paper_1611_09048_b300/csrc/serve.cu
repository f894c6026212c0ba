// serve.cu -- the serving loop: continuous batching of render requests
// against one device-resident volume.
//
// Requests (camera, image size, optionally their own transfer functions and
// functor chains) are queued by isaac_server_submit.  A worker thread admits
// them in arrival order while their device memory -- framebuffer, ray list,
// LUTs, parameter-table entry -- fits the server's budget and a stream is
// free, and launches everything admitted in a round as ONE batched frame:
// background, ray setup and march kernels that each cover all requests of the
// batch through a per-request parameter table and one combined ray list (each
// ray tagged with its request).  Batches are spread over several streams, so
// requests that arrive while others are on the GPU are admitted as soon as
// memory and a stream free up and their work overlaps on the device.  Every
// pixel depends only on its own request's parameters, so an image is the same
// alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.h"
#include "packed.cuh"
#include "raycast.cuh"

namespace isaac {

// --------------------------------------------------------- batched kernels

struct KBatch {
    const KParams *table;   // one entry per request
    const int *tile_off;    // setup tiles of requests [0, i) (nreq + 1 entries)
    int nreq;
    WsCounters *ctr;
    RayRec *rays;
};

static __global__ void k_batch_fill(const __grid_constant__ KBatch b)
{
    const int req = blockIdx.y;
    if (req == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        b.ctr->n_rays = 0u;
        b.ctr->next = 0u;
    }
    const KParams &p = b.table[req];
    const size_t total = (size_t)p.W * (size_t)p.H;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / (size_t)p.W), x = (int)(i - (size_t)y * p.W);
        if (x >= p.rx0 && x < p.rx1 && y >= p.ry0 && y < p.ry1) continue;
        write_pixel(p, (int)i, 0.0f, 0.0f, 0.0f, 0.0f, 0);
    }
}

static __global__ void __launch_bounds__(128) k_batch_setup(const __grid_constant__ KBatch b)
{
    int req = 0;
    while (req + 1 < b.nreq && (int)blockIdx.x >= b.tile_off[req + 1]) ++req;
    const KParams &p = b.table[req];
    const int t = blockIdx.x - b.tile_off[req];
    const int tiles_x = (p.rx1 - p.rx0 + 15) >> 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ty = t / tiles_x, tx = t - ty * tiles_x;
    const int px = p.rx0 + tx * 16 + (warp & 1) * 8 + (lane & 7);
    const int py = p.ry0 + ty * 8 + (warp >> 1) * 4 + (lane >> 3);
    const bool inside = px < p.rx1 && py < p.ry1;
    RayRec r;
    r.nsteps = 0;
    if (inside) r = setup_ray(p, px, py);
    r.reserved = req;
    const bool hit = inside && r.nsteps > 0;
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    unsigned base = 0;
    if (lane == 0 && m) base = atomicAdd(&b.ctr->n_rays, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (hit) {
        b.rays[base + __popc(m & ((1u << lane) - 1u))] = r;
    } else if (inside) {
        write_pixel(p, py * p.W + px, 0.0f, 0.0f, 0.0f, 0.0f, 0);
    }
}

// The persistent march over the batch's combined ray list: every ray is
// marched by march_ray with its own request's parameters (LUTs read from
// global memory, since a block may hold rays of several requests).
template <class Shader, int RL>
static __global__ void __launch_bounds__(kMarchThreads, kMarchBlocksPerSM) k_batch_march(const __grid_constant__ KBatch b)
{
    constexpr unsigned RAYS = 32 / RL;
    const int lane = threadIdx.x & 31;
    const unsigned n_rays = *(volatile unsigned *)&b.ctr->n_rays;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&b.ctr->next, RAYS);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_rays) break;
        const unsigned idx = base + (unsigned)(lane / RL);
        if (idx < n_rays) march_ray<Shader, RL, false>(b.table[b.rays[idx].reserved], nullptr, idx, lane);
    }
}

using BatchLaunch = void (*)(const KBatch &, dim3, cudaStream_t);

template <class Shader>
static void launch_batch_march(const KBatch &b, dim3 grid, cudaStream_t st)
{
    k_batch_march<Shader, 4><<<grid, kMarchThreads, 0, st>>>(b);
}

struct BatchEntry {
    bool packed;
    int nact;
    unsigned sig;   // zero-copy nibbles (f_dim | aos << 3) or packed f_dim nibbles; 0 = generic
    int interp;
    BatchLaunch fn;
};

#define ZC(N, S, I) {false, N, S, I, launch_batch_march<ZeroCopyShader<N, S, I, int, false>>}
#define PK(N, S, P, I) {true, N, S, I, launch_batch_march<PackedShader<N, S, ISAAC_BF16, P, I>>}
static const BatchEntry k_batch_entries[] = {
    ZC(1, 0x9u, 0), ZC(1, 0x9u, 1), ZC(3, 0x9BBu, 0), ZC(3, 0x9BBu, 1),
    ZC(1, 0u, 0), ZC(1, 0u, 1), ZC(2, 0u, 0), ZC(2, 0u, 1), ZC(3, 0u, 0), ZC(3, 0u, 1),
    ZC(4, 0u, 0), ZC(4, 0u, 1),
    PK(1, 0x1u, 1, 0), PK(1, 0x1u, 1, 1), PK(3, 0x133u, 8, 0), PK(3, 0x133u, 8, 1),
};
#undef ZC
#undef PK

// ------------------------------------------------------------- the server

static double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Request {
    isaac_request rq;
    std::vector<float> luts;      // the request's own transfer functions (empty: the server's)
    KChain chains[ISAAC_MAX_ACTIVE];
    bool own_chains = false;
    KParams frame;                // camera part, prepared at submit
    long long rect = 0;           // pixels of the rectangle that can hit the volume
    size_t bytes = 0;             // device memory the request adds to a batch
    double t_submit = 0.0;
};

struct Batch {
    std::vector<Request> reqs;
    size_t off = 0, bytes = 0;    // block of the arena
    bool busy = false;
    double t_launch = 0.0;
};

// First-fit allocator over the budget arena (host bookkeeping only).
class Arena {
public:
    explicit Arena(size_t bytes = 0)
    {
        if (bytes) free_.push_back({0, bytes});
    }
    bool alloc(size_t len, size_t *off)
    {
        for (size_t i = 0; i < free_.size(); ++i)
            if (free_[i].len >= len) {
                *off = free_[i].off;
                free_[i].off += len;
                free_[i].len -= len;
                if (!free_[i].len) free_.erase(free_.begin() + (long)i);
                return true;
            }
        return false;
    }
    bool fits(size_t len) const
    {
        for (const Range &r : free_)
            if (r.len >= len) return true;
        return false;
    }
    void release(size_t off, size_t len)
    {
        auto it = std::lower_bound(free_.begin(), free_.end(), off,
                                   [](const Range &r, size_t o) { return r.off < o; });
        it = free_.insert(it, {off, len});
        // merge with the next and the previous range
        if (it + 1 != free_.end() && it->off + it->len == (it + 1)->off) {
            it->len += (it + 1)->len;
            free_.erase(it + 1);
        }
        if (it != free_.begin() && (it - 1)->off + (it - 1)->len == it->off) {
            (it - 1)->len += it->len;
            free_.erase(it);
        }
    }

private:
    struct Range {
        size_t off, len;
    };
    std::vector<Range> free_;   // sorted by offset, never adjacent
};

// Bytes of a batch's block before the framebuffers: counters, tile offsets,
// parameter table, LUT copies.
static size_t batch_header(int nreq, size_t lut_bytes, size_t *o_tiles, size_t *o_table,
                           size_t *o_luts)
{
    *o_tiles = kWsHeader;
    *o_table = align256(*o_tiles + (size_t)(nreq + 1) * sizeof(int));
    *o_luts = align256(*o_table + (size_t)nreq * sizeof(KParams));
    return align256(*o_luts + (size_t)nreq * lut_bytes);
}

}  // namespace isaac

using namespace isaac;

struct isaac_server {
    int device = 0;
    int sms = 148;
    KParams base;                 // sources or packed copy, chains, LUTs, weights, options
    isaac_render_opts opts;
    std::vector<isaac_plane> clip;
    int n_src = 0;                // sources a request's LUT array and chain array cover
    int nact = 0;
    int src_index[ISAAC_MAX_ACTIVE] = {0};   // active slot -> source index
    size_t lut_bytes = 0;         // n_src * 256 RGBA floats
    BatchLaunch march = nullptr;
    isaac_server_config cfg;
    char *arena_dev = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;        // a batch's end (after its image copies), per stream
    std::vector<cudaEvent_t> events_start;  // a batch's start (before its header upload), per stream
    cudaEvent_t ev_ref = nullptr;           // the device clock's origin, recorded at creation
    std::vector<char *> staging;  // pinned batch headers, one per stream
    size_t staging_bytes = 0;
    std::vector<Batch> slots;     // the batch in flight on each stream
    std::deque<Request> pending;
    std::deque<isaac_result> results;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;
    double t0 = 0.0;
};

static void finish(isaac_server *s, const Request &r, int status, int batch_size, double t_launch,
                   double t_done, int stream = -1, double gpu_start = -1.0, double gpu_end = -1.0)
{
    isaac_result res;
    memset(&res, 0, sizeof res);
    res.tag = r.rq.tag;
    res.status = status;
    res.batch_size = batch_size;
    res.t_submit = r.t_submit - s->t0;
    res.t_launch = t_launch - s->t0;
    res.t_done = t_done - s->t0;
    res.t_gpu_start = gpu_start;
    res.t_gpu_end = gpu_end;
    res.stream = stream;
    s->results.push_back(res);
}

// Device-clock time of a completed event, in seconds since the server's
// reference event (-1 if it cannot be read).
static double gpu_time(const isaac_server *s, cudaEvent_t ev)
{
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, s->ev_ref, ev) != cudaSuccess) {
        cudaGetLastError();
        return -1.0;
    }
    return 1e-3 * (double)ms;
}

// Lay out, upload and launch one batch on stream `si` (worker thread, lock held).
// ISAAC_ENOMEM: the arena has no contiguous block for it yet.
static int launch_batch(isaac_server *s, Batch &b, int si)
{
    const int nreq = (int)b.reqs.size();
    const cudaStream_t st = s->streams[si];
    size_t o_tiles, o_table, o_luts;
    const size_t o_fb = batch_header(nreq, s->lut_bytes, &o_tiles, &o_table, &o_luts);
    size_t o_rays = o_fb;
    long long rays = 0;
    for (const Request &r : b.reqs) {
        o_rays += align256((size_t)r.rq.camera.width * r.rq.camera.height * 4);
        rays += r.rect;
    }
    const size_t need = align256(o_rays + (size_t)std::max(1LL, rays) * sizeof(RayRec));
    if (o_fb > s->staging_bytes) return fail(ISAAC_EINVAL, "batch header exceeds the staging buffer");
    if (!s->arena.alloc(need, &b.off)) return ISAAC_ENOMEM;
    b.bytes = need;
    char *blk = s->arena_dev + b.off;
    char *stg = s->staging[si];
    int *tile_off = reinterpret_cast<int *>(stg + o_tiles);
    KParams *table = reinterpret_cast<KParams *>(stg + o_table);
    size_t fb_at = o_fb;
    int tiles = 0;
    for (int i = 0; i < nreq; ++i) {
        const Request &r = b.reqs[i];
        // the request's frame (camera, rectangle, options) with the server's
        // volume part (sources or packed copy, chains, LUTs, weights)
        KParams q = r.frame;
        memcpy(q.src, s->base.src, sizeof q.src);
        memcpy(q.ch, s->base.ch, sizeof q.ch);
        memcpy(q.lut, s->base.lut, sizeof q.lut);
        memcpy(q.comp_off, s->base.comp_off, sizeof q.comp_off);
        q.rec = s->base.rec;
        q.scales = s->base.scales;
        q.pad = s->base.pad;
        q.bx = s->base.bx;
        q.by = s->base.by;
        q.grab = 1;
        q.longs = nullptr;
        q.fb8 = reinterpret_cast<uchar4 *>(blk + fb_at);
        q.fb32 = nullptr;
        q.nsamp = nullptr;
        q.touched = nullptr;
        q.ctr = reinterpret_cast<WsCounters *>(blk);
        q.rays = reinterpret_cast<RayRec *>(blk + o_rays);
        fb_at += align256((size_t)r.rq.camera.width * r.rq.camera.height * 4);
        if (!r.luts.empty()) {
            memcpy(stg + o_luts + i * s->lut_bytes, r.luts.data(), s->lut_bytes);
            const float4 *dl = reinterpret_cast<const float4 *>(blk + o_luts + i * s->lut_bytes);
            for (int a = 0; a < s->nact; ++a) q.lut[a] = dl + (size_t)s->src_index[a] * 256;
        }
        if (r.own_chains)
            for (int a = 0; a < s->nact; ++a) q.ch[a] = r.chains[a];
        tile_off[i] = tiles;
        tiles += ((q.rx1 - q.rx0 + 15) / 16) * ((q.ry1 - q.ry0 + 7) / 8);
        table[i] = q;
    }
    tile_off[nreq] = tiles;
    KBatch kb;
    kb.table = reinterpret_cast<const KParams *>(blk + o_table);
    kb.tile_off = reinterpret_cast<const int *>(blk + o_tiles);
    kb.nreq = nreq;
    kb.ctr = reinterpret_cast<WsCounters *>(blk);
    kb.rays = reinterpret_cast<RayRec *>(blk + o_rays);
    cudaEventRecord(s->events_start[si], st);
    cudaMemcpyAsync(blk + o_tiles, stg + o_tiles, o_fb - o_tiles, cudaMemcpyHostToDevice, st);
    int maxpix = 1;
    for (const Request &r : b.reqs) maxpix = std::max(maxpix, r.rq.camera.width * r.rq.camera.height);
    const int fill_x = std::max(1, std::min((maxpix + 255) / 256, 64));
    k_batch_fill<<<dim3(fill_x, nreq), 256, 0, st>>>(kb);
    if (tiles > 0) {
        k_batch_setup<<<tiles, 128, 0, st>>>(kb);
        // 128-thread blocks, 4 lanes per ray: 32 rays per block and chunk
        const long long want = (rays + 31) / 32;
        s->march(kb, dim3((unsigned)std::max(1LL, std::min(want, (long long)s->sms * 8))), st);
    }
    fb_at = o_fb;
    for (const Request &r : b.reqs) {
        const size_t bytes = (size_t)r.rq.camera.width * r.rq.camera.height * 4;
        cudaMemcpyAsync(r.rq.out, blk + fb_at, bytes, cudaMemcpyDefault, st);
        fb_at += align256(bytes);
    }
    cudaEventRecord(s->events[si], st);
    const cudaError_t e = cudaGetLastError();
    b.busy = true;
    b.t_launch = now_s();
    if (e != cudaSuccess) return fail(ISAAC_ECUDA, "server launch: %s", cudaGetErrorString(e));
    return ISAAC_OK;
}

static void worker_loop(isaac_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        // retire finished batches
        bool retired = false;
        for (size_t si = 0; si < s->slots.size(); ++si) {
            Batch &b = s->slots[si];
            if (!b.busy) continue;
            const cudaError_t q = cudaEventQuery(s->events[si]);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) cudaGetLastError();
            const double t = now_s();
            const double g0 = q == cudaSuccess ? gpu_time(s, s->events_start[si]) : -1.0;
            const double g1 = q == cudaSuccess ? gpu_time(s, s->events[si]) : -1.0;
            for (const Request &r : b.reqs)
                finish(s, r, q == cudaSuccess ? ISAAC_OK : ISAAC_ECUDA, (int)b.reqs.size(), b.t_launch, t,
                       (int)si, g0, g1);
            s->arena.release(b.off, b.bytes);
            b = Batch();
            retired = true;
        }
        if (retired) s->cv_done.notify_all();
        // admit pending requests in arrival order onto idle streams
        for (size_t si = 0; si < s->slots.size() && !s->pending.empty(); ++si) {
            if (s->slots[si].busy) continue;
            Batch b;
            size_t o_tiles, o_table, o_luts;
            size_t bytes = 0;
            while (!s->pending.empty() && (int)b.reqs.size() < s->cfg.max_batch) {
                const Request &r = s->pending.front();
                const size_t head = batch_header((int)b.reqs.size() + 1, s->lut_bytes, &o_tiles,
                                                 &o_table, &o_luts);
                if (!s->arena.fits(head + bytes + r.bytes + 256)) break;
                bytes += r.bytes;
                b.reqs.push_back(std::move(s->pending.front()));
                s->pending.pop_front();
            }
            if (b.reqs.empty()) break;   // the head of the queue waits for memory
            const int rc = launch_batch(s, b, (int)si);
            if (rc == ISAAC_ENOMEM) {
                for (auto it = b.reqs.rbegin(); it != b.reqs.rend(); ++it)
                    s->pending.push_front(std::move(*it));
                break;
            }
            if (rc != ISAAC_OK && !b.busy) {
                const double t = now_s();
                for (const Request &r : b.reqs) finish(s, r, rc, (int)b.reqs.size(), t, t);
                s->cv_done.notify_all();
                continue;
            }
            s->slots[si] = std::move(b);
        }
        bool busy = false;
        for (const Batch &b : s->slots) busy |= b.busy;
        if (s->stop && !busy && s->pending.empty()) break;
        if (busy)
            s->cv_work.wait_for(lock, std::chrono::microseconds(20));
        else
            s->cv_work.wait_for(lock, std::chrono::milliseconds(20),
                                [s] { return s->stop || !s->pending.empty(); });
    }
    s->cv_done.notify_all();
}

static bool host_or_device(const void *ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeDevice ||
           a.type == cudaMemoryTypeManaged;
}

extern "C" int isaac_server_create(const isaac_source *sources, const isaac_chain *chains,
                                   int32_t n_sources, const float *luts, const float *weights,
                                   const isaac_packed *vol, const isaac_render_opts *opts,
                                   const isaac_plane *clip, int32_t n_clip,
                                   const isaac_server_config *cfg, isaac_server **out)
{
    clear_error();
    if (!out) return fail(ISAAC_EINVAL, "out is required");
    *out = nullptr;
    if (!cfg || !opts || !chains || !weights || !luts)
        return fail(ISAAC_EINVAL, "cfg, opts, chains, weights and luts are required");
    if (cfg->n_streams < 1 || cfg->n_streams > 8) return fail(ISAAC_EINVAL, "n_streams must be 1..8");
    if (cfg->max_batch < 1 || cfg->max_batch > ISAAC_SERVER_MAX_BATCH)
        return fail(ISAAC_EINVAL, "max_batch must be 1..%d", ISAAC_SERVER_MAX_BATCH);
    if (cfg->budget_bytes < (1 << 20)) return fail(ISAAC_EINVAL, "budget below 1 MiB");
    if (((uintptr_t)luts) % 16) return fail(ISAAC_EINVAL, "luts must be 16-byte aligned");
    if (opts->flags & ISAAC_LUTS_HOST)
        return fail(ISAAC_EINVAL, "the server's LUTs are device memory (requests carry host LUTs)");
    if (n_clip < 0 || n_clip > ISAAC_MAX_CLIP || (n_clip > 0 && !clip))
        return fail(ISAAC_EINVAL, "n_clip %d outside 0..%d (or clip is NULL)", n_clip, ISAAC_MAX_CLIP);
    std::unique_ptr<isaac_server> s(new isaac_server());
    s->cfg = *cfg;
    s->opts = *opts;
    // The per-request part (camera, rectangle) comes at submit; validate the rest
    // with a unit camera.
    isaac_camera cam;
    memset(&cam, 0, sizeof cam);
    for (int i = 0; i < 16; i += 5) cam.modelview[i] = cam.projection[i] = 1.0;
    cam.width = cam.height = 1;
    memset(&s->base, 0, sizeof s->base);
    int rc = prepare_frame(&cam, clip, n_clip, opts, s->base);
    if (rc) return rc;
    if (n_clip > 0) s->clip.assign(clip, clip + n_clip);
    unsigned sig = 0;
    const bool packed = vol != nullptr;
    if (!packed) {
        bool wide = false;
        update_sources(n_sources, opts->active_mask);
        rc = prepare_sources(sources, chains, n_sources, luts, weights, opts, s->base, &s->nact, &sig, &wide);
        if (rc) return rc;
        if (wide) return fail(ISAAC_ENOTSUP, "the server needs 32-bit element offsets");
        s->n_src = n_sources;
        int a = 0;
        for (int i = 0; i < n_sources; ++i)
            if ((opts->active_mask >> i) & 1u) s->src_index[a++] = i;
    } else {
        if (vol->dtype != ISAAC_BF16) return fail(ISAAC_ENOTSUP, "the server serves BF16 packed copies");
        if (vol->n_src < 1 || vol->n_src > ISAAC_MAX_ACTIVE || opts->active_mask != (1u << vol->n_src) - 1u)
            return fail(ISAAC_EINVAL, "a packed volume is served with all its sources active");
        if (!vol->data || ((uintptr_t)vol->data) % 16) return fail(ISAAC_EINVAL, "vol->data misaligned");
        for (int a = 0; a < 3; ++a)
            if (opts->n[a] != vol->n[a]) return fail(ISAAC_EINVAL, "opts->n differs from the volume");
        int off = 0;
        for (int i = 0; i < vol->n_src; ++i) {
            if (vol->f_dim[i] < 1 || vol->f_dim[i] > 4) return fail(ISAAC_EINVAL, "packed f_dim %d", vol->f_dim[i]);
            if (!std::isfinite(weights[i])) return fail(ISAAC_EINVAL, "weight %d is not finite", i);
            rc = compile_chain(chains[i], vol->f_dim[i], i, s->base.ch[i]);
            if (rc) return rc;
            s->base.src[i].fdim = vol->f_dim[i];
            s->base.src[i].w = weights[i];
            s->base.comp_off[i] = off;
            s->base.lut[i] = reinterpret_cast<const float4 *>(luts) + (size_t)i * 256;
            s->src_index[i] = i;
            off += vol->f_dim[i];
            sig |= (unsigned)vol->f_dim[i] << (4 * i);
        }
        s->nact = s->n_src = vol->n_src;
        s->base.rec = static_cast<const unsigned char *>(vol->data);
        s->base.pad = vol->pad;
        s->base.bx = (int)((vol->n[0] + 9) / 8);
        s->base.by = (int)((vol->n[1] + 9) / 8);
        if (!((sig == 0x1u && vol->pad == 1) || (sig == 0x133u && vol->pad == 8)))
            return fail(ISAAC_ENOTSUP, "the server serves packed copies of {1} or {3,3,1} components");
    }
    for (int pass = 0; pass < 2 && !s->march; ++pass)
        for (const BatchEntry &e : k_batch_entries)
            if (e.packed == packed && e.nact == s->nact && e.interp == opts->interp &&
                e.sig == (pass == 0 ? sig : 0u))
                s->march = e.fn;
    if (!s->march) return fail(ISAAC_ENOTSUP, "no batched kernel for %d active sources", s->nact);
    s->lut_bytes = (size_t)s->n_src * 256 * 4 * sizeof(float);
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    if (cudaMalloc(&s->arena_dev, (size_t)cfg->budget_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ISAAC_ENOMEM, "cannot allocate the %lld-byte server budget", (long long)cfg->budget_bytes);
    }
    s->arena = Arena((size_t)cfg->budget_bytes);
    size_t o1, o2, o3;
    s->staging_bytes = batch_header(cfg->max_batch, s->lut_bytes, &o1, &o2, &o3);
    s->slots.resize(cfg->n_streams);
    for (int i = 0; i < cfg->n_streams; ++i) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr, ev0 = nullptr;
        char *stg = nullptr;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        cudaEventCreate(&ev);      // timed: the results carry device-clock intervals
        cudaEventCreate(&ev0);
        cudaHostAlloc(reinterpret_cast<void **>(&stg), s->staging_bytes, cudaHostAllocDefault);
        s->streams.push_back(st);
        s->events.push_back(ev);
        s->events_start.push_back(ev0);
        s->staging.push_back(stg);
    }
    cudaEventCreate(&s->ev_ref);
    if (s->ev_ref && !s->streams.empty() && s->streams[0]) {
        cudaEventRecord(s->ev_ref, s->streams[0]);
        cudaEventSynchronize(s->ev_ref);
    }
    rc = check_cuda("isaac_server_create");
    if (rc) {
        isaac_server_destroy(s.release());
        return rc;
    }
    s->t0 = now_s();
    isaac_server *raw = s.release();
    raw->worker = std::thread(worker_loop, raw);
    *out = raw;
    return ISAAC_OK;
}

extern "C" int isaac_server_submit(isaac_server *s, const isaac_request *rq)
{
    clear_error();
    if (!s || !rq) return fail(ISAAC_EINVAL, "server and request are required");
    if (!rq->out || !host_or_device(rq->out))
        return fail(ISAAC_EINVAL, "out must be pinned host memory or device memory");
    Request r;
    r.rq = *rq;
    r.rq.luts = nullptr;
    r.rq.chains = nullptr;
    r.t_submit = now_s();
    memset(&r.frame, 0, sizeof r.frame);
    int rc = prepare_frame(&rq->camera, s->clip.data(), (int32_t)s->clip.size(), &s->opts, r.frame);
    if (rc) return rc;
    if (rq->luts) {
        r.luts.assign(rq->luts, rq->luts + s->lut_bytes / sizeof(float));
        for (float v : r.luts)
            if (!std::isfinite(v)) return fail(ISAAC_EINVAL, "a request LUT entry is not finite");
    }
    if (rq->chains) {
        for (int a = 0; a < s->nact; ++a) {
            const int si = s->src_index[a];
            rc = compile_chain(rq->chains[si], s->base.src[a].fdim, si, r.chains[a]);
            if (rc) return rc;
        }
        r.own_chains = true;
    }
    r.rect = (long long)(r.frame.rx1 - r.frame.rx0) * (r.frame.ry1 - r.frame.ry0);
    r.bytes = align256((size_t)rq->camera.width * rq->camera.height * 4) + (size_t)r.rect * sizeof(RayRec);
    size_t o1, o2, o3;
    if (batch_header(1, s->lut_bytes, &o1, &o2, &o3) + r.bytes + 256 > (size_t)s->cfg.budget_bytes)
        return fail(ISAAC_ENOMEM, "a %dx%d request needs %zu bytes, over the server budget",
                    rq->camera.width, rq->camera.height, r.bytes);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return fail(ISAAC_EINVAL, "the server is shutting down");
        s->pending.push_back(std::move(r));
    }
    s->cv_work.notify_one();
    return ISAAC_OK;
}

extern "C" int isaac_server_poll(isaac_server *s, isaac_result *out, int32_t max, double wait_s)
{
    clear_error();
    if (!s || !out || max < 1) return fail(ISAAC_EINVAL, "server, out and max >= 1 are required");
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->results.empty() && wait_s > 0.0)
        s->cv_done.wait_for(lock, std::chrono::duration<double>(wait_s),
                            [s] { return !s->results.empty(); });
    int n = 0;
    while (n < max && !s->results.empty()) {
        out[n++] = s->results.front();
        s->results.pop_front();
    }
    return n;
}

extern "C" int isaac_server_outstanding(isaac_server *s)
{
    clear_error();
    if (!s) return fail(ISAAC_EINVAL, "server is required");
    std::lock_guard<std::mutex> lock(s->mu);
    int n = (int)s->pending.size();
    for (const Batch &b : s->slots) n += b.busy ? (int)b.reqs.size() : 0;
    return n;
}

extern "C" int isaac_server_destroy(isaac_server *s)
{
    clear_error();
    if (!s) return ISAAC_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t st : s->streams)
        if (st) cudaStreamSynchronize(st);
    for (cudaStream_t st : s->streams)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : s->events)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : s->events_start)
        if (ev) cudaEventDestroy(ev);
    if (s->ev_ref) cudaEventDestroy(s->ev_ref);
    for (char *p : s->staging)
        if (p) cudaFreeHost(p);
    if (s->arena_dev) cudaFree(s->arena_dev);
    delete s;
    return check_cuda("isaac_server_destroy");
}
