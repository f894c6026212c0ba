// packed_host.cu -- host side of the packed (reduced-precision) path:
// isaac_pack_layout, isaac_pack, isaac_render_packed.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cmath>
#include <cstring>

#include "common.h"
#include "packed.cuh"

namespace isaac {

extern const PackedTable k_packed_f32;
extern const PackedTable k_packed_bf16;
extern const PackedTable k_packed_f16;
extern const PackedTable k_packed_e4m3;

static const PackedTable *table_for(int dtype)
{
    switch (dtype) {
    case ISAAC_F32: return &k_packed_f32;
    case ISAAC_BF16: return &k_packed_bf16;
    case ISAAC_F16: return &k_packed_f16;
    case ISAAC_E4M3: return &k_packed_e4m3;
    default: return nullptr;
    }
}

static int elem_bytes(int dtype) { return dtype == ISAAC_F32 ? 4 : dtype == ISAAC_E4M3 ? 1 : 2; }
static int log2i(int v) { return v == 1 ? 0 : v == 2 ? 1 : v == 4 ? 2 : 3; }
static int next_pow2(int v) { return v <= 1 ? 1 : v <= 2 ? 2 : v <= 4 ? 4 : 8; }

static unsigned packed_sig(const int *fd, int nsrc)
{
    unsigned s = 0;
    for (int i = 0; i < nsrc; ++i) s |= (unsigned)fd[i] << (4 * i);
    return s;
}

static int sig_index(unsigned sig)
{
    for (int i = 0; i < k_n_packed_sigs; ++i)
        if (k_packed_sigs[i] == sig) return i;
    return -1;
}

static int layout_of(const isaac_source *sources, int32_t n_sources, uint32_t mask,
                     const int64_t n[3], int32_t dtype, isaac_packed *L, int64_t *data_bytes,
                     int64_t *scale_bytes)
{
    if (!sources || !n || !L) return fail(ISAAC_EINVAL, "sources, n and layout are required");
    if (!table_for(dtype)) return fail(ISAAC_EINVAL, "unknown dtype %d", dtype);
    if (n_sources < 1 || n_sources > ISAAC_MAX_SOURCES)
        return fail(ISAAC_EINVAL, "n_sources %d outside 1..%d", n_sources, ISAAC_MAX_SOURCES);
    if (mask >> n_sources) return fail(ISAAC_EINVAL, "mask has bits beyond n_sources");
    for (int a = 0; a < 3; ++a)
        if (n[a] < 1 || n[a] > 4096) return fail(ISAAC_EINVAL, "n[%d] = %lld outside 1..4096", a, (long long)n[a]);
    memset(L, 0, sizeof *L);
    int nc = 0;
    for (int s = 0; s < n_sources; ++s) {
        if (!((mask >> s) & 1u)) continue;
        if (L->n_src == ISAAC_MAX_ACTIVE)
            return fail(ISAAC_ENOTSUP, "more than %d packed sources", ISAAC_MAX_ACTIVE);
        if (sources[s].f_dim < 1 || sources[s].f_dim > 4)
            return fail(ISAAC_EINVAL, "source %d: f_dim %d outside 1..4", s, sources[s].f_dim);
        L->f_dim[L->n_src++] = sources[s].f_dim;
        nc += sources[s].f_dim;
    }
    if (L->n_src == 0) return fail(ISAAC_EINVAL, "mask selects no source");
    if (nc > 8) return fail(ISAAC_ENOTSUP, "%d components to pack (max 8)", nc);
    L->n_comp = nc;
    L->pad = sig_index(packed_sig(L->f_dim, L->n_src)) >= 0 ? next_pow2(nc) : 8;
    L->dtype = dtype;
    for (int a = 0; a < 3; ++a) L->n[a] = n[a];
    const int64_t cells = (n[0] + 2) * (n[1] + 2) * (n[2] + 2);
    *data_bytes = cells * L->pad * elem_bytes(dtype);
    const int64_t bricks = ((n[0] + 9) / 8) * ((n[1] + 9) / 8) * ((n[2] + 9) / 8);
    *scale_bytes = dtype == ISAAC_E4M3 ? bricks * L->pad * 4 : 0;
    return ISAAC_OK;
}

}  // namespace isaac

using namespace isaac;

extern "C" int isaac_pack_layout(const isaac_source *sources, int32_t n_sources, uint32_t mask,
                                 const int64_t n[3], int32_t dtype, isaac_packed *layout,
                                 int64_t *data_bytes, int64_t *scale_bytes)
{
    clear_error();
    if (!data_bytes || !scale_bytes) return fail(ISAAC_EINVAL, "size outputs are required");
    return layout_of(sources, n_sources, mask, n, dtype, layout, data_bytes, scale_bytes);
}

extern "C" int isaac_pack(const isaac_source *sources, int32_t n_sources, uint32_t mask,
                          const int64_t n[3], int32_t dtype, void *data, int64_t data_bytes,
                          float *scales, int64_t scale_bytes, isaac_packed *out, void *stream)
{
    clear_error();
    update_sources(n_sources, mask);
    isaac_packed L;
    int64_t need_d = 0, need_s = 0;
    int rc = layout_of(sources, n_sources, mask, n, dtype, &L, &need_d, &need_s);
    if (rc) return rc;
    if (!out) return fail(ISAAC_EINVAL, "out is required");
    if (!data || ((uintptr_t)data) % 16) return fail(ISAAC_EINVAL, "data must be 16-byte aligned device memory");
    if (data_bytes < need_d)
        return fail(ISAAC_ENOMEM, "data buffer has %lld bytes, the copy needs %lld",
                    (long long)data_bytes, (long long)need_d);
    if (dtype == ISAAC_E4M3) {
        if (!scales || ((uintptr_t)scales) % 16)
            return fail(ISAAC_EINVAL, "E4M3 needs 16-byte aligned device scales");
        if (scale_bytes < need_s)
            return fail(ISAAC_ENOMEM, "scale buffer has %lld bytes, needs %lld",
                        (long long)scale_bytes, (long long)need_s);
    }
    KPack kp;
    memset(&kp, 0, sizeof kp);
    for (int s = 0; s < n_sources; ++s) {
        if (!((mask >> s) & 1u)) continue;
        KSource ks;
        unsigned nib;
        bool wide;
        rc = prepare_source(sources[s], s, n, 1, 1.0f, 4, ks, &nib, &wide);
        if (rc) return rc;
        KPackSrc &q = kp.src[kp.nsrc++];
        q.base = ks.base;
        q.sx = ks.sx;
        q.sy = ks.sy;
        q.sz = ks.sz;
        q.sc = ks.sc;
        q.fdim = ks.fdim;
        q.guard = sources[s].guard;
        for (int c = 0; c < ks.fdim; ++c) {
            kp.slot_src[kp.ncomp] = kp.nsrc - 1;
            kp.slot_comp[kp.ncomp] = c;
            ++kp.ncomp;
        }
    }
    kp.nx = (int)n[0];
    kp.ny = (int)n[1];
    kp.nz = (int)n[2];
    kp.px = kp.nx + 2;
    kp.py = kp.ny + 2;
    kp.pz = kp.nz + 2;
    kp.bx = (kp.px + 7) / 8;
    kp.by = (kp.py + 7) / 8;
    kp.bz = (kp.pz + 7) / 8;
    kp.rec = static_cast<unsigned char *>(data);
    kp.scales = dtype == ISAAC_E4M3 ? scales : nullptr;
    table_for(dtype)->pack[log2i(L.pad)](kp, (cudaStream_t)stream);
    rc = check_cuda("isaac_pack launch");
    if (rc) return rc;
    L.data = data;
    L.scales = kp.scales;
    *out = L;
    return ISAAC_OK;
}

static int render_packed_impl(const isaac_packed *vol, const isaac_chain *chains,
                              const float *luts, const float *weights, const isaac_camera *camera,
                              const isaac_plane *clip, int32_t n_clip,
                              const isaac_render_opts *opts, const isaac_framebuffer *fb,
                              void *stream, const isaac_proposal *proposal)
{
    if (!vol || !chains || !weights || !opts)
        return fail(ISAAC_EINVAL, "vol, chains, weights and opts are required");
    const PackedTable *T = table_for(vol->dtype);
    if (!T) return fail(ISAAC_EINVAL, "unknown dtype %d", vol->dtype);
    if (vol->n_src < 1 || vol->n_src > ISAAC_MAX_ACTIVE)
        return fail(ISAAC_EINVAL, "packed volume has %d sources", vol->n_src);
    if (vol->pad != 1 && vol->pad != 2 && vol->pad != 4 && vol->pad != 8)
        return fail(ISAAC_EINVAL, "pad %d is not 1, 2, 4 or 8", vol->pad);
    int nc = 0;
    for (int i = 0; i < vol->n_src; ++i) {
        if (vol->f_dim[i] < 1 || vol->f_dim[i] > 4)
            return fail(ISAAC_EINVAL, "packed source %d: f_dim %d", i, vol->f_dim[i]);
        nc += vol->f_dim[i];
    }
    if (nc != vol->n_comp || nc > vol->pad) return fail(ISAAC_EINVAL, "inconsistent packed layout");
    if (!vol->data || ((uintptr_t)vol->data) % 16) return fail(ISAAC_EINVAL, "vol->data misaligned");
    if (vol->dtype == ISAAC_E4M3 && (!vol->scales || ((uintptr_t)vol->scales) % 16))
        return fail(ISAAC_EINVAL, "E4M3 volume needs 16-byte aligned scales");
    for (int a = 0; a < 3; ++a)
        if (opts->n[a] != vol->n[a])
            return fail(ISAAC_EINVAL, "opts->n differs from the packed volume");
    if (opts->active_mask >> vol->n_src)
        return fail(ISAAC_EINVAL, "active_mask 0x%x has bits beyond the %d packed sources",
                    opts->active_mask, vol->n_src);
    KParams p;
    memset(&p, 0, sizeof p);
    int rc = prepare_frame(camera, clip, n_clip, opts, p);
    if (rc) return rc;
    rc = prepare_fb(fb, p);
    if (rc) return rc;
    if (!luts || (!(opts->flags & ISAAC_LUTS_HOST) && ((uintptr_t)luts) % 16))
        return fail(ISAAC_EINVAL, "luts must be 16-byte aligned");
    if (opts->flags & ISAAC_LUTS_HOST) p.luts_host = 1;   // staged when the workspace is bound
    // Every packed source is evaluated (its components share the record); an
    // inactive one gets an identity chain and weight 0, which adds exactly +0.
    int off = 0;
    for (int s = 0; s < vol->n_src; ++s) {
        const bool on = (opts->active_mask >> s) & 1u;
        if (on) {
            if (!std::isfinite(weights[s])) return fail(ISAAC_EINVAL, "weight %d is not finite", s);
            rc = compile_chain(chains[s], vol->f_dim[s], s, p.ch[s]);
            if (rc) return rc;
        } else {
            isaac_chain none;
            memset(&none, 0, sizeof none);
            compile_chain(none, vol->f_dim[s], s, p.ch[s]);
        }
        p.src[s].fdim = vol->f_dim[s];
        p.src[s].w = on ? weights[s] : 0.0f;
        p.comp_off[s] = off;
        p.lut[s] = reinterpret_cast<const float4 *>(luts) + (size_t)s * 256;
        off += vol->f_dim[s];
    }
    p.rec = static_cast<const unsigned char *>(vol->data);
    p.scales = vol->scales;
    p.pad = vol->pad;
    p.bx = (int)((vol->n[0] + 9) / 8);
    p.by = (int)((vol->n[1] + 9) / 8);

    PackedLaunch fn = nullptr, fn_long = nullptr;
    int rl = 1;
    if (opts->active_mask != 0) {
        const long long rect = (long long)(p.rx1 - p.rx0) * (long long)(p.ry1 - p.ry0);
        const int want = choose_lanes(rect, opts->lanes_per_ray, vol->pad * elem_bytes(vol->dtype));
        const unsigned sig = packed_sig(vol->f_dim, vol->n_src);
        const bool spec = sig_index(sig) >= 0 && vol->pad == next_pow2(nc);
        const PackedEntry *best = nullptr;
        for (int i = 0; i < T->n_entries; ++i) {
            const PackedEntry &e = T->entries[i];
            if (e.nact != vol->n_src || e.interp != opts->interp || e.pad != vol->pad) continue;
            if (e.sig != (spec ? sig : 0u) || e.longpass) continue;
            if (!best || e.rl == want ||
                (best->rl != want && std::abs(e.rl - want) < std::abs(best->rl - want)))
                best = &e;
        }
        if (!best) return fail(ISAAC_ENOTSUP, "no packed kernel for this layout");
        fn = best->fn;
        rl = best->rl;
        if (proposal)
            for (int i = 0; i < T->n_entries; ++i) {
                const PackedEntry &e = T->entries[i];
                if (e.longpass && e.nact == vol->n_src && e.interp == opts->interp &&
                    e.pad == vol->pad && e.sig == (spec ? sig : 0u))
                    fn_long = e.fn;
            }
    }
    if (p.touched) return fail(ISAAC_ENOTSUP, "the footprint output is not offered for packed copies");
    FrameHook hook;
    rc = proposal_hook(proposal, opts, &hook);
    if (rc) return rc;
    return launch_frame_with(p, fn, rl, (cudaStream_t)stream, proposal ? &hook : nullptr, fn_long);
}

extern "C" int isaac_render_packed(const isaac_packed *vol, const isaac_chain *chains,
                                   const float *luts, const float *weights,
                                   const isaac_camera *camera, const isaac_plane *clip,
                                   int32_t n_clip, const isaac_render_opts *opts,
                                   const isaac_framebuffer *fb, void *stream)
{
    clear_error();
    return render_packed_impl(vol, chains, luts, weights, camera, clip, n_clip, opts, fb, stream,
                              nullptr);
}

extern "C" int isaac_render_packed_learned(const isaac_packed *vol, const isaac_chain *chains,
                                           const float *luts, const float *weights,
                                           const isaac_camera *camera, const isaac_plane *clip,
                                           int32_t n_clip, const isaac_render_opts *opts,
                                           const isaac_framebuffer *fb,
                                           const isaac_proposal *proposal, void *stream)
{
    clear_error();
    if (!proposal) return fail(ISAAC_EINVAL, "proposal is required");
    return render_packed_impl(vol, chains, luts, weights, camera, clip, n_clip, opts, fb, stream,
                              proposal);
}
