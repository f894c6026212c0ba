/*
 * isaac_b300.h -- C ABI of the B300-native ISAAC volume ray caster.
 *
 * ISAAC (Matthes et al., 2016) renders simulation fields in situ: the
 * application keeps its data where it is, describes each field as a "source"
 * (Sec. 3.2: a scalar or vector of up to 4 components per regularly spaced
 * cell, read through an accessor, optionally surrounded by guard cells), and
 * calls one render function that ray casts every pixel front to back over all
 * active sources (Sec. 3.2), each passed through its functor chain (Sec. 3.3)
 * and a transfer function.
 *
 * Everything here is plain C: device pointers, host structs, sizes.  The
 * library never allocates, frees or copies the caller's field data (Sec. 3.1
 * "zero copy"); every call is ordered on the caller's CUDA stream and returns
 * once the work is enqueued.  All entry points return ISAAC_OK (0) or a
 * negative isaac_status; isaac_last_error() then describes the failure (per
 * calling thread).  Invalid arguments are rejected on the host before any
 * launch, so a rejected call touches no device memory.
 */
#ifndef ISAAC_B300_H
#define ISAAC_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ISAAC_ABI_VERSION 3
#define ISAAC_MAX_SOURCES 8   /* sources described per call */
#define ISAAC_MAX_ACTIVE 4    /* sources rendered per call (active_mask bits) */
#define ISAAC_MAX_FUNCTORS 8  /* functors per chain */
#define ISAAC_MAX_CLIP 6      /* clipping planes per call */

typedef enum {
    ISAAC_OK = 0,
    ISAAC_EINVAL = -1,   /* malformed argument (sizes, dimensions, chain, NaN weight ...) */
    ISAAC_EGUARD = -2,   /* a source's reachable cells leave its allocation */
    ISAAC_ENOMEM = -3,   /* a caller-provided buffer or budget is too small */
    ISAAC_ECUDA = -4,    /* a CUDA launch or runtime call failed */
    ISAAC_ENOTSUP = -5   /* valid but outside what this build supports */
} isaac_status;

typedef enum { ISAAC_F32 = 0, ISAAC_BF16 = 1, ISAAC_F16 = 2, ISAAC_E4M3 = 3 } isaac_dtype;

/* Functors of Sec. 3.3, Table 1, plus the user functor LOG (Sec. 3.3 allows
 * application-defined functors).
 *   ADD(v), MUL(v): componentwise with v; one argument is broadcast to every
 *                   component (Sec. 3.3: add(1) adds (1,1,1)).
 *   LENGTH, SUM:    reduce the vector to a scalar.
 *   POW(v):         componentwise x^v; a non-positive base gives 0.
 *   LOG:            componentwise log(max(x, 1e-30)).
 * A chain that ends on a vector is reduced to its first component (Sec. 3.3). */
typedef enum {
    ISAAC_OP_ADD = 1, ISAAC_OP_MUL = 2, ISAAC_OP_LENGTH = 3,
    ISAAC_OP_SUM = 4, ISAAC_OP_POW = 5, ISAAC_OP_LOG = 6
} isaac_op;

/* One source (Sec. 3.2).  Element (x, y, z, c) of the interior, with x, y, z
 * in [0, n) and c in [0, f_dim), lives at
 *     ptr[offset + x*stride[0] + y*stride[1] + z*stride[2] + c*comp_stride]
 * (elements of the source's dtype; strides may have any sign, so any pitch
 * or axis order is described without a copy, Sec. 3.1 accessors).  Guard
 * cells (Sec. 3.1/3.2) extend every axis by `guard` cells on both sides with
 * the neighbour's data; with guard = 0 interpolation clamps at the border.
 * `extent` is the number of elements addressable from `ptr`; every cell the
 * renderer can reach must lie in [0, extent) or the call fails with
 * ISAAC_EGUARD.  Sources whose active_mask bit is clear are never read and
 * may be NULL (Sec. 3.2: deactivated sources are never read). */
typedef struct {
    const void *ptr;         /* device memory, owned by the caller */
    int64_t extent;
    int64_t offset;
    int64_t stride[3];
    int64_t comp_stride;
    int32_t f_dim;           /* 1..4 */
    int32_t guard;           /* >= 0 */
} isaac_source;

typedef struct {
    int32_t op;              /* isaac_op */
    int32_t n_args;          /* 0 for LENGTH/SUM/LOG; 1 (broadcast) or the current dimension */
    float arg[4];
} isaac_functor;

typedef struct {
    int32_t n_ops;           /* 0..ISAAC_MAX_FUNCTORS; 0 = identity (first component) */
    isaac_functor ops[ISAAC_MAX_FUNCTORS];
} isaac_chain;

/* Clipping plane (Sec. 3 feature list): points p (global voxel coordinates)
 * with n . p + d >= 0 are kept. */
typedef struct {
    double n[3];
    double d;
} isaac_plane;

/* OpenGL-style column-major matrices (element (r, c) at [4*c + r]).  World
 * coordinates are global voxel coordinates minus global_n / 2, so the global
 * box is centred on the origin with one world unit per cell.  Pixel (x, y),
 * row 0 at the top, shoots the ray from NDC (2(x+1/2)/W - 1, 1 - 2(y+1/2)/H,
 * -1) to the same point at depth +1. */
typedef struct {
    double modelview[16];
    double projection[16];
    int32_t width;
    int32_t height;
} isaac_camera;

typedef struct {
    int64_t n[3];            /* interior cells of the local volume (all sources share it) */
    int64_t global_n[3];     /* cells of the global volume; {0,0,0} = equal to n */
    int64_t offset[3];       /* first cell of the local volume inside the global one */
    float step;              /* sample spacing along the ray, in voxels, > 0 */
    int32_t interp;          /* 1 = trilinear (Sec. 3 feature list: interpolation), 0 = nearest cell */
    float term_alpha;        /* a ray stops once its opacity A >= term_alpha; > 1 disables */
    float bg[4];             /* background RGBA (premultiplied) blended behind the volume */
    uint32_t active_mask;    /* bit s set: source s is rendered (Sec. 3.2) */
    int32_t lanes_per_ray;   /* 0 = automatic, else 1, 2, 4, 8 or 16 threads cooperating on one
                                ray; a hint (the nearest compiled variant is used) that
                                never changes the image, only the speed */
    uint32_t flags;          /* ISAAC_LUTS_HOST, ISAAC_MARCH_STAGED, or 0; other bits are
                                rejected (ISAAC_EINVAL) */
} isaac_render_opts;

/* opts.flags: `luts` is a HOST array (any host memory).  The call copies the
 * active sources' LUTs before it returns (so the caller may reuse the array
 * at once) into a library-owned pinned staging slot, and from there, on the
 * call's stream, into the stream's workspace.  A stream has 8 such slots; a
 * call waits only when the copy issued 8 calls earlier on that stream has not
 * run yet.  Without the flag `luts` is device memory, read by the kernels. */
#define ISAAC_LUTS_HOST 1u

/* opts.flags: march with per-warp shared-memory staging of the field instead
 * of the default gather march: one thread per ray; per slab of up to 16
 * samples a warp copies the box of cells its 32 rays read into shared memory
 * with coalesced loads, then gathers from there.  Used by isaac_render when
 * the frame allows it (trilinear; one scalar source, or E/B/rho-shaped
 * sources, with 32-bit offsets and equal guard reach; no footprint output),
 * ignored otherwise.  The image is the same bit for bit either way.  On B300
 * it measured slower than the gather march at every camera distance tried
 * (0.14x at twice the box diagonal to ~0.96x with rays 0.2-0.5 voxels
 * apart), so it is off by default; it is offered for comparison. */
#define ISAAC_MARCH_STAGED 2u

/* Output buffers (device, owned by the caller), row-major, row 0 at the top. */
typedef struct {
    uint8_t *rgba8;          /* required: width*height*4 bytes */
    float *rgba32;           /* optional: width*height*4 floats before quantisation */
    int32_t *nsamples;       /* optional: width*height composited-sample counts */
    /* optional footprint: one bit per cell of [-1, n]^3 that any composited
     * sample read, cell (x,y,z) at bit ((z+1)*(ny+2) + (y+1))*(nx+2) + (x+1)
     * of an array of ceil((nx+2)(ny+2)(nz+2)/32) words.  Bits are OR-ed in;
     * the caller clears the array.  Measurement aid (slower path). */
    uint32_t *touched;
    /* optional: width*height floats, the distance along the pixel's ray (unit
     * direction, from the near plane) to its first sample on the global grid,
     * +inf where it has none: the per-pixel visibility key of sort-last
     * compositing (isaac_composite). */
    float *depth;
} isaac_framebuffer;

/*
 * isaac_render -- one frame of the volume ray caster (Sec. 3.2: at every
 * sample point each active source passes its functor chain and transfer
 * function, the sources combine into one colour and opacity, and the ray
 * composites front to back).  Per pixel:
 *   ray through the pixel centre; entry t0 into the global box (not before
 *   the near plane); the local box and the clip planes bound [t_in, t_out];
 *   samples t0 + k*step with t_in <= t < t_out (one global sample grid); per
 *   active source the value at the sample (trilinear with guards, or nearest),
 *   the source's functor chain, the source's 256-entry RGBA LUT (entries at
 *   j/255, linear in between, input clamped to [0,1]); the sample colour is
 *   sum_s weights[s] * rgba_s with alpha clamped to [0,1]; front-to-back
 *   C += (1-A) a rgb, A += (1-A) a until A >= term_alpha; output
 *   (C, A) + (1-A) bg, quantised to round(255 * clamp(x, 0, 1)).
 *
 * sources, chains, weights: host arrays of n_sources (1..ISAAC_MAX_SOURCES).
 * luts: n_sources * 256 * 4 floats (RGBA, source-major), owned by the
 *       caller: a DEVICE array, 16-byte aligned, or with opts->flags &
 *       ISAAC_LUTS_HOST a host array (copied before the call returns).
 * camera, clip (n_clip <= ISAAC_MAX_CLIP, may be NULL if 0), opts, fb: host
 *       structs, read before the call returns; the caller may reuse them.
 * stream: cudaStream_t to order the work on (NULL = legacy default stream).
 * The current CUDA device must own every device pointer.
 * Workspace: the library keeps one device workspace per (device, stream) for
 * the frame's ray list (32 bytes per pixel of the screen rectangle the box can
 * cover, plus 256 bytes), allocated on first use and grown (after
 * synchronising that stream) when a larger rectangle comes; frames on one
 * stream share it in order, frames on different streams never share.
 * isaac_release_workspaces() frees them; ISAAC_ENOMEM if allocation fails.
 */
int isaac_render(const isaac_source *sources, const isaac_chain *chains, int32_t n_sources,
                 const float *luts, const float *weights, const isaac_camera *camera,
                 const isaac_plane *clip, int32_t n_clip, const isaac_render_opts *opts,
                 const isaac_framebuffer *fb, void *stream);

/*
 * Reduced-precision storage.  Not part of the paper, whose renderer always
 * reads the application's own arrays (Sec. 3.1 zero copy): these calls make a
 * packed copy of the active sources when memory bandwidth matters more than
 * the copy.  One record per cell over the cells [-1, n]^3 holds every packed
 * source's components in order (guard cells where a source has them, else
 * the border cell repeated, which is what clamping reads), `pad` components
 * per record (the next power of two of the component total for the
 * source lists the library specialises, else 8), stored as:
 *   ISAAC_F32   float32;
 *   ISAAC_BF16  bfloat16, round to nearest even;
 *   ISAAC_F16   IEEE binary16, round to nearest even;
 *   ISAAC_E4M3  FP8 E4M3 codes of value / scale (the quotient correctly
 *               rounded to float32, then to E4M3 with ties to even),
 *               saturating at +-448, with one float32 scale per 8^3 brick of
 *               the [-1, n]^3 box (bricks counted from cell -1) and component:
 *               scale = absmax / 448 over the brick, 1 for an all-zero brick.
 * Sampling dequantises to float32 and interpolates, classifies and
 * composites in float32 exactly as isaac_render does.
 */
typedef struct {
    void *data;              /* device records, owned by the caller */
    float *scales;           /* device brick scales (E4M3), owned by the caller; else NULL */
    int64_t n[3];            /* interior cells */
    int32_t dtype;           /* isaac_dtype */
    int32_t n_src;           /* packed sources, in their original order */
    int32_t f_dim[ISAAC_MAX_ACTIVE];
    int32_t n_comp;          /* sum of f_dim, <= 8 */
    int32_t pad;             /* components per record: 1, 2, 4 or 8 */
} isaac_packed;

/* Sizes of the packed copy of the sources selected by `mask` (at most
 * ISAAC_MAX_ACTIVE, together at most 8 components): fills layout (everything
 * but data/scales) and the device bytes the caller must provide. */
int isaac_pack_layout(const isaac_source *sources, int32_t n_sources, uint32_t mask,
                      const int64_t n[3], int32_t dtype, isaac_packed *layout,
                      int64_t *data_bytes, int64_t *scale_bytes);

/* Fill the packed copy (one kernel, stream-ordered).  data (16-byte aligned,
 * data_bytes) and, for E4M3, scales (16-byte aligned, scale_bytes) are
 * device buffers of at least the sizes isaac_pack_layout reports; sources are
 * validated as in isaac_render (trilinear reach).  *out describes the copy. */
int isaac_pack(const isaac_source *sources, int32_t n_sources, uint32_t mask, const int64_t n[3],
               int32_t dtype, void *data, int64_t data_bytes, float *scales, int64_t scale_bytes,
               isaac_packed *out, void *stream);

/* isaac_render over a packed copy.  chains, weights (host) and luts (device,
 * n_src * 256 * 4 floats) are indexed by packed source; opts->n must equal
 * vol->n and opts->active_mask selects among the packed sources. */
int isaac_render_packed(const isaac_packed *vol, const isaac_chain *chains, const float *luts,
                        const float *weights, const isaac_camera *camera, const isaac_plane *clip,
                        int32_t n_clip, const isaac_render_opts *opts, const isaac_framebuffer *fb,
                        void *stream);

/*
 * isaac_opacity_grid -- the max-opacity grid over macro cells of `cell`^3
 * cells (a coarse map of where the transfer functions make the volume
 * visible; the paper has no such structure, it serves empty-space skipping
 * and the learned interval proposal).  Macro cell (i,j,k) covers the cells
 * [i*cell-1, (i+1)*cell] per axis, clipped to [-1, n] (the apron trilinear
 * samples inside it read); its value is the largest blended opacity
 * clamp(sum_s weights[s] * LUT_s(chain_s(v_s)).alpha, 0, 1) over those cells,
 * each active source read at the cell itself (clamped without guards).
 * cell: 2..1024.  grid: device, ceil(n/cell) values per axis, x fastest;
 * grid_len its length (the first ceil(n/cell)^3 values are overwritten).
 * Sources, chains, luts, weights and opts (n, active_mask) as in
 * isaac_render.
 */
int isaac_opacity_grid(const isaac_source *sources, const isaac_chain *chains, int32_t n_sources,
                       const float *luts, const float *weights, const isaac_render_opts *opts,
                       int32_t cell, float *grid, int64_t grid_len, void *stream);

/*
 * Classical empty-space skipping (no counterpart in the paper, which skips
 * only deactivated sources, Sec. 3.2).
 *
 * isaac_range_grid -- per macro cell of `cell`^3 cells (the boxes of
 * isaac_opacity_grid, i.e. with the one-cell trilinear apron) and per
 * component of each active source, the smallest and largest value read from
 * the box's cells ([-inf, +inf] if any is NaN).  ranges: device floats,
 * ceil(n/cell)^3 cells x (sum of the active sources' f_dim) x 2, layout
 * [cell (x fastest)][component, active sources in order][min, max].  It
 * depends on the data only: recompute it when the fields change, not when
 * the transfer functions or chains do.  cell: 2..1024.
 */
int isaac_range_grid(const isaac_source *sources, int32_t n_sources, const isaac_render_opts *opts,
                     int32_t cell, float *ranges, int64_t ranges_len, void *stream);

/*
 * isaac_render_skip -- isaac_render (same arguments, same image bit for bit)
 * that jumps over macro cells where no sample can be visible: from `ranges`
 * (isaac_range_grid of the same sources, n, cell and active_mask) it bounds,
 * with outward-rounded interval arithmetic, each source's chain result over
 * the cell and the LUT opacity over the entries that result can reach; a
 * cell where every source with weight > 0 gets opacity exactly 0 (and every
 * reachable LUT entry is finite) is skipped along each ray.  Those samples
 * would composite nothing, so only the nsamples output differs: it counts
 * the samples actually evaluated.
 */
int isaac_render_skip(const isaac_source *sources, const isaac_chain *chains, int32_t n_sources,
                      const float *luts, const float *weights, const isaac_camera *camera,
                      const isaac_plane *clip, int32_t n_clip, const isaac_render_opts *opts,
                      const isaac_framebuffer *fb, const float *ranges, int64_t ranges_len,
                      int32_t cell, void *stream);

/*
 * isaac_render_iso -- iso-surface rendering (Sec. 3 feature list; the
 * renderings of Sec. 4.2).  The paper gives no algorithm; this call
 * implements one reading:
 *   the samples of isaac_render (same grid, same [t_in, t_out]); at each,
 *   every active source's chain value v_s; the surface is met at the first
 *   sample where some v_s >= iso_values[s]; each crossing source refines the
 *   crossing by one secant step towards the previous sample (none at the
 *   ray's first sample), the nearest crossing wins (ties: lower source);
 *   the normal is that source's central-difference gradient (one voxel,
 *   same interpolation; the two positions are clamped to what the source's
 *   cells can interpolate: [1/2 - g, n + g - 1/2] with g = min(guard, 2)
 *   guard layers, [0, n] without guards or with interpolation off, so that
 *   with two guard layers a sub-volume shades its hits as the whole volume
 *   does), turned towards the viewer; with a headlight,
 *   rgb = LUT_s(iso_values[s]).rgb * (1/4 + 3/4 * n.v) + 1/4 * (n.v)^32,
 *   clamped to [0, 1], alpha 1.  Rays without a crossing show the background.
 * iso_values: host, n_sources floats (finite for active sources).  The
 * other arguments as for isaac_render (weights are not used); nsamples, if
 * given, counts the samples evaluated.
 */
int isaac_render_iso(const isaac_source *sources, const isaac_chain *chains, int32_t n_sources,
                     const float *luts, const float *iso_values, const isaac_camera *camera,
                     const isaac_plane *clip, int32_t n_clip, const isaac_render_opts *opts,
                     const isaac_framebuffer *fb, void *stream);

/*
 * isaac_render_noalloc -- the frame of isaac_render (same arguments, same
 * kernels, same image) for callers that must not allocate device memory.
 * The paper has no counterpart.  isaac_render allocates its per-stream ray
 * list with cudaMalloc; in-situ hosts often cannot allow that: a simulation
 * typically reserves nearly all device memory at start-up and serves later
 * requests from its own pool (a library-side cudaMalloc then fails or
 * fragments that memory), and a host rendering from inside its time-step
 * loop may forbid allocation there because cudaMalloc can synchronise the
 * device.  This call keeps the ray list in a fixed array compiled into the
 * library instead (about 12 MiB of static device memory on every GPU that
 * loads the library, held until the process exits), so it allocates and
 * frees nothing.
 *   Limit: the screen rectangle the local box can cover must hold at most
 *   262,144 pixels (e.g. 512x512); beyond that the call fails with
 *   ISAAC_ENOMEM before any launch.  The footprint output (fb->touched) is
 *   not offered (ISAAC_ENOTSUP).
 *   Set-up: the first call on each device looks up the array's device
 *   address (cudaGetSymbolAddress, which may load the library's device code);
 *   make that first call before any stream capture.
 *   Sharing: every call on a device uses that device's one copy of the array,
 *   which keeps the previous call's contents; each call's first kernel resets
 *   the counters it needs, so calls ordered one after another (one stream) are
 *   independent, but calls on the same device that overlap on the GPU (for
 *   example on two streams) race and corrupt each other's rays.
 */
int isaac_render_noalloc(const isaac_source *sources, const isaac_chain *chains,
                         int32_t n_sources, const float *luts, const float *weights,
                         const isaac_camera *camera, const isaac_plane *clip, int32_t n_clip,
                         const isaac_render_opts *opts, const isaac_framebuffer *fb,
                         void *stream);

/*
 * Learned ray-interval proposal.  Not in the paper: a small MLP predicts, per
 * ray, which part of its samples can have nonzero opacity, so the march can
 * skip empty space; the plain march is its fallback (confidence below a
 * threshold) and its teacher (labels).
 *
 * Ray record of the frame's compact ray list (what isaac_trace returns).
 */
typedef struct {
    float e[3];          /* local voxel position of the ray's first sample */
    int32_t nsteps;      /* samples on the global grid inside the box and clip planes */
    float d[3];          /* unit direction */
    int32_t pix;         /* pixel index y * width + x */
    int32_t kbeg;        /* first sample marched (0 for the plain march) */
    int32_t jf, jl;      /* first / last composited sample with opacity > 0, -1 if none */
    int32_t reserved;
} isaac_ray;

/*
 * Model: inputs (224) = for each of the 6 scalars e/n and d, sin and cos of
 * pi * 2^(k/2) * s for k = 0..15 (192 values), then the max-opacity grid at
 * 32 points e + ((i + 1/2)/32 * nsteps * step) * d, i = 0..31; network
 * 224 -> 64 -> 64 -> 64 -> 3 with ReLU; outputs u: te = sigmoid(u0), tx =
 * sigmoid(u1) = start / end of the visible samples as fractions of nsteps,
 * conf = sigmoid(u2).  A confident ray (conf >= threshold) marches samples
 * [floor(te*nsteps) - margin, ceil(tx*nsteps) + margin) clipped to the ray.
 * Parameters (float32, ISAAC_MLP_PARAMS): W1[224][64] (input-major), b1[64],
 * W2[64][64], b2[64], W3[64][64], b3[64], W4[64][3], b4[3].
 * Tensor-core kernels use an FP16 copy (ISAAC_MLP_HALF halves) refreshed by
 * isaac_mlp_sync and every training step.  All buffers are device memory
 * owned by the caller, 16-byte aligned; `step` counts Adam steps.
 */
#define ISAAC_MLP_PARAMS 22915
#define ISAAC_MLP_HALF 32256
#define ISAAC_MLP_INPUTS 224
typedef struct {
    float *params;
    float *grads;        /* training only */
    float *adam_m;       /* training only, zero-initialised by the caller */
    float *adam_v;       /* training only, zero-initialised by the caller */
    uint16_t *half_w;
    int32_t step;
} isaac_mlp;

/* Refresh the FP16 kernel copy from the float32 parameters. */
int isaac_mlp_sync(const isaac_mlp *model, void *stream);

/* isaac_mlp_create -- allocate a model's device buffers in one block
 * (params, and with `train` grads, adam_m, adam_v; then half_w), fill the
 * weights He-uniform, U(-sqrt(6/fan_in), sqrt(6/fan_in)), from the SplitMix64
 * stream of `seed`, biases, gradients and moments with 0, step 0, and the
 * FP16 copy.  Synchronises `stream`.  ISAAC_ENOMEM if allocation fails.
 * isaac_mlp_destroy frees a model made by isaac_mlp_create (and zeroes the
 * struct); a model whose buffers the caller owns is rejected (ISAAC_EINVAL). */
int isaac_mlp_create(isaac_mlp *model, int32_t train, uint64_t seed, void *stream);
int isaac_mlp_destroy(isaac_mlp *model);

/*
 * Checkpoint / resume of the proposal network.  Image layout (host memory,
 * little-endian): a 64-byte header {char magic[8] = "ISAACMLP"; uint32
 * version = 1; uint32 count = ISAAC_MLP_PARAMS; int32 step; uint32 flags
 * (bit 0: Adam moments present); uint64 tag; uint32 crc; zero padding} then
 * float32 params[count] and, with bit 0, adam_m[count] and adam_v[count].
 * crc is the CRC-32 (zlib's) of everything after the header; tag is the
 * caller's (e.g. the position of its training-data sampler).
 * isaac_mlp_checkpoint_bytes: the image size with or without Adam moments.
 * isaac_mlp_save writes the image of `model` (Adam moments when the model
 * has them) after the work already queued on `stream`; it synchronises the
 * stream and returns with the image complete.  ISAAC_ENOMEM if `bytes` is
 * too small.
 * isaac_mlp_load checks magic, version, count, size and CRC on the host
 * before touching the device (ISAAC_EINVAL on any mismatch), then copies the
 * parameters (and, for a model with Adam buffers, the moments and step; an
 * image without moments gives such a model zero moments and step 0) and
 * refreshes the FP16 copy; it synchronises the stream.  *tag (optional)
 * receives the header's tag.
 * Training is bitwise reproducible (the batch gradient is reduced in a fixed
 * order), so a run resumed from a checkpoint equals the uninterrupted run
 * when it is given the same batches.
 */
#define ISAAC_MLP_CKPT_HEADER 64
int64_t isaac_mlp_checkpoint_bytes(int32_t with_adam);
int isaac_mlp_save(const isaac_mlp *model, uint64_t tag, void *image, int64_t bytes, void *stream);
int isaac_mlp_load(isaac_mlp *model, const void *image, int64_t bytes, uint64_t *tag, void *stream);

/* Inputs of n_rays records into X (device, n_rays * 224 FP16, row-major);
 * grid as written by isaac_opacity_grid for the same volume size and cell. */
int isaac_mlp_features(const isaac_ray *rays, int64_t n_rays, const int64_t vol_n[3], float step,
                       const float *grid, int32_t cell, uint16_t *X, void *stream);

/* Raw outputs u (device, n_rays * 3 floats) for inputs X. */
int isaac_mlp_forward(const isaac_mlp *model, const uint16_t *X, int64_t n_rays, float *U,
                      void *stream);

/* One Adam step (lr; beta1 0.9, beta2 0.999, eps 1e-8) on the batch mean of
 * per-ray loss huber(te - ye) + huber(tx - yx) + 0.1 * BCE(conf, c), huber
 * delta 0.02, targets ye = jf/nsteps, yx = (jl+1)/nsteps (1 and 0 for a ray
 * with no visible sample), c = 1 when the proposed range with `margin`
 * covers [jf, jl] (always for an empty ray).  rays supply jf, jl, nsteps.
 * model->grads holds the batch gradient afterwards; loss_sum (device,
 * optional) accumulates the batch's mean loss.  The gradient is summed per
 * 64-ray tile, per block over its tiles in order, then over at most 148
 * blocks in block order (partial sums in the stream's workspace): the same
 * inputs give the same bits on any run and any device. */
int isaac_mlp_train_step(isaac_mlp *model, const uint16_t *X, const isaac_ray *rays,
                         int64_t n_rays, float lr, int32_t margin, float *loss_sum, void *stream);

/* The interval proposal applied to one frame.
 * widen != 0: a confident ray's range becomes the hull of the network's
 * range (when not empty) and every sample of the ray whose position lies in a
 * macro cell (floor(p / cell), clamped to the grid) with a nonzero grid
 * value, then is clipped to the ray; two 3D-DDA walks over the macro cells
 * per ray find the first and the last such sample (a kernel after the
 * network's; a sample within FP32 rounding of a cell face may count on either
 * side).  The network may tighten a range within what the grid marks as
 * possibly visible, never cut such a part.  The grid holds the max opacity at
 * the cells' values, so a sample whose LUT opacity is nonzero while that of
 * every cell around it is zero (a transfer function zero around a nonzero
 * bump) can still be cut; where the opacity is nonzero exactly above (or
 * below) a threshold, nothing can.
 * model == NULL with widen != 0: no network runs; every ray's range is the
 * hull of its samples in nonzero macro cells (empty-space skipping by the
 * max-opacity grid alone); `stats` is not updated. */
typedef struct {
    const isaac_mlp *model;   /* params + half_w are read (NULL: see above) */
    const float *grid;        /* device max-opacity grid of this frame (isaac_opacity_grid) */
    int32_t cell;             /* its macro-cell size */
    float threshold;          /* confidence needed to restrict a ray (e.g. 0.9) */
    int32_t margin;           /* samples added on both sides of the proposed range */
    int32_t *stats;           /* optional device int32[2]: += rays seen, rays restricted */
    int32_t widen;            /* 1: keep the grid's nonzero chord segments (see above) */
} isaac_proposal;

/*
 * isaac_trace -- isaac_render that also returns the frame's ray list: every
 * ray that enters the box (first sample, direction, sample count, pixel) with
 * its visible span jf/jl (first and last composited sample with opacity > 0,
 * counted from the ray's first sample; -1 if none).  With a proposal the
 * records show the restricted range (kbeg, nsteps) and the span within it.
 * rays: device array of `capacity` records (16-byte aligned); count: device
 * int32 receiving the number of rays (records beyond capacity are dropped).
 * The footprint output is not offered here.
 */
int isaac_trace(const isaac_source *sources, const isaac_chain *chains, int32_t n_sources,
                const float *luts, const float *weights, const isaac_camera *camera,
                const isaac_plane *clip, int32_t n_clip, const isaac_render_opts *opts,
                const isaac_framebuffer *fb, const isaac_proposal *proposal, isaac_ray *rays,
                int64_t capacity, int32_t *count, void *stream);

/* isaac_render with the interval proposal: after ray setup the MLP runs on
 * every ray of the frame (tensor cores); confident rays march only their
 * proposed sample range (same global sample grid, so where the range covers
 * every sample with opacity > 0 the pixel is bit-identical to isaac_render),
 * the others the whole ray. */
int isaac_render_learned(const isaac_source *sources, const isaac_chain *chains,
                         int32_t n_sources, const float *luts, const float *weights,
                         const isaac_camera *camera, const isaac_plane *clip, int32_t n_clip,
                         const isaac_render_opts *opts, const isaac_framebuffer *fb,
                         const isaac_proposal *proposal, void *stream);

/* isaac_render_packed with the interval proposal. */
int isaac_render_packed_learned(const isaac_packed *vol, const isaac_chain *chains,
                                const float *luts, const float *weights,
                                const isaac_camera *camera, const isaac_plane *clip,
                                int32_t n_clip, const isaac_render_opts *opts,
                                const isaac_framebuffer *fb, const isaac_proposal *proposal,
                                void *stream);

/*
 * Serving loop.  The paper has no counterpart kernel: its central server
 * (Sec. 3.5, steering through a central server)
 * forwards one application's frames to many clients, each of which may steer
 * the camera, transfer functions and functor chains.  Here one process renders
 * many such viewers' requests against one device-resident volume with
 * continuous batching:
 *
 *   isaac_server_submit queues a request (its camera and image size, and
 *   optionally its own transfer functions and functor chains).  A worker
 *   thread admits queued requests in arrival order while the device memory
 *   they need (RGBA8 image, ray list, table entry, LUT copy) fits the
 *   server's budget, at most max_batch per batch, and launches each batch as
 *   one frame: one background, one ray-setup and one march launch over all
 *   its requests, each ray carrying its request's constants.  Up to
 *   n_streams batches are in flight on their own streams, so requests that
 *   arrive while others render start as soon as memory and a stream free up.
 *   The image reaches request->out when the request's result is returned by
 *   isaac_server_poll.  A request's image does not depend on which other
 *   requests share its batch: it equals the same request rendered alone.
 *
 * The server never allocates during serving: the budget is one device
 * allocation made by isaac_server_create (ISAAC_ENOMEM if it fails).
 */
#define ISAAC_SERVER_MAX_BATCH 64

typedef struct isaac_server isaac_server;

typedef struct {
    int64_t budget_bytes;   /* device memory for requests in flight, >= 1 MiB */
    int32_t n_streams;      /* batches in flight at once, 1..8 */
    int32_t max_batch;      /* requests per batch, 1..ISAAC_SERVER_MAX_BATCH */
} isaac_server_config;

typedef struct {
    isaac_camera camera;        /* view and image size of this request */
    const float *luts;          /* host, n_sources * 256 RGBA floats (layout of isaac_render's
                                   luts), or NULL for the server's; copied at submit */
    const isaac_chain *chains;  /* host, n_sources chains, or NULL for the server's; compiled
                                   at submit */
    void *out;                  /* RGBA8 image, width * height * 4 bytes, row 0 at the top:
                                   pinned host memory (cudaHostAlloc / registered) or device
                                   memory; written when the result is reported */
    int64_t tag;                /* returned with the result */
} isaac_request;

typedef struct {
    int64_t tag;
    int32_t status;             /* ISAAC_OK, or the error that failed the request's batch */
    int32_t batch_size;         /* requests in the batch that rendered it */
    double t_submit;            /* seconds since isaac_server_create: queued, */
    double t_launch;            /* its batch enqueued on the GPU, */
    double t_done;              /* its image in `out` (completion seen by the worker) */
    double t_gpu_start;         /* device clock (CUDA events, seconds since create): its batch's */
    double t_gpu_end;           /* work began on its stream, and its images were copied; -1 on error */
    int32_t stream;             /* the server stream that ran its batch (-1: none) */
    int32_t reserved;
} isaac_result;

/*
 * Create a server for one volume: either zero-copy sources (vol == NULL;
 * sources, chains, n_sources, luts, weights as for isaac_render; at most 4
 * active; 32-bit element offsets) or a BF16 packed copy (vol != NULL; sources
 * ignored; all packed sources active; component sets {1} or {3,3,1}).  luts
 * is a device array that must stay valid for the server's lifetime, as must
 * the source data or the packed copy; opts and clip are copied.  The server
 * renders on the current device.  ISAAC_ENOTSUP for source sets without a
 * batched kernel.
 */
int isaac_server_create(const isaac_source *sources, const isaac_chain *chains, int32_t n_sources,
                        const float *luts, const float *weights, const isaac_packed *vol,
                        const isaac_render_opts *opts, const isaac_plane *clip, int32_t n_clip,
                        const isaac_server_config *cfg, isaac_server **out);

/* Queue a request (thread-safe).  Rejected on the host (nothing queued) for a
 * malformed camera, a non-finite LUT entry, an invalid chain, an `out` that is
 * neither pinned host nor device memory, or a request larger than the budget
 * (ISAAC_ENOMEM). */
int isaac_server_submit(isaac_server *server, const isaac_request *request);

/* Move up to `max` finished requests' results into `out`, waiting up to
 * wait_s seconds for the first one.  Returns how many (>= 0) or an error. */
int isaac_server_poll(isaac_server *server, isaac_result *out, int32_t max, double wait_s);

/* Requests queued or in flight whose results are not yet available. */
int isaac_server_outstanding(isaac_server *server);

/* Finish every queued request, then free the server (results not yet polled
 * are dropped).  NULL is a no-op. */
int isaac_server_destroy(isaac_server *server);

/* Measurement aid (no counterpart in the paper): while set, every frame the
 * calling thread renders with isaac_render, isaac_render_packed or their
 * learned variants records start_event and stop_event (cudaEvent_t handles,
 * created by the caller) on the frame's stream immediately before and after
 * its march kernel, so cudaEventElapsedTime gives that kernel's duration.
 * NULL, NULL stops it; one NULL and one event is ISAAC_EINVAL. */
int isaac_time_march(void *start_event, void *stop_event);

/*
 * isaac_composite -- sort-last compositing of partial images (Sec. 3.4: the
 * nodes' images of their sub-volumes are merged in visibility order; the
 * paper uses IceT over MPI).  layers_rgba32 / layers_depth: host arrays of
 * n_layers (1..16) device pointers to the rgba32 and depth outputs of frames
 * of disjoint local boxes of one global volume, rendered with the same camera
 * and a zero background.  Per pixel the layers are taken front to back by
 * depth (ties keep layer order; a NaN depth counts as +inf) and merged with the over operator
 * C += (1-A) c, A += (1-A) a; the background bg (host, 4 floats) is blended
 * behind the result, which goes to rgba8 (required) and rgba32 (optional),
 * both device, width*height pixels.  With early termination off the result
 * equals the frame of the whole volume up to FP32 rounding (one global
 * sample grid); with it, each layer terminates on its own.
 */
int isaac_composite(const float *const *layers_rgba32, const float *const *layers_depth,
                    int32_t n_layers, int32_t width, int32_t height, const float *bg,
                    uint8_t *rgba8, float *rgba32, void *stream);

/*
 * isaac_opacity_grid_packed -- isaac_opacity_grid over a packed copy (built by
 * isaac_pack): the same macro cells and rule, each cell's values read from
 * its record of the [-1, n]^3 box (the apron holds the guards, or the
 * repeated border, exactly the values isaac_opacity_grid reads there) and
 * dequantised as isaac_render_packed does.  The result is the grid of the
 * dequantised fields, with half (16-bit) or a quarter (E4M3) of the bytes to
 * read.  chains, weights (host) and luts (device) are indexed by packed source
 * as in isaac_render_packed; opts->n must equal vol->n; opts->active_mask
 * selects packed sources.  Errors as isaac_opacity_grid and
 * isaac_render_packed.
 */
int isaac_opacity_grid_packed(const isaac_packed *vol, const isaac_chain *chains, const float *luts,
                              const float *weights, const isaac_render_opts *opts, int32_t cell,
                              float *grid, int64_t grid_len, void *stream);

/*
 * The rest of the source contract (Sec. 3.2): the per-source update callback
 * and sources whose memory is not persistent.
 *
 * isaac_set_update_hook -- installs fn for the calling host thread (NULL
 * removes it; returns ISAAC_OK).  While set, these calls made by that thread
 * call fn(s, enabled, user) for every source s = 0 .. n_sources-1 in order,
 * enabled = bit s of the active mask, before they read any source descriptor:
 * isaac_render, isaac_trace, isaac_render_learned, isaac_render_skip,
 * isaac_render_iso, isaac_opacity_grid, isaac_range_grid, isaac_pack and
 * isaac_server_create.  The render calls validate the camera and options
 * first; a call that fails there, or whose n_sources is outside
 * 1..ISAAC_MAX_SOURCES, calls no hook.  The hook is where an application
 * passes per-frame information to its sources or (re)computes a derived field:
 * it may enqueue device work on the frame's stream and rewrite, through its
 * own pointer, the descriptor array the caller passed (the library reads it
 * only after the hooks return).  isaac_render_noalloc calls no hook: its host
 * path does nothing but validate and launch.
 *
 * isaac_copy_source -- for a source whose memory is not persistent (say one
 * scratch buffer that several derived fields take turns in): copies, through
 * the accessor (strides, component stride, guards), every cell a frame can
 * read -- the interior and, when the source has guard cells, one guard layer
 * -- into dst, and describes the copy in *out; a frame renders *out exactly
 * like the original.  dst: device memory, 16-byte aligned, dst_bytes >=
 * 4 f_dim (n0+2g)(n1+2g)(n2+2g) with g = min(guard, 1), cells x fastest with
 * their components adjacent; the caller owns it.  The copy is enqueued on
 * `stream`: work that the application orders after it on that stream (for
 * example the next source's update) may overwrite the original.  Errors:
 * ISAAC_EINVAL (NULL pointers, n outside 1..2^20, misaligned dst, a
 * descriptor the renderer would reject), ISAAC_EGUARD (the reachable cells
 * leave the extent), ISAAC_ENOMEM (dst too small); nothing is enqueued then.
 */
typedef void (*isaac_update_fn)(int32_t source, int32_t enabled, void *user);
int isaac_set_update_hook(isaac_update_fn fn, void *user);
int isaac_copy_source(const isaac_source *src, const int64_t n[3], void *dst, int64_t dst_bytes,
                      isaac_source *out, void *stream);

/* Measurement aid (no counterpart in the paper): read `bytes` of device/* Measurement aid (no counterpart in the paper): read `bytes` of device
 * memory at `buf` (16-byte aligned) `passes` times with 16-byte loads cached
 * in L2 only; sink: device memory of 1024 uint32 the kernel may write.  The
 * bench times it on a buffer of half the L2 for the L2 bandwidth it reports. */
int isaac_probe_read(const void *buf, int64_t bytes, int32_t passes, uint32_t *sink, void *stream);

/* Free the render workspaces of the current device (synchronises the device). */
int isaac_release_workspaces(void);

/* Text of the last error reported to the calling thread ("" if none). */
const char *isaac_last_error(void);

/* ISAAC_ABI_VERSION of the loaded library. */
int isaac_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ISAAC_B300_H */
