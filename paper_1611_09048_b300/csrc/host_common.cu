// host_common.cu -- host-side validation shared by every entry point:
// error reporting, the FP64 camera inverse, functor-chain compilation, source
// and frame validation.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "common.h"
#include "raycast.cuh"

namespace isaac {

static thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

void clear_error() { g_last_error.clear(); }

const char *last_error() { return g_last_error.c_str(); }

int check_cuda(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ISAAC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return ISAAC_OK;
}

// ---------------------------------------------------------------- camera

// Column-major 4x4 product C = A * B.
static void mat_mul(const double *A, const double *B, double *C)
{
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s = fma(A[4 * k + r], B[4 * c + k], s);
            C[4 * c + r] = s;
        }
}

// Inverse by cofactor expansion (adjugate / determinant), in double.
static bool mat_inverse(const double *m, double *inv)
{
    double a[16];
    a[0] = m[5] * m[10] * m[15] - m[5] * m[11] * m[14] - m[9] * m[6] * m[15] + m[9] * m[7] * m[14] +
           m[13] * m[6] * m[11] - m[13] * m[7] * m[10];
    a[4] = -m[4] * m[10] * m[15] + m[4] * m[11] * m[14] + m[8] * m[6] * m[15] - m[8] * m[7] * m[14] -
           m[12] * m[6] * m[11] + m[12] * m[7] * m[10];
    a[8] = m[4] * m[9] * m[15] - m[4] * m[11] * m[13] - m[8] * m[5] * m[15] + m[8] * m[7] * m[13] +
           m[12] * m[5] * m[11] - m[12] * m[7] * m[9];
    a[12] = -m[4] * m[9] * m[14] + m[4] * m[10] * m[13] + m[8] * m[5] * m[14] - m[8] * m[6] * m[13] -
            m[12] * m[5] * m[10] + m[12] * m[6] * m[9];
    a[1] = -m[1] * m[10] * m[15] + m[1] * m[11] * m[14] + m[9] * m[2] * m[15] - m[9] * m[3] * m[14] -
           m[13] * m[2] * m[11] + m[13] * m[3] * m[10];
    a[5] = m[0] * m[10] * m[15] - m[0] * m[11] * m[14] - m[8] * m[2] * m[15] + m[8] * m[3] * m[14] +
           m[12] * m[2] * m[11] - m[12] * m[3] * m[10];
    a[9] = -m[0] * m[9] * m[15] + m[0] * m[11] * m[13] + m[8] * m[1] * m[15] - m[8] * m[3] * m[13] -
           m[12] * m[1] * m[11] + m[12] * m[3] * m[9];
    a[13] = m[0] * m[9] * m[14] - m[0] * m[10] * m[13] - m[8] * m[1] * m[14] + m[8] * m[2] * m[13] +
            m[12] * m[1] * m[10] - m[12] * m[2] * m[9];
    a[2] = m[1] * m[6] * m[15] - m[1] * m[7] * m[14] - m[5] * m[2] * m[15] + m[5] * m[3] * m[14] +
           m[13] * m[2] * m[7] - m[13] * m[3] * m[6];
    a[6] = -m[0] * m[6] * m[15] + m[0] * m[7] * m[14] + m[4] * m[2] * m[15] - m[4] * m[3] * m[14] -
           m[12] * m[2] * m[7] + m[12] * m[3] * m[6];
    a[10] = m[0] * m[5] * m[15] - m[0] * m[7] * m[13] - m[4] * m[1] * m[15] + m[4] * m[3] * m[13] +
            m[12] * m[1] * m[7] - m[12] * m[3] * m[5];
    a[14] = -m[0] * m[5] * m[14] + m[0] * m[6] * m[13] + m[4] * m[1] * m[14] - m[4] * m[2] * m[13] -
            m[12] * m[1] * m[6] + m[12] * m[2] * m[5];
    a[3] = -m[1] * m[6] * m[11] + m[1] * m[7] * m[10] + m[5] * m[2] * m[11] - m[5] * m[3] * m[10] -
           m[9] * m[2] * m[7] + m[9] * m[3] * m[6];
    a[7] = m[0] * m[6] * m[11] - m[0] * m[7] * m[10] - m[4] * m[2] * m[11] + m[4] * m[3] * m[10] +
           m[8] * m[2] * m[7] - m[8] * m[3] * m[6];
    a[11] = -m[0] * m[5] * m[11] + m[0] * m[7] * m[9] + m[4] * m[1] * m[11] - m[4] * m[3] * m[9] -
            m[8] * m[1] * m[7] + m[8] * m[3] * m[5];
    a[15] = m[0] * m[5] * m[10] - m[0] * m[6] * m[9] - m[4] * m[1] * m[10] + m[4] * m[2] * m[9] +
            m[8] * m[1] * m[6] - m[8] * m[2] * m[5];
    const double det = m[0] * a[0] + m[1] * a[4] + m[2] * a[8] + m[3] * a[12];
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
    const double id = 1.0 / det;
    for (int i = 0; i < 16; ++i) inv[i] = a[i] * id;
    return true;
}

// ------------------------------------------------------------ validation

static bool finite_n(const float *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Compile one public chain into the kernel's op list.  Consecutive ADD/MUL
// functors fold into one AFFINE op (a*x + b per component, one FMA), identity
// ADD(0)/MUL(1) disappear, POW with every exponent 1/2 becomes SQRT.  Folding
// changes rounding only at the level of one float32 operation per functor.
int compile_chain(const isaac_chain &in, int fdim, int s, KChain &out)
{
    if (in.n_ops < 0 || in.n_ops > ISAAC_MAX_FUNCTORS)
        return fail(ISAAC_EINVAL, "source %d: chain has %d functors (max %d)", s, in.n_ops,
                    ISAAC_MAX_FUNCTORS);
    int dim = fdim, n = 0;
    bool open_affine = false;   // the last emitted op is an AFFINE that can absorb more
    for (int i = 0; i < in.n_ops; ++i) {
        const isaac_functor &f = in.ops[i];
        float arg[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (f.op == ISAAC_OP_ADD || f.op == ISAAC_OP_MUL || f.op == ISAAC_OP_POW) {
            if (f.n_args != 1 && f.n_args != dim)
                return fail(ISAAC_EINVAL,
                            "source %d functor %d: %d arguments for a %d-component value "
                            "(need 1 or %d)", s, i, f.n_args, dim, dim);
            if (!finite_n(f.arg, f.n_args))
                return fail(ISAAC_EINVAL, "source %d functor %d: non-finite argument", s, i);
            for (int c = 0; c < 4; ++c) arg[c] = f.n_args == 1 ? f.arg[0] : (c < dim ? f.arg[c] : 0.0f);
        }
        switch (f.op) {
        case ISAAC_OP_ADD:
        case ISAAC_OP_MUL: {
            const bool add = f.op == ISAAC_OP_ADD;
            bool identity = true;
            for (int c = 0; c < dim; ++c) identity &= add ? arg[c] == 0.0f : arg[c] == 1.0f;
            if (identity) break;
            if (!open_affine) {
                KOp &o = out.op[n++];
                o.code = K_AFFINE;
                o.dim = dim;
                for (int c = 0; c < 4; ++c) {
                    o.a[c] = 1.0f;
                    o.b[c] = 0.0f;
                }
                open_affine = true;
            }
            KOp &o = out.op[n - 1];
            for (int c = 0; c < 4; ++c) {
                if (add) {
                    o.b[c] += arg[c];
                } else {
                    o.a[c] *= arg[c];
                    o.b[c] *= arg[c];
                }
            }
        } break;
        case ISAAC_OP_POW: {
            KOp &o = out.op[n++];
            o.dim = dim;
            bool all_half = true;
            for (int c = 0; c < dim; ++c) all_half &= (arg[c] == 0.5f);
            o.code = all_half ? K_SQRT : K_POW;
            for (int c = 0; c < 4; ++c) {
                o.a[c] = arg[c];
                o.b[c] = 0.0f;
            }
            open_affine = false;
        } break;
        case ISAAC_OP_LENGTH:
        case ISAAC_OP_SUM:
        case ISAAC_OP_LOG: {
            KOp &o = out.op[n++];
            o.dim = dim;
            o.code = f.op == ISAAC_OP_LENGTH ? K_LENGTH : f.op == ISAAC_OP_SUM ? K_SUM : K_LOG;
            for (int c = 0; c < 4; ++c) o.a[c] = o.b[c] = 0.0f;
            if (f.op != ISAAC_OP_LOG) dim = 1;
            open_affine = false;
        } break;
        default:
            return fail(ISAAC_EINVAL, "source %d functor %d: unknown op %d", s, i, f.op);
        }
    }
    out.n = n;
    const int c0 = n > 0 ? out.op[0].code : 0, c1 = n > 1 ? out.op[1].code : 0;
    const int c2 = n > 2 ? out.op[2].code : 0;
    out.shape = CH_GENERIC;
    if (n == 0) out.shape = CH_IDENTITY;
    else if (n == 1 && c0 == K_AFFINE) out.shape = CH_AFFINE;
    else if (n == 1 && c0 == K_LENGTH) out.shape = CH_LENGTH;
    else if (n == 2 && c0 == K_LENGTH && c1 == K_AFFINE) out.shape = CH_LENGTH_AFFINE;
    else if (n == 3 && c0 == K_LENGTH && c1 == K_AFFINE && c2 == K_SQRT) out.shape = CH_LENGTH_AFFINE_SQRT;
    else if (n == 1 && c0 == K_LOG) out.shape = CH_LOG;
    else if (n == 2 && c0 == K_LOG && c1 == K_AFFINE) out.shape = CH_LOG_AFFINE;
    for (int i = n; i < ISAAC_MAX_FUNCTORS; ++i) {
        out.op[i].code = 0;
        out.op[i].dim = 1;
        for (int c = 0; c < 4; ++c) out.op[i].a[c] = out.op[i].b[c] = 0.0f;
    }
    return ISAAC_OK;
}

// Validate one source's reachable cells against its extent and fill the
// kernel descriptor.  elem = bytes per element.  Returns the signature
// nibble via *nib and whether 64-bit offsets are needed via *wide.
int prepare_source(const isaac_source &src, int s, const int64_t n[3], int interp, float weight,
                   int elem, KSource &ks, unsigned *nib, bool *wide, int reach)
{
    if (!src.ptr) return fail(ISAAC_EINVAL, "source %d: NULL pointer for an active source", s);
    if (src.f_dim < 1 || src.f_dim > 4)
        return fail(ISAAC_EINVAL, "source %d: f_dim %d outside 1..4", s, src.f_dim);
    if (src.guard < 0) return fail(ISAAC_EINVAL, "source %d: negative guard", s);
    if (src.extent <= 0 || src.offset < 0)
        return fail(ISAAC_EINVAL, "source %d: extent %lld / offset %lld", s, (long long)src.extent,
                    (long long)src.offset);
    if (((uintptr_t)src.ptr) % (uintptr_t)elem != 0)
        return fail(ISAAC_EINVAL, "source %d: pointer not aligned to its element size", s);
    // guard layers read: one for the samples (positions in [0, n)), up to
    // `reach` for positions beyond the box (iso-surface gradients)
    const int g1 = interp ? std::min(src.guard, std::max(reach, 1)) : 0;
    // smallest and largest element index any sample can read
    long double lo = (long double)src.offset, hi = lo, span = 0.0L;
    for (int a = 0; a < 3; ++a) {
        const long double i0 = -g1, i1 = (long double)(n[a] - 1 + g1);
        const long double st = (long double)src.stride[a];
        lo += std::fmin(i0 * st, i1 * st);
        hi += std::fmax(i0 * st, i1 * st);
        span += std::fmax(std::fabs(i0 * st), std::fabs(i1 * st));
    }
    const long double cst = (long double)(src.f_dim - 1) * (long double)src.comp_stride;
    lo += std::fmin(0.0L, cst);
    hi += std::fmax(0.0L, cst);
    span += std::fabs(cst);
    if (lo < 0.0L || hi >= (long double)src.extent)
        return fail(ISAAC_EGUARD,
                    "source %d: cells reachable with guard %d span elements [%.0Lf, %.0Lf] but the "
                    "extent is %lld", s, src.guard, lo, hi, (long long)src.extent);
    *wide = span >= 2147483647.0L;
    ks.base = reinterpret_cast<const float *>(static_cast<const char *>(src.ptr) +
                                              (size_t)src.offset * (size_t)elem);
    ks.sx = src.stride[0];
    ks.sy = src.stride[1];
    ks.sz = src.stride[2];
    ks.sc = src.comp_stride;
    ks.fdim = src.f_dim;
    ks.lo = -g1;
    ks.hi_pad = g1;
    ks.w = weight;
    *nib = (unsigned)src.f_dim | ((src.f_dim == 1 || src.comp_stride == 1) ? 8u : 0u);
    return ISAAC_OK;
}

// A double as the nearest float plus the float nearest to the remainder.
static ff split_ff(double v)
{
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

// Common validation of everything but the sources; fills the geometric part
// of KParams.
int prepare_frame(const isaac_camera *cam, const isaac_plane *clip, int32_t n_clip,
                  const isaac_render_opts *opt, KParams &p)
{
    if (!cam || !opt) return fail(ISAAC_EINVAL, "camera and opts are required");
    if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
        return fail(ISAAC_EINVAL, "image size %dx%d outside 1..32768", cam->width, cam->height);
    for (int a = 0; a < 3; ++a) {
        if (opt->n[a] < 1 || opt->n[a] > (1 << 30))
            return fail(ISAAC_EINVAL, "volume size n[%d] = %lld", a, (long long)opt->n[a]);
        if (opt->offset[a] < 0) return fail(ISAAC_EINVAL, "negative offset[%d]", a);
    }
    const bool same = opt->global_n[0] == 0 && opt->global_n[1] == 0 && opt->global_n[2] == 0;
    int64_t gn[3];
    for (int a = 0; a < 3; ++a) {
        gn[a] = same ? opt->n[a] : opt->global_n[a];
        if (opt->offset[a] + opt->n[a] > gn[a])
            return fail(ISAAC_EINVAL, "local box [%lld, %lld) exceeds the global size %lld on axis %d",
                        (long long)opt->offset[a], (long long)(opt->offset[a] + opt->n[a]),
                        (long long)gn[a], a);
    }
    if (opt->flags & ~(ISAAC_LUTS_HOST | ISAAC_MARCH_STAGED)) return fail(ISAAC_EINVAL, "unknown opts.flags bits 0x%x", opt->flags);
    if (!(opt->step > 0.0f) || !std::isfinite(opt->step))
        return fail(ISAAC_EINVAL, "step must be positive and finite");
    if (opt->interp != 0 && opt->interp != 1) return fail(ISAAC_EINVAL, "interp must be 0 or 1");
    if (std::isnan(opt->term_alpha)) return fail(ISAAC_EINVAL, "term_alpha is NaN");
    if (!finite_n(opt->bg, 4)) return fail(ISAAC_EINVAL, "background is not finite");
    const int lpr = opt->lanes_per_ray;
    if (lpr != 0 && lpr != 1 && lpr != 2 && lpr != 4 && lpr != 8 && lpr != 16)
        return fail(ISAAC_EINVAL, "lanes_per_ray must be 0, 1, 2, 4, 8 or 16");
    if (n_clip < 0 || n_clip > ISAAC_MAX_CLIP)
        return fail(ISAAC_EINVAL, "%d clip planes (max %d)", n_clip, ISAAC_MAX_CLIP);
    if (n_clip > 0 && !clip) return fail(ISAAC_EINVAL, "clip is NULL with n_clip > 0");
    for (int i = 0; i < n_clip; ++i)
        for (int j = 0; j < 4; ++j) {
            const double v = j < 3 ? clip[i].n[j] : clip[i].d;
            if (!std::isfinite(v)) return fail(ISAAC_EINVAL, "clip plane %d is not finite", i);
            p.clip[i][j] = v;
        }
    p.n_clip = n_clip;

    double M[16];
    mat_mul(cam->projection, cam->modelview, M);
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(M[i])) return fail(ISAAC_EINVAL, "camera matrices are not finite");
    if (!mat_inverse(M, p.minv)) return fail(ISAAC_EINVAL, "projection * modelview is singular");

    p.W = cam->width;
    p.H = cam->height;
    p.ndc_sx = 2.0 / (double)cam->width;
    p.ndc_sy = 2.0 / (double)cam->height;
    p.nx = (int)opt->n[0];
    p.ny = (int)opt->n[1];
    p.nz = (int)opt->n[2];
    for (int a = 0; a < 3; ++a) {
        p.gn[a] = (double)gn[a];
        p.half_g[a] = 0.5 * (double)gn[a];
        p.llo[a] = (double)opt->offset[a];
        p.lhi[a] = (double)(opt->offset[a] + opt->n[a]);
    }
    p.local_is_global = 1;
    for (int a = 0; a < 3; ++a)
        if (opt->offset[a] != 0 || opt->n[a] != gn[a]) p.local_is_global = 0;
    p.step = opt->step;
    p.step_d = (double)opt->step;
    p.inv_step_d = 1.0 / p.step_d;

    // Float-float copies for the device ray setup.  With X = px + 1/2 - W/2
    // and Y = py + 1/2 - H/2 the NDC coordinates are xn = X (2/W) and
    // yn = -Y (2/H); the homogeneous point at depth z is
    // minv (xn, yn, z, 1), moved to global voxel coordinates by adding
    // half_g times its w component before the division.
    p.pix_cx = 0.5f * (float)(cam->width - 1);
    p.pix_cy = 0.5f * (float)(cam->height - 1);
    for (int e = 0; e < 2; ++e) {
        const double z = e == 0 ? -1.0 : 1.0;
        double c[3][4];
        for (int i = 0; i < 4; ++i) {
            c[0][i] = p.minv[8 + i] * z + p.minv[12 + i];
            c[1][i] = p.minv[i] * p.ndc_sx;
            c[2][i] = -p.minv[4 + i] * p.ndc_sy;
        }
        for (int k = 0; k < 3; ++k) {
            for (int a = 0; a < 3; ++a) c[k][a] += p.half_g[a] * c[k][3];
            for (int i = 0; i < 4; ++i) p.ray[e][k][i] = split_ff(c[k][i]);
        }
    }
    for (int a = 0; a < 3; ++a) {
        p.gn_f[a] = split_ff(p.gn[a]);
        p.llo_f[a] = split_ff(p.llo[a]);
        p.lhi_f[a] = split_ff(p.lhi[a]);
    }
    for (int i = 0; i < n_clip; ++i)
        for (int j = 0; j < 4; ++j) p.clip_f[i][j] = split_ff(p.clip[i][j]);
    p.inv_step_f = split_ff(p.inv_step_d);
    // every ray's samples lie on one chord of the local box
    const double diag = std::sqrt((double)opt->n[0] * opt->n[0] + (double)opt->n[1] * opt->n[1] +
                                  (double)opt->n[2] * opt->n[2]);
    const double max_steps = std::ceil(diag / (double)opt->step) + 2.0;
    if (max_steps > (double)(1 << 24))
        return fail(ISAAC_EINVAL, "step %g gives up to %.0f samples per ray (max %d)",
                    (double)opt->step, max_steps, 1 << 24);
    p.max_steps = (int)max_steps;
    p.term = opt->term_alpha;
    for (int c = 0; c < 4; ++c) p.bg[c] = opt->bg[c];

    // Screen rectangle: project the 8 corners of the local box, cut by the
    // axis-aligned clip planes (others are ignored, which only widens it); a
    // pixel whose ray can reach a sample lies in their bounding box (one-pixel
    // margin for rounding).  A box cut to nothing keeps one face, so rays that
    // graze it stay inside the margin.
    double blo[3], bhi[3];
    for (int a = 0; a < 3; ++a) {
        blo[a] = p.llo[a];
        bhi[a] = p.lhi[a];
    }
    for (int i = 0; i < n_clip; ++i) {
        const double *pl = p.clip[i];
        int axis = -1, nonzero = 0;
        for (int a = 0; a < 3; ++a)
            if (pl[a] != 0.0) {
                axis = a;
                ++nonzero;
            }
        if (nonzero != 1) continue;
        const double c = -pl[3] / pl[axis];    // keep x_axis >= c (normal > 0) or <= c
        if (pl[axis] > 0.0)
            blo[axis] = std::fmin(std::fmax(blo[axis], c), bhi[axis]);
        else
            bhi[axis] = std::fmax(std::fmin(bhi[axis], c), blo[axis]);
    }
    bool full = false;
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int c = 0; c < 8; ++c) {
        const double w[3] = {((c & 1) ? bhi[0] : blo[0]) - p.half_g[0],
                             ((c & 2) ? bhi[1] : blo[1]) - p.half_g[1],
                             ((c & 4) ? bhi[2] : blo[2]) - p.half_g[2]};
        double v[4];
        for (int r = 0; r < 4; ++r) v[r] = M[r] * w[0] + M[4 + r] * w[1] + M[8 + r] * w[2] + M[12 + r];
        if (!(v[3] > 1e-12)) {
            full = true;
            break;
        }
        const double sx = (v[0] / v[3] + 1.0) * 0.5 * cam->width - 0.5;
        const double sy = (1.0 - v[1] / v[3]) * 0.5 * cam->height - 0.5;
        xmin = std::fmin(xmin, sx);
        xmax = std::fmax(xmax, sx);
        ymin = std::fmin(ymin, sy);
        ymax = std::fmax(ymax, sy);
    }
    if (full) {
        p.rx0 = p.ry0 = 0;
        p.rx1 = cam->width;
        p.ry1 = cam->height;
    } else {
        p.rx0 = (int)std::fmax(0.0, std::fmin((double)cam->width, std::floor(xmin) - 1.0));
        p.rx1 = (int)std::fmax(0.0, std::fmin((double)cam->width, std::ceil(xmax) + 2.0));
        p.ry0 = (int)std::fmax(0.0, std::fmin((double)cam->height, std::floor(ymin) - 1.0));
        p.ry1 = (int)std::fmax(0.0, std::fmin((double)cam->height, std::ceil(ymax) + 2.0));
        if (p.rx1 <= p.rx0 || p.ry1 <= p.ry0) p.rx0 = p.rx1 = p.ry0 = p.ry1 = 0;
    }
    return ISAAC_OK;
}

int prepare_fb(const isaac_framebuffer *fb, KParams &p)
{
    if (!fb || !fb->rgba8) return fail(ISAAC_EINVAL, "fb->rgba8 is required");
    if (((uintptr_t)fb->rgba8) % 4 || ((uintptr_t)fb->rgba32) % 16 || ((uintptr_t)fb->nsamples) % 4)
        return fail(ISAAC_EINVAL, "framebuffer pointers are misaligned");
    p.fb8 = reinterpret_cast<uchar4 *>(fb->rgba8);
    p.fb32 = reinterpret_cast<float4 *>(fb->rgba32);
    p.nsamp = fb->nsamples;
    if (((uintptr_t)fb->touched) % 4) return fail(ISAAC_EINVAL, "fb->touched is misaligned");
    p.touched = reinterpret_cast<unsigned *>(fb->touched);
    if (((uintptr_t)fb->depth) % 4) return fail(ISAAC_EINVAL, "fb->depth is misaligned");
    p.depth = fb->depth;
    return ISAAC_OK;
}

}  // namespace isaac
