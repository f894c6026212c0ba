/*
 * isaac_oracle.c -- plain, slow FP64 CPU reference of ISAAC's per-pixel
 * volume ray caster (Matthes et al., "In situ, steerable, hardware-independent
 * and data-structure agnostic visualization with ISAAC", 2016).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file: it exists so that tests, the smoke check and the CPU baseline
 * leg of the benchmark can compare the CUDA path against an independent
 * definition.  It shares no code, header, table or constant with the CUDA
 * library; its own structures below are deliberately separate.
 *
 * What it computes, per pixel, serially and in double precision (Sec. 3.2:
 * at every sample point of a pixel's ray, each source's value goes through
 * its functor chain and transfer function, the sources' colours and
 * opacities are combined into one, and the ray composites front to back):
 *
 *   1. camera: M = P * MV, inverted by Gauss-Jordan elimination with partial
 *      pivoting; the pixel centre is unprojected at NDC depth -1 and +1 and
 *      mapped from world to global voxel coordinates (world = voxel - gn/2);
 *   2. the slab test against the global box [0,gn)^3 gives the ray's entry
 *      t0 (not before the near plane, t >= 0); the node's local box
 *      [off, off+n)^3 (Sec. 3.1: every node owns a disjoint cuboid of the
 *      global volume) and every clip plane (keep nx*x+ny*y+nz*z+d >= 0 in
 *      global voxel coordinates, Sec. 3 feature list: clipping planes) give
 *      the sampled interval [t_in, t_out];
 *   3. samples t_k = t0 + k*step for integer k with t_in <= t_k < t_out: one
 *      sample grid anchored at the unclipped global entry, so that local
 *      images of neighbouring nodes composite to the image of the whole;
 *   4. per active source (Sec. 3.2 compiles one render function per subset
 *      of active sources: inactive sources are never read): cell-centred trilinear interpolation (value i sits at
 *      i + 1/2; guard cells are read when present, otherwise indices clamp to
 *      the border, Sec. 3.1/3.2 guard cells), or the nearest cell when
 *      interpolation is off; then the source's functor chain (Sec. 3.3,
 *      Table 1, default reduction to the first component), then the 256-entry
 *      RGBA transfer function with linear interpolation between entries;
 *   5. weighted sum of the sources' RGBA, alpha clamped to [0,1];
 *   6. front-to-back compositing C += (1-A)*a*rgb, A += (1-A)*a, stopping
 *      once A >= term;
 *   7. background blend out = (C,A) + (1-A)*bg, and 8-bit quantisation
 *      min(255, floor(255*clamp(x,0,1) + 1/2)).
 *
 * Beside the image it reports, per pixel, the sample count and the decision
 * margins of every discrete choice (entry and exit sample index, termination
 * step, nearest-cell choice) and, for the termination step, the alternative
 * result that the nearer opposite decision would give.  A reduced-precision
 * implementation may legitimately take the other side of a decision whose
 * margin is below its own rounding error; the alternative lets a test accept
 * exactly that and nothing else.
 *
 * Readings of points the paper leaves open are fixed in the build's design
 * notes and restated at each function below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_OPS 16
#define ORC_MAX_CLIP 16
#define ORC_MAX_SRC 16
#define ORC_INF 1.0e300

enum { ORC_ADD = 1, ORC_MUL = 2, ORC_LENGTH = 3, ORC_SUM = 4, ORC_POW = 5, ORC_LOG = 6 };

typedef struct {
    const float *data;   /* host storage of the source */
    int64_t offset;      /* element index of interior cell (0,0,0), component 0 */
    int64_t stride[3];   /* elements between neighbouring cells along x, y, z */
    int64_t cstride;     /* elements between components */
    int32_t fdim;        /* feature dimension 1..4 (Sec. 3.2) */
    int32_t guard;       /* ghost cells per side present in the storage */
} orc_source;

typedef struct {
    int32_t op;          /* ORC_ADD .. ORC_LOG */
    int32_t nargs;       /* 1 = scalar broadcast (Sec. 3.3: add(1) = (1,1,1)), else one per component */
    double arg[4];
} orc_functor;

typedef struct {
    int32_t nops;
    orc_functor ops[ORC_MAX_OPS];
} orc_chain;

typedef struct {
    int64_t n[3];               /* interior cells of the local volume */
    int64_t gn[3];              /* cells of the global volume (Sec. 3.1) */
    int64_t off[3];             /* position of the local volume inside the global one */
    double modelview[16];       /* column-major */
    double projection[16];      /* column-major */
    int32_t width, height;
    int32_t n_clip;
    double clip[ORC_MAX_CLIP][4];
    double step;
    int32_t interp;             /* 1 trilinear, 0 nearest */
    double term;                /* early termination threshold on A */
    double bg[4];
    uint32_t active_mask;
} orc_params;

typedef struct {
    double *rgba;        /* 4 per pixel, unquantised */
    double *rgba_alt;    /* 4 per pixel, result of the nearer opposite termination decision */
    uint8_t *rgba8;      /* 4 per pixel */
    uint8_t *rgba8_alt;  /* 4 per pixel */
    int32_t *nsamp;      /* composited samples */
    int32_t *nsamp_alt;
    double *margin;      /* 4 per pixel: entry, exit (in steps), termination (in A), nearest (in voxels) */
    int32_t *kfirst;     /* first sample index on the global grid, -1 on a miss */
    int32_t *jspan;      /* 2 per pixel: first and last composited sample with opacity > 0,
                            counted from the ray's first sample; -1 if none */
} orc_outputs;

/* ---------------------------------------------------------------- camera */

/* C = A * B for column-major 4x4 matrices. */
static void orc_matmul4(const double *A, const double *B, double *C)
{
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += A[k * 4 + r] * B[c * 4 + k];
            C[c * 4 + r] = s;
        }
}

/* Gauss-Jordan elimination with partial pivoting; returns 0 on success. */
int orc_invert4(const double *M, double *Minv)
{
    double a[4][8];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            a[r][c] = M[c * 4 + r];
            a[r][c + 4] = (r == c) ? 1.0 : 0.0;
        }
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int c = 0; c < 8; ++c) { double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t; }
        double inv = 1.0 / a[col][col];
        for (int c = 0; c < 8; ++c) a[col][c] *= inv;
        for (int r = 0; r < 4; ++r) {
            if (r == col) continue;
            double f = a[r][col];
            if (f != 0.0)
                for (int c = 0; c < 8; ++c) a[r][c] -= f * a[col][c];
        }
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) Minv[c * 4 + r] = a[r][c + 4];
    return 0;
}

/* Unproject NDC (x, y, z) through Minv and dehomogenise. */
static void orc_unproject(const double *Minv, double x, double y, double z, double out[3])
{
    double v[4];
    for (int r = 0; r < 4; ++r)
        v[r] = Minv[0 * 4 + r] * x + Minv[1 * 4 + r] * y + Minv[2 * 4 + r] * z + Minv[3 * 4 + r];
    out[0] = v[0] / v[3];
    out[1] = v[1] / v[3];
    out[2] = v[2] / v[3];
}

/* ------------------------------------------------------------- sampling */

static int64_t orc_axis_index(int64_t i, int64_t n, int32_t guard)
{
    /* guard == 0: no neighbour data, clamp to the border cell; otherwise the
     * guard cells hold the neighbour's values (Sec. 3.1/3.2).  Every position
     * the readings below interpolate at reads inside [-guard, n - 1 + guard];
     * the clamp to that range only keeps a corner of weight zero at the edge
     * of the guard layers (an iso-surface gradient position) in the array. */
    if (guard == 0) {
        if (i < 0) return 0;
        if (i > n - 1) return n - 1;
    }
    if (i < -(int64_t)guard) return -(int64_t)guard;
    if (i > n - 1 + guard) return n - 1 + guard;
    return i;
}

static void orc_fetch(const orc_source *s, int64_t ix, int64_t iy, int64_t iz, double *v)
{
    const float *b = s->data + s->offset + ix * s->stride[0] + iy * s->stride[1] + iz * s->stride[2];
    for (int c = 0; c < s->fdim; ++c) v[c] = (double)b[c * s->cstride];
}

/* Value of a source at voxel position p: cell-centred trilinear interpolation,
 * or the containing cell when interpolation is off (Sec. 3 feature list:
 * optional interpolation). */
static void orc_sample(const orc_source *s, const int64_t n[3], const double p[3], int interp,
                       double *v)
{
    int fd = s->fdim;
    if (!interp) {
        int64_t idx[3];
        for (int a = 0; a < 3; ++a) {
            int64_t i = (int64_t)floor(p[a]);
            if (i < 0) i = 0;
            if (i > n[a] - 1) i = n[a] - 1;
            idx[a] = i;
        }
        orc_fetch(s, idx[0], idx[1], idx[2], v);
        return;
    }
    int64_t i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double q = p[a] - 0.5;
        double fl = floor(q);
        i0[a] = (int64_t)fl;
        f[a] = q - fl;
    }
    for (int c = 0; c < fd; ++c) v[c] = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double w = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) * (cz ? f[2] : 1.0 - f[2]);
                double corner[4];
                orc_fetch(s, orc_axis_index(i0[0] + cx, n[0], s->guard),
                          orc_axis_index(i0[1] + cy, n[1], s->guard),
                          orc_axis_index(i0[2] + cz, n[2], s->guard), corner);
                for (int c = 0; c < fd; ++c) v[c] += w * corner[c];
            }
}

/* ---------------------------------------------------------- functor chain */

static double orc_arg(const orc_functor *f, int c) { return f->nargs == 1 ? f->arg[0] : f->arg[c]; }

/* Sec. 3.3, Table 1: add(v), mul(v) componentwise with scalar broadcast;
 * length and sum reduce to a scalar; pow(v) exponentiates componentwise.
 * Readings: pow of a non-positive base gives 0; the user functor log takes
 * log(max(x, 1e-30)).  Without an explicit reduction the first component is
 * used (Sec. 3.3). */
static double orc_chain_apply(const orc_chain *ch, double *v, int dim)
{
    for (int i = 0; i < ch->nops; ++i) {
        const orc_functor *f = &ch->ops[i];
        switch (f->op) {
        case ORC_ADD:
            for (int c = 0; c < dim; ++c) v[c] += orc_arg(f, c);
            break;
        case ORC_MUL:
            for (int c = 0; c < dim; ++c) v[c] *= orc_arg(f, c);
            break;
        case ORC_LENGTH: {
            double s = 0.0;
            for (int c = 0; c < dim; ++c) s += v[c] * v[c];
            v[0] = sqrt(s);
            dim = 1;
        } break;
        case ORC_SUM: {
            double s = 0.0;
            for (int c = 0; c < dim; ++c) s += v[c];
            v[0] = s;
            dim = 1;
        } break;
        case ORC_POW:
            for (int c = 0; c < dim; ++c) v[c] = v[c] > 0.0 ? pow(v[c], orc_arg(f, c)) : 0.0;
            break;
        case ORC_LOG:
            for (int c = 0; c < dim; ++c) v[c] = log(v[c] > 1e-30 ? v[c] : 1e-30);
            break;
        default:
            break;
        }
    }
    return v[0];
}

/* Validate a chain against a source's feature dimension; returns 0 if valid. */
static int orc_chain_check(const orc_chain *ch, int dim)
{
    if (ch->nops < 0 || ch->nops > ORC_MAX_OPS) return -1;
    for (int i = 0; i < ch->nops; ++i) {
        const orc_functor *f = &ch->ops[i];
        switch (f->op) {
        case ORC_ADD: case ORC_MUL: case ORC_POW:
            if (f->nargs != 1 && f->nargs != dim) return -1;
            break;
        case ORC_LENGTH: case ORC_SUM:
            dim = 1;
            break;
        case ORC_LOG:
            break;
        default:
            return -1;
        }
    }
    return 0;
}

/* ------------------------------------------------------- classification */

/* Transfer function (Sec. 3 feature list: user-defined transfer functions): the
 * scalar is clamped to [0,1] (NaN -> 0) and the 256 RGBA entries, entry j at
 * j/255, are interpolated linearly. */
static void orc_classify(const float *lut, double x, double rgba[4])
{
    if (!(x >= 0.0)) x = 0.0;
    if (x > 1.0) x = 1.0;
    double pos = 255.0 * x;
    int j = (int)floor(pos);
    if (j > 254) j = 254;
    double f = pos - (double)j;
    for (int c = 0; c < 4; ++c)
        rgba[c] = (1.0 - f) * (double)lut[j * 4 + c] + f * (double)lut[(j + 1) * 4 + c];
}

static uint8_t orc_quant8(double x)
{
    if (!(x >= 0.0)) x = 0.0;
    if (x > 1.0) x = 1.0;
    double q = floor(255.0 * x + 0.5);
    return (uint8_t)(q > 255.0 ? 255.0 : q);
}

static double orc_dist_int(double x)
{
    return fabs(x - floor(x + 0.5));
}

/* ------------------------------------------------------------- the frame */

typedef struct {
    const orc_params *p;
    const orc_source *src;
    const orc_chain *ch;
    const float *luts;
    const double *w;
    int32_t n_src;
    double Minv[16];
} orc_frame;

typedef struct {
    double C[3], A;
    int32_t n;
    int64_t jf, jl;   /* first / last composited sample index with opacity > 0, -1 if none */
} orc_state;

/* Composite the samples k in [k_begin, k_end) starting from state *st.
 * Termination is tested after every composited sample unless k equals
 * skip_term_at.  Returns the index of the sample at which it stopped, or -1. */
static int64_t orc_march(const orc_frame *F, const double o[3], const double d[3], double t0,
                         int64_t k_begin, int64_t k_end, int64_t skip_term_at, orc_state *st,
                         orc_state *before_stop, double *m_near)
{
    const orc_params *p = F->p;
    for (int64_t k = k_begin; k < k_end; ++k) {
        double t = t0 + (double)k * p->step;
        double pos[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        if (!p->interp && m_near)
            for (int a = 0; a < 3; ++a) {
                /* only boundaries between two interior cells are decisions: at
                 * the faces 0 and n both sides clamp to the same cell */
                double r = floor(pos[a] + 0.5);
                if (r <= 0.0 || r >= (double)p->n[a]) continue;
                double m = fabs(pos[a] - r);
                if (m < *m_near) *m_near = m;
            }
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int s = 0; s < F->n_src; ++s) {
            if (!((p->active_mask >> s) & 1u)) continue;
            double v[4];
            orc_sample(&F->src[s], p->n, pos, p->interp, v);
            double x = orc_chain_apply(&F->ch[s], v, F->src[s].fdim);
            double rgba[4];
            orc_classify(F->luts + (size_t)s * 256 * 4, x, rgba);
            for (int c = 0; c < 4; ++c) acc[c] += F->w[s] * rgba[c];
        }
        double a = acc[3];
        if (!(a >= 0.0)) a = 0.0;
        if (a > 1.0) a = 1.0;
        if (before_stop) *before_stop = *st;
        if (a > 0.0) {
            if (st->jf < 0) st->jf = k;
            st->jl = k;
        }
        double tf = (1.0 - st->A) * a;
        for (int c = 0; c < 3; ++c) st->C[c] += tf * acc[c];
        st->A += tf;
        st->n += 1;
        if (k != skip_term_at && st->A >= p->term) return k;
    }
    return -1;
}

static void orc_finish(const orc_params *p, const orc_state *st, double out[4])
{
    for (int c = 0; c < 3; ++c) out[c] = st->C[c] + (1.0 - st->A) * p->bg[c];
    out[3] = st->A + (1.0 - st->A) * p->bg[3];
}

static void orc_pixel(const orc_frame *F, int64_t pix, const orc_outputs *out, int64_t slot)
{
    const orc_params *p = F->p;
    int64_t px = pix % p->width, py = pix / p->width;
    double res[4], alt[4];
    double m_in = ORC_INF, m_out = ORC_INF, m_term = ORC_INF, m_near = ORC_INF;
    int32_t ns = 0, ns_alt = 0;
    int64_t kf_out = -1;

    double xn = 2.0 * ((double)px + 0.5) / (double)p->width - 1.0;
    double yn = 1.0 - 2.0 * ((double)py + 0.5) / (double)p->height;
    double nw[3], fw[3], o[3], d[3];
    orc_unproject(F->Minv, xn, yn, -1.0, nw);
    orc_unproject(F->Minv, xn, yn, 1.0, fw);
    for (int a = 0; a < 3; ++a) {
        o[a] = nw[a] + 0.5 * (double)p->gn[a];
        d[a] = fw[a] - nw[a];
    }
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int a = 0; a < 3; ++a) d[a] /= len;

    int miss = 0;
    double t0 = 0.0, tg1 = ORC_INF;       /* global box */
    double tl0 = 0.0, t_out = ORC_INF;    /* local box */
    for (int a = 0; a < 3; ++a) {
        double g_lo = 0.0, g_hi = (double)p->gn[a];
        double l_lo = (double)p->off[a], l_hi = (double)(p->off[a] + p->n[a]);
        if (d[a] != 0.0) {
            double ta = (g_lo - o[a]) / d[a], tb = (g_hi - o[a]) / d[a];
            double lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
            if (lo > t0) t0 = lo;
            if (hi < tg1) tg1 = hi;
            ta = (l_lo - o[a]) / d[a];
            tb = (l_hi - o[a]) / d[a];
            lo = ta < tb ? ta : tb;
            hi = ta < tb ? tb : ta;
            if (lo > tl0) tl0 = lo;
            if (hi < t_out) t_out = hi;
        } else if (o[a] < l_lo || o[a] >= l_hi) {
            miss = 1;
        }
    }
    if (t0 >= tg1) miss = 1;
    double t_in = tl0 > t0 ? tl0 : t0;
    for (int i = 0; i < p->n_clip && !miss; ++i) {
        const double *pl = p->clip[i];
        double s = pl[0] * o[0] + pl[1] * o[1] + pl[2] * o[2] + pl[3];
        double r = pl[0] * d[0] + pl[1] * d[1] + pl[2] * d[2];
        if (r > 0.0) {
            double tc = -s / r;
            if (tc > t_in) t_in = tc;
        } else if (r < 0.0) {
            double tc = -s / r;
            if (tc < t_out) t_out = tc;
        } else if (s < 0.0) {
            miss = 1;
        }
    }
    int raised = t_in > t0;
    double ol[3] = {o[0] - (double)p->off[0], o[1] - (double)p->off[1], o[2] - (double)p->off[2]};
    orc_state st = {{0.0, 0.0, 0.0}, 0.0, 0, -1, -1};
    orc_state alt_st = st;
    if (!miss && t_in < t_out) {
        double ein = (t_in - t0) / p->step, eout = (t_out - t0) / p->step;
        int64_t kf = raised ? (int64_t)ceil(ein) : 0;
        int64_t ke = (int64_t)ceil(eout);
        if (raised) m_in = orc_dist_int(ein);
        m_out = orc_dist_int(eout);
        if (ke > kf) {
            kf_out = kf;
            orc_state before = st;
            int64_t kstop = orc_march(F, ol, d, t0, kf, ke, -1, &st, &before, &m_near);
            alt_st = st;
            if (kstop >= 0) {
                double over = st.A - p->term;          /* >= 0 */
                double under = p->term - before.A;     /* > 0 */
                if (kstop == kf) under = p->term;      /* nothing composited before */
                if (over <= under) {
                    m_term = over;
                    /* nearer opposite decision: do not stop at kstop */
                    alt_st = st;
                    orc_march(F, ol, d, t0, kstop + 1, ke, -1, &alt_st, NULL, NULL);
                } else {
                    m_term = under;
                    /* nearer opposite decision: stop one sample earlier */
                    alt_st = before;
                }
            } else {
                m_term = p->term - st.A;
            }
        }
    }
    ns = st.n;
    ns_alt = alt_st.n;
    orc_finish(p, &st, res);
    orc_finish(p, &alt_st, alt);

    if (out->rgba) memcpy(out->rgba + slot * 4, res, sizeof res);
    if (out->rgba_alt) memcpy(out->rgba_alt + slot * 4, alt, sizeof alt);
    if (out->rgba8)
        for (int c = 0; c < 4; ++c) out->rgba8[slot * 4 + c] = orc_quant8(res[c]);
    if (out->rgba8_alt)
        for (int c = 0; c < 4; ++c) out->rgba8_alt[slot * 4 + c] = orc_quant8(alt[c]);
    if (out->nsamp) out->nsamp[slot] = ns;
    if (out->nsamp_alt) out->nsamp_alt[slot] = ns_alt;
    if (out->kfirst) out->kfirst[slot] = (int32_t)kf_out;
    if (out->jspan) {
        out->jspan[slot * 2] = st.jf < 0 ? -1 : (int32_t)(st.jf - kf_out);
        out->jspan[slot * 2 + 1] = st.jl < 0 ? -1 : (int32_t)(st.jl - kf_out);
    }
    if (out->margin) {
        out->margin[slot * 4 + 0] = m_in;
        out->margin[slot * 4 + 1] = m_out;
        out->margin[slot * 4 + 2] = m_term;
        out->margin[slot * 4 + 3] = m_near;
    }
}

/* ------------------------------------------------------- iso surfaces */

/* Iso-surface rendering (Sec. 3 feature list; Sec. 4.2 shows such images).
 * The paper states no algorithm; this is the reading both sides implement:
 *
 *   samples t_k = t0 + k*step exactly as in the volume mode (same sample grid,
 *   same [t_in, t_out]); at each sample every active source s gives its chain
 *   value v_s (interpolated as in the volume mode);
 *   the surface is met at the first sample k where some v_s(k) >= iso[s];
 *   for each such source the crossing is refined by one secant step between
 *   k-1 and k: t = t_{k-1} + step*(iso - v(k-1)) / (v(k) - v(k-1)), or t = t_k
 *   when k is the ray's first sample; the smallest t wins (ties: lower s);
 *   at the hit point q the winning source's gradient is taken by central
 *   differences g_a = (v(q+) - v(q-)) / (q+ - q-)_a with q+- = q +- e_a, each
 *   clamped along a into the positions the source's own cells can
 *   interpolate (same interpolation): [1/2 - g, n + g - 1/2] with g >= 1
 *   guard cells (Sec. 3.1/3.2: guards carry the neighbour's values so that
 *   interpolation across a sub-volume face needs no exchange; from g = 2 on
 *   no hit inside the box is clamped, and a sub-volume's gradients equal the
 *   whole volume's), [0, n] without guards or with interpolation off;
 *   n = -g/|g| (n = -d if g = 0), turned towards the viewer (n.(-d) >= 0);
 *   headlight Blinn-Phong with light, view and half vector all -d:
 *   rgb = LUT_s(iso[s]).rgb * (1/4 + 3/4 * n.(-d)) + 1/4 * (n.(-d))^32,
 *   clamped to [0, 1], alpha 1; a ray without a hit shows the background.
 *
 * margin[6] per pixel: entry and exit (steps, as in the volume mode), the
 * smallest |v_s(k) - iso[s]| over the samples up to the hit (or all samples),
 * |v(k) - v(k-1)| of the winning refinement (INF at a first-sample hit),
 * |g|, and the hit distance t (-1 without a hit). */
static double orc_source_value(const orc_frame *F, int s, const double pos[3])
{
    double v[4];
    orc_sample(&F->src[s], F->p->n, pos, F->p->interp, v);
    return orc_chain_apply(&F->ch[s], v, F->src[s].fdim);
}

static void orc_pixel_iso(const orc_frame *F, const double *iso, int64_t pix, double *rgba,
                          uint8_t *rgba8, double *margin)
{
    const orc_params *p = F->p;
    int64_t px = pix % p->width, py = pix / p->width;
    double m_in = ORC_INF, m_out = ORC_INF, m_iso = ORC_INF, m_slope = ORC_INF, m_grad = ORC_INF;
    double t_hit = -1.0;
    double res[4] = {p->bg[0], p->bg[1], p->bg[2], p->bg[3]};

    double xn = 2.0 * ((double)px + 0.5) / (double)p->width - 1.0;
    double yn = 1.0 - 2.0 * ((double)py + 0.5) / (double)p->height;
    double nw[3], fw[3], o[3], d[3];
    orc_unproject(F->Minv, xn, yn, -1.0, nw);
    orc_unproject(F->Minv, xn, yn, 1.0, fw);
    for (int a = 0; a < 3; ++a) {
        o[a] = nw[a] + 0.5 * (double)p->gn[a];
        d[a] = fw[a] - nw[a];
    }
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int a = 0; a < 3; ++a) d[a] /= len;
    int miss = 0;
    double t0 = 0.0, tg1 = ORC_INF, tl0 = 0.0, t_out = ORC_INF;
    for (int a = 0; a < 3; ++a) {
        double g_lo = 0.0, g_hi = (double)p->gn[a];
        double l_lo = (double)p->off[a], l_hi = (double)(p->off[a] + p->n[a]);
        if (d[a] != 0.0) {
            double ta = (g_lo - o[a]) / d[a], tb = (g_hi - o[a]) / d[a];
            double lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
            if (lo > t0) t0 = lo;
            if (hi < tg1) tg1 = hi;
            ta = (l_lo - o[a]) / d[a];
            tb = (l_hi - o[a]) / d[a];
            lo = ta < tb ? ta : tb;
            hi = ta < tb ? tb : ta;
            if (lo > tl0) tl0 = lo;
            if (hi < t_out) t_out = hi;
        } else if (o[a] < l_lo || o[a] >= l_hi) {
            miss = 1;
        }
    }
    if (t0 >= tg1) miss = 1;
    double t_in = tl0 > t0 ? tl0 : t0;
    for (int i = 0; i < p->n_clip && !miss; ++i) {
        const double *pl = p->clip[i];
        double sd = pl[0] * o[0] + pl[1] * o[1] + pl[2] * o[2] + pl[3];
        double r = pl[0] * d[0] + pl[1] * d[1] + pl[2] * d[2];
        if (r > 0.0) {
            double tc = -sd / r;
            if (tc > t_in) t_in = tc;
        } else if (r < 0.0) {
            double tc = -sd / r;
            if (tc < t_out) t_out = tc;
        } else if (sd < 0.0) {
            miss = 1;
        }
    }
    int raised = t_in > t0;
    double ol[3] = {o[0] - (double)p->off[0], o[1] - (double)p->off[1], o[2] - (double)p->off[2]};
    if (!miss && t_in < t_out) {
        double ein = (t_in - t0) / p->step, eout = (t_out - t0) / p->step;
        int64_t kf = raised ? (int64_t)ceil(ein) : 0;
        int64_t ke = (int64_t)ceil(eout);
        if (raised) m_in = orc_dist_int(ein);
        m_out = orc_dist_int(eout);
        double prev[ORC_MAX_SRC];
        int win = -1;
        for (int64_t k = kf; k < ke && win < 0; ++k) {
            double t = t0 + (double)k * p->step;
            double pos[3] = {ol[0] + t * d[0], ol[1] + t * d[1], ol[2] + t * d[2]};
            double best = ORC_INF;
            for (int s = 0; s < F->n_src; ++s) {
                if (!((p->active_mask >> s) & 1u)) continue;
                double v = orc_source_value(F, s, pos);
                double m = fabs(v - iso[s]);
                if (m < m_iso) m_iso = m;
                if (v >= iso[s]) {
                    double th = t, slope = ORC_INF;
                    if (k > kf) {
                        slope = v - prev[s];
                        th = t - p->step + p->step * (iso[s] - prev[s]) / slope;
                    }
                    if (th < best) {
                        best = th;
                        win = s;
                        m_slope = fabs(slope);
                    }
                }
                prev[s] = v;
            }
            if (win >= 0) t_hit = best;
        }
        if (win >= 0) {
            double q[3] = {ol[0] + t_hit * d[0], ol[1] + t_hit * d[1], ol[2] + t_hit * d[2]};
            double g[3];
            const int32_t gw = p->interp ? F->src[win].guard : 0;
            for (int a = 0; a < 3; ++a) {
                double qp[3] = {q[0], q[1], q[2]}, qm[3] = {q[0], q[1], q[2]};
                const double lo = gw > 0 ? 0.5 - (double)gw : 0.0;
                const double hi = gw > 0 ? (double)p->n[a] + (double)gw - 0.5 : (double)p->n[a];
                qp[a] = q[a] + 1.0 < hi ? q[a] + 1.0 : hi;
                qm[a] = q[a] - 1.0 > lo ? q[a] - 1.0 : lo;
                double h = qp[a] - qm[a];
                g[a] = h > 0.0 ? (orc_source_value(F, win, qp) - orc_source_value(F, win, qm)) / h : 0.0;
            }
            double gl = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            m_grad = gl;
            double nrm[3];
            for (int a = 0; a < 3; ++a) nrm[a] = gl > 0.0 ? -g[a] / gl : -d[a];
            double ndl = -(nrm[0] * d[0] + nrm[1] * d[1] + nrm[2] * d[2]);
            if (ndl < 0.0) ndl = -ndl;
            double spec = pow(ndl, 32.0);
            double col[4];
            orc_classify(F->luts + (size_t)win * 256 * 4, iso[win], col);
            for (int c = 0; c < 3; ++c) {
                double x = col[c] * (0.25 + 0.75 * ndl) + 0.25 * spec;
                res[c] = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
            }
            res[3] = 1.0;
        }
    }
    memcpy(rgba, res, sizeof res);
    for (int c = 0; c < 4; ++c) rgba8[c] = orc_quant8(res[c]);
    margin[0] = m_in;
    margin[1] = m_out;
    margin[2] = m_iso;
    margin[3] = m_slope;
    margin[4] = m_grad;
    margin[5] = t_hit;
}

int orc_render_iso(const orc_params *p, const orc_source *src, const orc_chain *ch,
                   const float *luts, const double *iso, int32_t n_src, double *rgba,
                   uint8_t *rgba8, double *margin, int32_t n_threads)
{
    if (!p || !src || !ch || !luts || !iso || !rgba || !rgba8 || !margin) return -1;
    if (n_src < 1 || n_src > ORC_MAX_SRC || p->width < 1 || p->height < 1 || !(p->step > 0.0))
        return -1;
    if (p->n_clip < 0 || p->n_clip > ORC_MAX_CLIP) return -1;
    for (int a = 0; a < 3; ++a)
        if (p->n[a] < 1 || p->off[a] < 0 || p->off[a] + p->n[a] > p->gn[a]) return -1;
    for (int s = 0; s < n_src; ++s)
        if (((p->active_mask >> s) & 1u) &&
            (src[s].fdim < 1 || src[s].fdim > 4 || orc_chain_check(&ch[s], src[s].fdim)))
            return -1;
    orc_frame F;
    F.p = p;
    F.src = src;
    F.ch = ch;
    F.luts = luts;
    F.w = NULL;
    F.n_src = n_src;
    double M[16];
    orc_matmul4(p->projection, p->modelview, M);
    if (orc_invert4(M, F.Minv)) return -1;
    int64_t count = (int64_t)p->width * p->height;
#ifdef _OPENMP
    if (n_threads < 1) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(n_threads)
#endif
    for (int64_t i = 0; i < count; ++i)
        orc_pixel_iso(&F, iso, i, rgba + i * 4, rgba8 + i * 4, margin + i * 6);
    (void)n_threads;
    return 0;
}

/* Render the listed pixels (row-major index y*width + x; NULL = all pixels
 * in order) of one frame.  Output slot i belongs to the i-th listed pixel.
 * Returns 0, or -1 on invalid arguments. */
int orc_render(const orc_params *p, const orc_source *src, const orc_chain *ch,
               const float *luts, const double *weights, int32_t n_src,
               const int64_t *pixels, int64_t n_pixels, const orc_outputs *out,
               int32_t n_threads)
{
    if (!p || !src || !ch || !luts || !weights || !out) return -1;
    if (n_src < 1 || n_src > ORC_MAX_SRC || p->width < 1 || p->height < 1) return -1;
    if (!(p->step > 0.0) || p->n_clip < 0 || p->n_clip > ORC_MAX_CLIP) return -1;
    for (int a = 0; a < 3; ++a)
        if (p->n[a] < 1 || p->off[a] < 0 || p->off[a] + p->n[a] > p->gn[a]) return -1;
    for (int s = 0; s < n_src; ++s) {
        if (!((p->active_mask >> s) & 1u)) continue;
        if (src[s].fdim < 1 || src[s].fdim > 4 || src[s].guard < 0) return -1;
        if (orc_chain_check(&ch[s], src[s].fdim)) return -1;
    }
    orc_frame F;
    F.p = p; F.src = src; F.ch = ch; F.luts = luts; F.w = weights; F.n_src = n_src;
    double M[16];
    orc_matmul4(p->projection, p->modelview, M);
    if (orc_invert4(M, F.Minv)) return -1;
    int64_t count = pixels ? n_pixels : (int64_t)p->width * p->height;
#ifdef _OPENMP
    if (n_threads < 1) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(n_threads)
#endif
    for (int64_t i = 0; i < count; ++i) {
        int64_t pix = pixels ? pixels[i] : i;
        orc_pixel(&F, pix, out, i);
    }
    (void)n_threads;
    return 0;
}

/* Number of threads an OpenMP region would use with n_threads < 1. */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Max-opacity grid.  Macro cell (i, j, k) of `cell`^3 cells covers the cells
 * [i*cell - 1, (i+1)*cell] per axis (a one-cell apron, what trilinear
 * samples inside the macro cell read), clipped to [-1, n]; its value is the
 * largest blended opacity clamp(sum_s w_s * LUT_s(chain_s(v_s)).alpha, 0, 1)
 * over those cells, each source read at the cell itself (clamped to the
 * border when it has no guard cells).  grid: ceil(n/cell) per axis, x fastest. */
int orc_opacity_grid(const orc_source *src, const orc_chain *ch, const float *luts,
                     const double *w, int32_t n_src, const int64_t n[3], uint32_t mask,
                     int32_t cell, double *grid, int32_t n_threads)
{
    if (!src || !ch || !luts || !w || !grid || cell < 1 || n_src < 1 || n_src > ORC_MAX_SRC)
        return -1;
    for (int s = 0; s < n_src; ++s)
        if (((mask >> s) & 1u) && (src[s].fdim < 1 || src[s].fdim > 4 || orc_chain_check(&ch[s], src[s].fdim)))
            return -1;
    int64_t G[3] = {(n[0] + cell - 1) / cell, (n[1] + cell - 1) / cell, (n[2] + cell - 1) / cell};
    int64_t total = G[0] * G[1] * G[2];
#ifdef _OPENMP
    if (n_threads < 1) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(n_threads)
#endif
    for (int64_t g = 0; g < total; ++g) {
        int64_t gi = g % G[0], gj = (g / G[0]) % G[1], gk = g / (G[0] * G[1]);
        int64_t lo[3] = {gi * cell - 1, gj * cell - 1, gk * cell - 1};
        int64_t hi[3] = {(gi + 1) * cell, (gj + 1) * cell, (gk + 1) * cell};
        for (int a = 0; a < 3; ++a) {
            if (lo[a] < -1) lo[a] = -1;
            if (hi[a] > n[a]) hi[a] = n[a];
        }
        double best = 0.0;
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                    double a = 0.0;
                    for (int s = 0; s < n_src; ++s) {
                        if (!((mask >> s) & 1u)) continue;
                        double v[4];
                        orc_fetch(&src[s], orc_axis_index(x, n[0], src[s].guard),
                                  orc_axis_index(y, n[1], src[s].guard),
                                  orc_axis_index(z, n[2], src[s].guard), v);
                        double rgba[4];
                        orc_classify(luts + (size_t)s * 256 * 4, orc_chain_apply(&ch[s], v, src[s].fdim), rgba);
                        a += w[s] * rgba[3];
                    }
                    if (!(a >= 0.0)) a = 0.0;
                    if (a > 1.0) a = 1.0;
                    if (a > best) best = a;
                }
        grid[g] = best;
    }
    (void)n_threads;
    return 0;
}

/* Value-range grid (the data of classical empty-space skipping).  For macro
 * cell g -- the same box as in orc_opacity_grid, [i*cell - 1, (i+1)*cell]
 * per axis clipped to [-1, n] -- and each component of each active source,
 * the smallest and largest value read from the box's cells, each cell read
 * as the renderer reads it (guard cells when present, else the clamped
 * border).  Any NaN among them makes that component's range [-inf, +inf].
 * out[(g * slots + slot) * 2 + {0: min, 1: max}], slot running over the
 * active sources' components in source order; slots <= 16. */
int orc_range_grid(const orc_source *src, int32_t n_src, const int64_t n[3], uint32_t mask,
                   int32_t cell, float *out, int32_t n_threads)
{
    if (!src || !out || cell < 1 || n_src < 1 || n_src > ORC_MAX_SRC) return -1;
    int slots = 0;
    for (int s = 0; s < n_src; ++s)
        if ((mask >> s) & 1u) {
            if (src[s].fdim < 1 || src[s].fdim > 4) return -1;
            slots += src[s].fdim;
        }
    if (slots < 1 || slots > 16) return -1;
    int64_t G[3] = {(n[0] + cell - 1) / cell, (n[1] + cell - 1) / cell, (n[2] + cell - 1) / cell};
    int64_t total = G[0] * G[1] * G[2];
#ifdef _OPENMP
    if (n_threads < 1) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(n_threads)
#endif
    for (int64_t g = 0; g < total; ++g) {
        int64_t gi = g % G[0], gj = (g / G[0]) % G[1], gk = g / (G[0] * G[1]);
        int64_t lo[3] = {gi * cell - 1, gj * cell - 1, gk * cell - 1};
        int64_t hi[3] = {(gi + 1) * cell, (gj + 1) * cell, (gk + 1) * cell};
        for (int a = 0; a < 3; ++a) {
            if (lo[a] < -1) lo[a] = -1;
            if (hi[a] > n[a]) hi[a] = n[a];
        }
        double mn[16], mx[16];
        int nan[16];
        for (int k = 0; k < 16; ++k) {
            mn[k] = INFINITY;
            mx[k] = -INFINITY;
            nan[k] = 0;
        }
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                    int slot = 0;
                    for (int s = 0; s < n_src; ++s) {
                        if (!((mask >> s) & 1u)) continue;
                        double v[4];
                        orc_fetch(&src[s], orc_axis_index(x, n[0], src[s].guard),
                                  orc_axis_index(y, n[1], src[s].guard),
                                  orc_axis_index(z, n[2], src[s].guard), v);
                        for (int c = 0; c < src[s].fdim; ++c, ++slot) {
                            if (v[c] != v[c]) nan[slot] = 1;
                            if (v[c] < mn[slot]) mn[slot] = v[c];
                            if (v[c] > mx[slot]) mx[slot] = v[c];
                        }
                    }
                }
        for (int k = 0; k < slots; ++k) {
            out[(g * slots + k) * 2] = nan[k] ? -INFINITY : (float)mn[k];
            out[(g * slots + k) * 2 + 1] = nan[k] ? INFINITY : (float)mx[k];
        }
    }
    (void)n_threads;
    return 0;
}

/* Test hook: apply a functor chain to one value of dimension dim (Sec. 3.3).
 * Returns 0, or -1 if the chain is invalid for that dimension. */
int orc_chain_eval(const orc_chain *ch, const double *v_in, int32_t dim, double *out)
{
    if (dim < 1 || dim > 4 || orc_chain_check(ch, dim)) return -1;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < dim; ++c) v[c] = v_in[c];
    *out = orc_chain_apply(ch, v, dim);
    return 0;
}

/* Test hook: classify one scalar through a 256-entry RGBA LUT. */
void orc_classify_eval(const float *lut, double x, double *rgba)
{
    orc_classify(lut, x, rgba);
}

/* ------------------------------------------------- reduced-precision copy */

/* Round x to the nearest value of a binary floating-point format with
 * `mant` stored mantissa bits, normal exponents down to `emin`, largest finite
 * value `maxv`; ties to even (the C default rounding mode of nearbyint).
 * Beyond maxv: +-inf when `saturate` is 0, +-maxv otherwise.  Subnormals keep
 * the fixed quantum 2^(emin - mant).  Computed in double: every step is exact
 * for the formats used here (bf16, fp16, e4m3). */
static double orc_round_format(double x, int mant, int emin, double maxv, int saturate)
{
    if (x != x) return x;
    if (x == 0.0) return x;
    double ax = fabs(x);
    int e;
    frexp(ax, &e);              /* ax = f * 2^e, f in [0.5, 1) -> exponent e - 1 */
    int ex = e - 1;
    if (ex < emin) ex = emin;
    double quantum = ldexp(1.0, ex - mant);
    double r = nearbyint(ax / quantum) * quantum;
    if (r > maxv) r = saturate ? maxv : INFINITY;
    return x < 0 ? -r : r;
}

enum { ORC_BF16 = 1, ORC_F16 = 2, ORC_E4M3 = 3 };

/* Value a float32 takes after storage in the format (bfloat16: 7 stored
 * mantissa bits, 8-bit exponent; IEEE binary16: 10 bits, emin -14, max 65504;
 * E4M3 (OCP fn variant): 3 bits, emin -6, max 448, saturating). */
float orc_quantize_value(float x, int32_t fmt)
{
    switch (fmt) {
    case ORC_BF16: return (float)orc_round_format((double)x, 7, -126, 3.3895313892515355e38, 0);
    case ORC_F16: return (float)orc_round_format((double)x, 10, -14, 65504.0, 0);
    case ORC_E4M3: return (float)orc_round_format((double)x, 3, -6, 448.0, 1);
    default: return x;
    }
}

/* Reduced-precision copy of one source over the cells [-1, n]^3 (a one-cell
 * apron: guard cells when the source has them, else copies of the border
 * cell, which is what clamping reads).  out: (n+2)^3 * fdim floats, cell
 * (x,y,z) component c at ((((z+1)*(ny+2) + y+1)*(nx+2) + x+1)*fdim + c), each
 * holding the value the stored code represents.  For E4M3 every 8^3 brick of
 * that apron box (bricks counted from cell -1) and component gets
 * scale = absmax / 448 (1 if the brick is all zero), computed in float32; the
 * stored value is quantize(v / scale) * scale, both operations in float32.
 * scales_out (optional): ceil((n+2)/8)^3 * fdim floats, brick-major. */
int orc_lowp_copy(const orc_source *s, const int64_t n[3], int32_t fmt, float *out,
                  float *scales_out)
{
    if (!s || !out || s->fdim < 1 || s->fdim > 4) return -1;
    int64_t P[3] = {n[0] + 2, n[1] + 2, n[2] + 2};
    int fd = s->fdim;
    for (int64_t z = 0; z < P[2]; ++z)
        for (int64_t y = 0; y < P[1]; ++y)
            for (int64_t x = 0; x < P[0]; ++x) {
                double v[4];
                orc_fetch(s, orc_axis_index(x - 1, n[0], s->guard), orc_axis_index(y - 1, n[1], s->guard),
                          orc_axis_index(z - 1, n[2], s->guard), v);
                float *o = out + ((z * P[1] + y) * P[0] + x) * fd;
                for (int c = 0; c < fd; ++c) o[c] = (float)v[c];
            }
    if (fmt == 0) return 0;   /* float32 copy: values as stored */
    if (fmt == ORC_BF16 || fmt == ORC_F16) {
        int64_t total = P[0] * P[1] * P[2] * fd;
        for (int64_t i = 0; i < total; ++i) out[i] = orc_quantize_value(out[i], fmt);
        return 0;
    }
    if (fmt != ORC_E4M3) return -1;
    int64_t B[3] = {(P[0] + 7) / 8, (P[1] + 7) / 8, (P[2] + 7) / 8};
    for (int64_t bz = 0; bz < B[2]; ++bz)
        for (int64_t by = 0; by < B[1]; ++by)
            for (int64_t bx = 0; bx < B[0]; ++bx)
                for (int c = 0; c < fd; ++c) {
                    float amax = 0.0f;
                    for (int64_t z = bz * 8; z < bz * 8 + 8 && z < P[2]; ++z)
                        for (int64_t y = by * 8; y < by * 8 + 8 && y < P[1]; ++y)
                            for (int64_t x = bx * 8; x < bx * 8 + 8 && x < P[0]; ++x) {
                                float a = fabsf(out[((z * P[1] + y) * P[0] + x) * fd + c]);
                                if (a > amax) amax = a;
                            }
                    volatile float scale = amax > 0.0f ? amax / 448.0f : 1.0f;
                    if (scales_out) scales_out[((bz * B[1] + by) * B[0] + bx) * fd + c] = scale;
                    for (int64_t z = bz * 8; z < bz * 8 + 8 && z < P[2]; ++z)
                        for (int64_t y = by * 8; y < by * 8 + 8 && y < P[1]; ++y)
                            for (int64_t x = bx * 8; x < bx * 8 + 8 && x < P[0]; ++x) {
                                float *o = &out[((z * P[1] + y) * P[0] + x) * fd + c];
                                volatile float q = *o / scale;
                                volatile float deq = orc_quantize_value(q, ORC_E4M3) * scale;
                                *o = deq;
                            }
                }
    return 0;
}
