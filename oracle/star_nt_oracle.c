/*
 * star_nt_oracle.c -- plain, slow CPU oracle of the STAR-NT per-frame hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path and never calls it.
 *
 * Every function follows a passage of the paper (STAR-NT, arXiv 2606.16747)
 * and evaluates it in the most direct way: per pixel, per fragment, per node,
 * in float64 unless a rule below fixes another precision.  Build with
 * -O2 -ffp-contract=off so that float expressions round after every operation.
 *
 * Fixed conventions (the paper is silent on these; both implementations are
 * written independently from the same statement):
 *  - Vertex transform and depth use float32 with one IEEE round-to-nearest per
 *    operation in the order written here; coverage is exact int64 arithmetic on
 *    vertices snapped to 1/256 pixel; pixel centres are at (x+0.5, y+0.5);
 *    ties on an edge are owned by edges with dy > 0, or dy == 0 and dx < 0.
 *  - A fragment's key is (z, primitive id); fragments are composited in
 *    ascending key order.
 *  - Colours are straight RGBA8: c = c8/255, alpha = a8/255.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_SUB 256      /* sub-pixel steps per pixel */
#define ORC_GUARD 32768.0f /* |screen coordinate| limit in pixels */

/* ------------------------------------------------------------------------ */
/* Rasterisation (Sec. 3: the geometry passes rasterise the scene at the     */
/* pass's own render-target size).                                           */

typedef struct {
    int64_t X[3], Y[3]; /* snapped screen positions, 1/256 px */
    float z0, dz1, dz2; /* NDC depth at v0 and differences */
    int64_t area;       /* twice the signed area, made positive */
} orc_tri;

static int orc_tri_setup(const float *v, const float *m, int W, int H, orc_tri *t)
{
    float sx[3], sy[3], zn[3];
    for (int k = 0; k < 3; ++k) {
        const float *p = v + 4 * k;
        float c[4];
        for (int i = 0; i < 4; ++i) {
            float acc = m[4 * i + 0] * p[0];
            acc = acc + m[4 * i + 1] * p[1];
            acc = acc + m[4 * i + 2] * p[2];
            acc = acc + m[4 * i + 3] * p[3];
            c[i] = acc;
        }
        if (!(c[3] > 0.0f))
            return 0;
        float nx = c[0] / c[3];
        float ny = c[1] / c[3];
        float nz = c[2] / c[3];
        if (!(nz >= 0.0f && nz <= 1.0f))
            return 0;
        sx[k] = (nx * 0.5f + 0.5f) * (float)W;
        sy[k] = (0.5f - ny * 0.5f) * (float)H;
        if (!(fabsf(sx[k]) <= ORC_GUARD && fabsf(sy[k]) <= ORC_GUARD))
            return 0;
        zn[k] = nz + 0.0f;
    }
    int64_t X[3], Y[3];
    for (int k = 0; k < 3; ++k) {
        X[k] = (int64_t)rintf(sx[k] * (float)ORC_SUB);
        Y[k] = (int64_t)rintf(sy[k] * (float)ORC_SUB);
    }
    int64_t area = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
    if (area == 0)
        return 0;
    int o[3] = {0, 1, 2};
    if (area < 0) { /* no culling: reorder so the area is positive */
        o[1] = 2;
        o[2] = 1;
        area = -area;
    }
    for (int k = 0; k < 3; ++k) {
        t->X[k] = X[o[k]];
        t->Y[k] = Y[o[k]];
    }
    t->z0 = zn[o[0]];
    t->dz1 = zn[o[1]] - zn[o[0]];
    t->dz2 = zn[o[2]] - zn[o[0]];
    t->area = area;
    return 1;
}

static int64_t orc_edge(const orc_tri *t, int a, int b, int64_t px, int64_t py)
{
    return (t->X[b] - t->X[a]) * (py - t->Y[a]) - (t->Y[b] - t->Y[a]) * (px - t->X[a]);
}

static int orc_owner(const orc_tri *t, int a, int b)
{
    int64_t dx = t->X[b] - t->X[a], dy = t->Y[b] - t->Y[a];
    return dy > 0 || (dy == 0 && dx < 0);
}

static int orc_inside(int64_t e, int own) { return e > 0 || (e == 0 && own); }

static int64_t floor_div(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0)
        --q;
    return q;
}

/* Visit every fragment of triangles [0, n_tris) in rows [y0, y1).
 * mode 0: counts[p] += 1.  mode 1: write (z, prim) at offsets[p] + cursor[p]++. */
static int64_t orc_raster_rows(const float *verts, int32_t n_tris, const float *vp, int32_t W,
                               int32_t H, int32_t y0, int32_t y1, int mode, uint32_t *counts,
                               const int64_t *offsets, uint32_t *cursor, float *z_out,
                               int32_t *prim_out)
{
    int64_t total = 0;
    for (int32_t tri = 0; tri < n_tris; ++tri) {
        orc_tri t;
        if (!orc_tri_setup(verts + 12 * (int64_t)tri, vp, W, H, &t))
            continue;
        int64_t minx = t.X[0], maxx = t.X[0], miny = t.Y[0], maxy = t.Y[0];
        for (int k = 1; k < 3; ++k) {
            if (t.X[k] < minx) minx = t.X[k];
            if (t.X[k] > maxx) maxx = t.X[k];
            if (t.Y[k] < miny) miny = t.Y[k];
            if (t.Y[k] > maxy) maxy = t.Y[k];
        }
        /* pixel x has its centre at 256 x + 128 */
        int64_t xa = -floor_div(-(minx - 128), ORC_SUB), xb = floor_div(maxx - 128, ORC_SUB);
        int64_t ya = -floor_div(-(miny - 128), ORC_SUB), yb = floor_div(maxy - 128, ORC_SUB);
        if (xa < 0) xa = 0;
        if (xb > W - 1) xb = W - 1;
        if (ya < y0) ya = y0;
        if (yb > y1 - 1) yb = y1 - 1;
        int own01 = orc_owner(&t, 0, 1), own12 = orc_owner(&t, 1, 2), own20 = orc_owner(&t, 2, 0);
        float r = 1.0f / (float)t.area;
        for (int64_t y = ya; y <= yb; ++y) {
            for (int64_t x = xa; x <= xb; ++x) {
                int64_t px = x * ORC_SUB + ORC_SUB / 2, py = y * ORC_SUB + ORC_SUB / 2;
                int64_t e01 = orc_edge(&t, 0, 1, px, py);
                int64_t e12 = orc_edge(&t, 1, 2, px, py);
                int64_t e20 = orc_edge(&t, 2, 0, px, py);
                if (!(orc_inside(e01, own01) && orc_inside(e12, own12) && orc_inside(e20, own20)))
                    continue;
                int64_t p = y * (int64_t)W + x;
                ++total;
                if (mode == 0) {
                    counts[p] += 1;
                } else {
                    float b1 = (float)e20 * r; /* barycentric weight of v1 */
                    float b2 = (float)e01 * r; /* barycentric weight of v2 */
                    float z = (t.z0 + b1 * t.dz1) + b2 * t.dz2;
                    z = z + 0.0f;
                    int64_t q = offsets[p] + cursor[p]++;
                    z_out[q] = z;
                    prim_out[q] = tri;
                }
            }
        }
    }
    return total;
}

int64_t orc_raster_count(const float *verts, int32_t n_tris, const float *vp, int32_t W,
                         int32_t H, int32_t y0, int32_t y1, uint32_t *counts)
{
    return orc_raster_rows(verts, n_tris, vp, W, H, y0, y1, 0, counts, 0, 0, 0, 0);
}

int64_t orc_raster_fill(const float *verts, int32_t n_tris, const float *vp, int32_t W,
                        int32_t H, int32_t y0, int32_t y1, const int64_t *offsets,
                        uint32_t *cursor, float *z_out, int32_t *prim_out)
{
    return orc_raster_rows(verts, n_tris, vp, W, H, y0, y1, 1, 0, offsets, cursor, z_out,
                           prim_out);
}

/* ------------------------------------------------------------------------ */
/* Per-pixel resolve from the sorted fragment list.                          */
/*  A-buffer (Sec. 2; Eq. 1 with premultiplied C_p = alpha_p c_p) and the     */
/*  quantities of Sec. 3.3 / Eq. 4: the two nearest layers, the tail          */
/*  statistics and the exact tail colour.                                    */

typedef struct {
    float z;
    int32_t prim;
} orc_frag;

static int orc_frag_cmp(const void *a, const void *b)
{
    const orc_frag *x = (const orc_frag *)a, *y = (const orc_frag *)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return (x->prim > y->prim) - (x->prim < y->prim);
}

static double ch(uint32_t rgba, int c) { return (double)((rgba >> (8 * c)) & 255u) / 255.0; }
static uint32_t ch8(uint32_t rgba, int c) { return (rgba >> (8 * c)) & 255u; }

void orc_resolve(const int64_t *offsets, const float *z, const int32_t *prim,
                 const uint32_t *rgba8, int32_t W, int32_t y0, int32_t y1, const double *bg,
                 int32_t *id1, float *z1, int32_t *id2, uint32_t *n_out, uint32_t *a_tail,
                 uint32_t *s_tail, double *t_tail, double *abuf, double *tail_rgb,
                 double *front2, double *layer2, double *t_all)
{
    int64_t cap = 0;
    orc_frag *buf = 0;
    for (int64_t y = y0; y < y1; ++y) {
        for (int64_t x = 0; x < W; ++x) {
            int64_t p = y * (int64_t)W + x;
            int64_t n = offsets[p + 1] - offsets[p];
            if (n > cap) {
                cap = 2 * n;
                buf = (orc_frag *)realloc(buf, sizeof(orc_frag) * (size_t)cap);
            }
            for (int64_t i = 0; i < n; ++i) {
                buf[i].z = z[offsets[p] + i];
                buf[i].prim = prim[offsets[p] + i];
            }
            qsort(buf, (size_t)n, sizeof(orc_frag), orc_frag_cmp);

            if (id1) id1[p] = n >= 1 ? buf[0].prim : -1;
            if (z1) z1[p] = n >= 1 ? buf[0].z : 1.0f;
            if (id2) id2[p] = n >= 2 ? buf[1].prim : -1;
            if (n_out) n_out[p] = (uint32_t)n;

            /* tail = fragments 3..n in key order */
            uint32_t A = 0, S[3] = {0, 0, 0};
            double tt = 1.0, tail[3] = {0, 0, 0};
            for (int64_t i = 2; i < n; ++i) {
                uint32_t c = rgba8[buf[i].prim];
                uint32_t a8 = ch8(c, 3);
                double al = (double)a8 / 255.0;
                A += a8;
                for (int k = 0; k < 3; ++k) {
                    S[k] += a8 * ch8(c, k);
                    tail[k] += al * ch(c, k) * tt; /* C_tail: over within the tail */
                }
                tt *= (1.0 - al);
            }
            if (a_tail) a_tail[p] = A;
            if (s_tail) for (int k = 0; k < 3; ++k) s_tail[3 * p + k] = S[k];
            if (t_tail) t_tail[p] = tt;
            if (tail_rgb) for (int k = 0; k < 3; ++k) tail_rgb[3 * p + k] = tail[k];

            /* exact two-layer composite and its transmittance (Eq. 4) */
            double a1 = 0, a2 = 0, c1[3] = {0, 0, 0}, c2[3] = {0, 0, 0};
            if (n >= 1) {
                a1 = ch(rgba8[buf[0].prim], 3);
                for (int k = 0; k < 3; ++k) c1[k] = ch(rgba8[buf[0].prim], k);
            }
            if (n >= 2) {
                a2 = ch(rgba8[buf[1].prim], 3);
                for (int k = 0; k < 3; ++k) c2[k] = ch(rgba8[buf[1].prim], k);
            }
            if (front2) {
                for (int k = 0; k < 3; ++k)
                    front2[4 * p + k] = a1 * c1[k] + (1.0 - a1) * a2 * c2[k];
                front2[4 * p + 3] = (1.0 - a1) * (1.0 - a2);
            }
            if (layer2) {
                for (int k = 0; k < 3; ++k) layer2[4 * p + k] = a2 * c2[k];
                layer2[4 * p + 3] = a2;
            }
            /* A-buffer: front-to-back over of every fragment, then background */
            double T = 1.0, acc[3] = {0, 0, 0};
            for (int64_t i = 0; i < n; ++i) {
                uint32_t c = rgba8[buf[i].prim];
                double al = ch(c, 3);
                for (int k = 0; k < 3; ++k) acc[k] += T * al * ch(c, k);
                T *= (1.0 - al);
            }
            if (t_all) t_all[p] = T;
            if (abuf)
                for (int k = 0; k < 3; ++k) abuf[3 * p + k] = acc[k] + T * bg[k];
        }
    }
    free(buf);
}

/* Naive renderer of the Q metric (Sec. 4.4): "over" in submission order. */
void orc_unsorted_over(const int64_t *offsets, const int32_t *prim, const uint32_t *rgba8,
                       int64_t P, const double *bg, double *out)
{
    for (int64_t p = 0; p < P; ++p) {
        double T = 1.0, acc[3] = {0, 0, 0};
        for (int64_t i = offsets[p]; i < offsets[p + 1]; ++i) {
            uint32_t c = rgba8[prim[i]];
            double al = ch(c, 3);
            for (int k = 0; k < 3; ++k) acc[k] += T * al * ch(c, k);
            T *= (1.0 - al);
        }
        for (int k = 0; k < 3; ++k) out[3 * p + k] = acc[k] + T * bg[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Weighted blended OIT (McGuire and Bavoil 2013), the baseline OIT method of */
/* the evaluation (Sec. 4), with the authors' recommended depth weight:      */
/* w(d, a) = a clamp(10 / (1e-5 + (d/5)^2 + (d/200)^6), 1e-2, 3e3), d the     */
/* view depth.  C = (sum (a c) w / max(sum a w, 1e-5)) (1 - T) + T C_b with   */
/* T = prod (1 - a).  NDC depth z in [0, 1] maps back to the view depth       */
/* d = n f / (f - z (f - n)).                                                */

static double wboit_weight(double d, double a)
{
    double w = 10.0 / (1e-5 + pow(d / 5.0, 2.0) + pow(d / 200.0, 6.0));
    if (w < 1e-2) w = 1e-2;
    if (w > 3e3) w = 3e3;
    return a * w;
}

void orc_wboit(const int64_t *offsets, const float *z, const int32_t *prim, const uint32_t *rgba8,
               int64_t P, double znear, double zfar, const double *bg, double *out)
{
    for (int64_t p = 0; p < P; ++p) {
        double num[3] = {0, 0, 0}, den = 0.0, T = 1.0;
        for (int64_t i = offsets[p]; i < offsets[p + 1]; ++i) {
            uint32_t c = rgba8[prim[i]];
            double a = ch(c, 3);
            double d = znear * zfar / (zfar - (double)z[i] * (zfar - znear));
            double w = wboit_weight(d, a);
            for (int k = 0; k < 3; ++k) num[k] += a * ch(c, k) * w;
            den += a * w;
            T *= 1.0 - a;
        }
        double inv = 1.0 / (den > 1e-5 ? den : 1e-5);
        for (int k = 0; k < 3; ++k) out[3 * p + k] = num[k] * inv * (1.0 - T) + T * bg[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Bilinear upscale of a reduced-resolution pass to the framebuffer          */
/* (Sec. 3.2, last paragraph).  Half-pixel centres, clamp to edge: the       */
/* source coordinate of output pixel x is u = (x + 0.5) Wp / W - 0.5, i.e.    */
/* u * 2W = (2x + 1) Wp - W, an exact integer.                               */

static void orc_axis(int64_t x, int64_t Wp, int64_t W, int64_t *i0, int64_t *i1, int64_t *rem,
                     int64_t *den)
{
    int64_t num = (2 * x + 1) * Wp - W;
    *den = 2 * W;
    int64_t q = floor_div(num, *den);
    *rem = num - q * (*den);
    *i0 = q < 0 ? 0 : (q > Wp - 1 ? Wp - 1 : q);
    *i1 = q + 1 < 0 ? 0 : (q + 1 > Wp - 1 ? Wp - 1 : q + 1);
}

void orc_upscale(const double *src, int32_t Wp, int32_t Hp, int32_t C, int32_t W, int32_t H,
                 double *dst)
{
    for (int64_t y = 0; y < H; ++y) {
        int64_t j0, j1, ry, dy;
        orc_axis(y, Hp, H, &j0, &j1, &ry, &dy);
        double wy = (double)ry / (double)dy;
        for (int64_t x = 0; x < W; ++x) {
            int64_t i0, i1, rx, dx;
            orc_axis(x, Wp, W, &i0, &i1, &rx, &dx);
            double wx = (double)rx / (double)dx;
            for (int c = 0; c < C; ++c) {
                double v00 = src[(j0 * Wp + i0) * C + c], v10 = src[(j0 * Wp + i1) * C + c];
                double v01 = src[(j1 * Wp + i0) * C + c], v11 = src[(j1 * Wp + i1) * C + c];
                double top = (1.0 - wx) * v00 + wx * v10;
                double bot = (1.0 - wx) * v01 + wx * v11;
                dst[(y * W + x) * C + c] = (1.0 - wy) * top + wy * bot;
            }
        }
    }
}

/* Tail-present flag at full resolution: upscaled N > 2, decided exactly on
 * integers (the bilinear weights are rationals with denominator 2W * 2H). */
void orc_tail_flag(const uint32_t *n, int32_t Wp, int32_t Hp, int32_t W, int32_t H,
                   uint8_t *flag)
{
    for (int64_t y = 0; y < H; ++y) {
        int64_t j0, j1, ry, dy;
        orc_axis(y, Hp, H, &j0, &j1, &ry, &dy);
        for (int64_t x = 0; x < W; ++x) {
            int64_t i0, i1, rx, dx;
            orc_axis(x, Wp, W, &i0, &i1, &rx, &dx);
            int64_t s = (dy - ry) * ((dx - rx) * (int64_t)n[j0 * Wp + i0] + rx * (int64_t)n[j0 * Wp + i1]) +
                        ry * ((dx - rx) * (int64_t)n[j1 * Wp + i0] + rx * (int64_t)n[j1 * Wp + i1]);
            flag[y * W + x] = s > 2 * dx * dy;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Network input and the composite terms at full resolution (Sec. 3.3).      */
/* x = [N * kappa_n, t_tail, C_acc / alpha_acc] with C_acc / alpha_acc        */
/* = sum(a8 c8) / (255 sum a8), zero when the tail has no alpha.             */
/* front.rgb = C_exact,2 + T_all C_b and front.w = T_2, T_all = T_2 t_tail.    */

void orc_features(int64_t P, const int32_t *id1, const uint32_t *rgba8, const double *layer2,
                  const double *n_up, const double *a_up, const double *s_up,
                  const double *t_up, const double *bg, double kappa_n, double *x,
                  double *front)
{
    for (int64_t p = 0; p < P; ++p) {
        double a1 = 0, c1[3] = {0, 0, 0};
        if (id1[p] >= 0) {
            a1 = ch(rgba8[id1[p]], 3);
            for (int k = 0; k < 3; ++k) c1[k] = ch(rgba8[id1[p]], k);
        }
        double a2 = layer2[4 * p + 3];
        double T2 = (1.0 - a1) * (1.0 - a2);
        double Tall = T2 * t_up[p];
        for (int k = 0; k < 3; ++k)
            front[4 * p + k] = a1 * c1[k] + (1.0 - a1) * layer2[4 * p + k] + Tall * bg[k];
        front[4 * p + 3] = T2;
        x[5 * p + 0] = n_up[p] * kappa_n;
        x[5 * p + 1] = t_up[p];
        for (int k = 0; k < 3; ++k)
            x[5 * p + 2 + k] = a_up[p] > 0.0 ? s_up[3 * p + k] / (255.0 * a_up[p]) : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Tail-colour MLP, 5 -> 32 -> 16 -> 3 (Sec. 3.3), ReLU on every layer.      */
/* Parameters in order w1[32][5], b1[32], w2[16][32], b2[16], w3[3][16], b3[3]. */
/* The output is zero where the tail is empty (flag == 0).                   */

enum { OW1 = 0, OB1 = 160, OW2 = 192, OB2 = 704, OW3 = 720, OB3 = 768, ONP = 771 };

static double relu(double v) { return v > 0.0 ? v : 0.0; }

static void orc_mlp_one(const double *prm, const double *x, double *h1, double *h2, double *f)
{
    for (int o = 0; o < 32; ++o) {
        double s = prm[OB1 + o];
        for (int i = 0; i < 5; ++i) s += prm[OW1 + 5 * o + i] * x[i];
        h1[o] = relu(s);
    }
    for (int o = 0; o < 16; ++o) {
        double s = prm[OB2 + o];
        for (int i = 0; i < 32; ++i) s += prm[OW2 + 32 * o + i] * h1[i];
        h2[o] = relu(s);
    }
    for (int o = 0; o < 3; ++o) {
        double s = prm[OB3 + o];
        for (int i = 0; i < 16; ++i) s += prm[OW3 + 16 * o + i] * h2[i];
        f[o] = relu(s);
    }
}

void orc_mlp_forward(const double *prm, const double *x, const uint8_t *flag, int64_t n,
                     double *f)
{
    double h1[32], h2[16];
    for (int64_t p = 0; p < n; ++p) {
        if (flag && !flag[p]) {
            f[3 * p] = f[3 * p + 1] = f[3 * p + 2] = 0.0;
            continue;
        }
        orc_mlp_one(prm, x + 5 * p, h1, h2, f + 3 * p);
    }
}

/* Mean squared error over n samples x 3 channels and its gradient with
 * respect to the 771 parameters (backpropagation through the three layers). */
double orc_mlp_mse_grad(const double *prm, const double *x, const double *y, int64_t n,
                        double *grad)
{
    double h1[32], h2[16], f[3];
    double loss = 0.0;
    memset(grad, 0, sizeof(double) * ONP);
    if (n == 0)
        return 0.0;
    double scale = 1.0 / (3.0 * (double)n);
    for (int64_t p = 0; p < n; ++p) {
        const double *xp = x + 5 * p;
        orc_mlp_one(prm, xp, h1, h2, f);
        double g3[3], g2[16], g1[32];
        for (int o = 0; o < 3; ++o) {
            double d = f[o] - y[3 * p + o];
            loss += d * d * scale;
            g3[o] = f[o] > 0.0 ? 2.0 * d * scale : 0.0; /* through the output ReLU */
        }
        for (int o = 0; o < 3; ++o) {
            grad[OB3 + o] += g3[o];
            for (int i = 0; i < 16; ++i) grad[OW3 + 16 * o + i] += g3[o] * h2[i];
        }
        for (int i = 0; i < 16; ++i) {
            double s = 0.0;
            for (int o = 0; o < 3; ++o) s += prm[OW3 + 16 * o + i] * g3[o];
            g2[i] = h2[i] > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < 16; ++o) {
            grad[OB2 + o] += g2[o];
            for (int i = 0; i < 32; ++i) grad[OW2 + 32 * o + i] += g2[o] * h1[i];
        }
        for (int i = 0; i < 32; ++i) {
            double s = 0.0;
            for (int o = 0; o < 16; ++o) s += prm[OW2 + 32 * o + i] * g2[o];
            g1[i] = h1[i] > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < 32; ++o) {
            grad[OB1 + o] += g1[o];
            for (int i = 0; i < 5; ++i) grad[OW1 + 5 * o + i] += g1[o] * xp[i];
        }
    }
    return loss;
}

/* ------------------------------------------------------------------------ */
/* The comparison network of Sec. 3.3: the original DFAOIT predicts the     */
/* whole transparency colour C_t from the features the paper lists for it   */
/* (the exact Porter-Duff blend of the two front fragments, the average     */
/* colour and average opacity of the remaining n-2 fragments, the           */
/* accumulated premultiplied colour and the fragment count), composited as  */
/* C = C_t + C_b prod_i (1 - a_i), with a sigmoid output.  The list has     */
/* eleven scalars although the text says ten; all eleven are kept:          */
/*   x[0..2] = a1 c1 + (1 - a1) a2 c2          (two front fragments, over)  */
/*   x[3..5] = sum_{i>=3} c_i / (n - 2)         (tail colour, straight mean) */
/*   x[6]    = sum_{i>=3} a_i / (n - 2)         (tail opacity, mean)         */
/*   x[7..9] = sum_{i>=3} a_i c_i               (tail, premultiplied sum)    */
/*   x[10]   = kappa_n n                                                      */
/* (tail means 0 when n <= 2), fragments in (z, primitive id) order, and     */
/* t_all = prod_i (1 - a_i).                                                  */

void orc_dfaoit_features(const int64_t *offsets, const float *z, const int32_t *prim,
                         const uint32_t *rgba8, int64_t p0, int64_t p1, double kappa_n, double *x,
                         double *t_all)
{
    int64_t cap = 0;
    orc_frag *buf = 0;
    for (int64_t p = p0; p < p1; ++p) {
        int64_t n = offsets[p + 1] - offsets[p];
        if (n > cap) {
            cap = 2 * n;
            buf = (orc_frag *)realloc(buf, sizeof(orc_frag) * (size_t)cap);
        }
        for (int64_t i = 0; i < n; ++i) {
            buf[i].z = z[offsets[p] + i];
            buf[i].prim = prim[offsets[p] + i];
        }
        qsort(buf, (size_t)n, sizeof(orc_frag), orc_frag_cmp);
        double *xp = x + 11 * p;
        for (int k = 0; k < 11; ++k) xp[k] = 0.0;
        double a1 = 0, a2 = 0;
        if (n >= 1) a1 = ch(rgba8[buf[0].prim], 3);
        if (n >= 2) a2 = ch(rgba8[buf[1].prim], 3);
        for (int k = 0; k < 3; ++k) {
            double c1 = n >= 1 ? ch(rgba8[buf[0].prim], k) : 0.0;
            double c2 = n >= 2 ? ch(rgba8[buf[1].prim], k) : 0.0;
            xp[k] = a1 * c1 + (1.0 - a1) * a2 * c2;
        }
        double T = 1.0;
        for (int64_t i = 0; i < n; ++i) T *= 1.0 - ch(rgba8[buf[i].prim], 3);
        t_all[p] = T;
        if (n > 2) {
            double sc[3] = {0, 0, 0}, sa = 0.0, sp[3] = {0, 0, 0};
            for (int64_t i = 2; i < n; ++i) {
                uint32_t c = rgba8[buf[i].prim];
                double al = ch(c, 3);
                sa += al;
                for (int k = 0; k < 3; ++k) {
                    sc[k] += ch(c, k);
                    sp[k] += al * ch(c, k);
                }
            }
            double m = (double)(n - 2);
            for (int k = 0; k < 3; ++k) {
                xp[3 + k] = sc[k] / m;
                xp[7 + k] = sp[k];
            }
            xp[6] = sa / m;
        }
        xp[10] = kappa_n * (double)n;
    }
    free(buf);
}

/* Parameters w1[32][11], b1[32], w2[16][32], b2[16], w3[3][16], b3[3]; ReLU
 * hidden layers, sigmoid output; f = 0 where flag == 0 (no fragment). */
enum { DW1 = 0, DB1 = 352, DW2 = 384, DB2 = 896, DW3 = 912, DB3 = 960, DNP = 963 };

static double sigmoid(double v) { return 1.0 / (1.0 + exp(-v)); }

static void orc_dfaoit_one(const double *prm, const double *x, double *h1, double *h2, double *f)
{
    for (int o = 0; o < 32; ++o) {
        double s = prm[DB1 + o];
        for (int i = 0; i < 11; ++i) s += prm[DW1 + 11 * o + i] * x[i];
        h1[o] = relu(s);
    }
    for (int o = 0; o < 16; ++o) {
        double s = prm[DB2 + o];
        for (int i = 0; i < 32; ++i) s += prm[DW2 + 32 * o + i] * h1[i];
        h2[o] = relu(s);
    }
    for (int o = 0; o < 3; ++o) {
        double s = prm[DB3 + o];
        for (int i = 0; i < 16; ++i) s += prm[DW3 + 16 * o + i] * h2[i];
        f[o] = sigmoid(s);
    }
}

void orc_mlp_dfaoit_forward(const double *prm, const double *x, const uint8_t *flag, int64_t n,
                            double *f)
{
    double h1[32], h2[16];
    for (int64_t p = 0; p < n; ++p) {
        if (flag && !flag[p]) {
            f[3 * p] = f[3 * p + 1] = f[3 * p + 2] = 0.0;
            continue;
        }
        orc_dfaoit_one(prm, x + 11 * p, h1, h2, f + 3 * p);
    }
}

/* MSE over n samples x 3 channels and its gradient with respect to the 963
 * parameters; the sigmoid's derivative is f (1 - f). */
double orc_mlp_dfaoit_mse_grad(const double *prm, const double *x, const double *y, int64_t n,
                               double *grad)
{
    double h1[32], h2[16], f[3];
    double loss = 0.0;
    memset(grad, 0, sizeof(double) * DNP);
    if (n == 0)
        return 0.0;
    double scale = 1.0 / (3.0 * (double)n);
    for (int64_t p = 0; p < n; ++p) {
        const double *xp = x + 11 * p;
        orc_dfaoit_one(prm, xp, h1, h2, f);
        double g3[3], g2[16], g1[32];
        for (int o = 0; o < 3; ++o) {
            double d = f[o] - y[3 * p + o];
            loss += d * d * scale;
            g3[o] = 2.0 * d * scale * f[o] * (1.0 - f[o]);
        }
        for (int o = 0; o < 3; ++o) {
            grad[DB3 + o] += g3[o];
            for (int i = 0; i < 16; ++i) grad[DW3 + 16 * o + i] += g3[o] * h2[i];
        }
        for (int i = 0; i < 16; ++i) {
            double s = 0.0;
            for (int o = 0; o < 3; ++o) s += prm[DW3 + 16 * o + i] * g3[o];
            g2[i] = h2[i] > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < 16; ++o) {
            grad[DB2 + o] += g2[o];
            for (int i = 0; i < 32; ++i) grad[DW2 + 32 * o + i] += g2[o] * h1[i];
        }
        for (int i = 0; i < 32; ++i) {
            double s = 0.0;
            for (int o = 0; o < 16; ++o) s += prm[DW2 + 32 * o + i] * g2[o];
            g1[i] = h1[i] > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < 32; ++o) {
            grad[DB1 + o] += g1[o];
            for (int i = 0; i < 11; ++i) grad[DW1 + 11 * o + i] += g1[o] * xp[i];
        }
    }
    return loss;
}

/* Adam (Kingma and Ba) with bias correction; step counts from 1. */
void orc_adam(double *prm, const double *g, double *m, double *v, int64_t n, int64_t step,
              double lr, double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        prm[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Composite, Eq. 4: C = C_exact,2 + T_2 f(x) + T_all C_b (front carries the  */
/* first and last terms), and its 8-bit quantisation (round half to even).   */

void orc_composite(const double *front, const double *f, int64_t P, double *out)
{
    for (int64_t p = 0; p < P; ++p)
        for (int k = 0; k < 3; ++k) out[3 * p + k] = front[4 * p + k] + front[4 * p + 3] * f[3 * p + k];
}

void orc_quantize(const double *rgb, int64_t P, uint32_t *rgba8)
{
    for (int64_t p = 0; p < P; ++p) {
        uint32_t v = 255u << 24;
        for (int k = 0; k < 3; ++k) {
            double c = rgb[3 * p + k];
            c = c < 0.0 ? 0.0 : (c > 1.0 ? 1.0 : c);
            v |= (uint32_t)rint(c * 255.0) << (8 * k);
        }
        rgba8[p] = v;
    }
}

/* ------------------------------------------------------------------------ */
/* Adaptive screen-space tiles (Sec. 3.1) and tile-guided resolution         */
/* (Sec. 3.2, Eq. 2).                                                        */
/*                                                                           */
/* A base tile of B x B pixels holds a four-level quadtree (levels 0..3).     */
/* Its 21-bit mask stores one "split" bit per node of levels 0..2: bit 0 for  */
/* the root, bits 1..4 for level-1 node c1 and bits 5..20 for level-2 node    */
/* 4 c1 + c2, where a child index is 2 * (y half) + (x half).  Level-3 nodes  */
/* are leaves whenever their parent is split.                                */
/* D_i is the mean of the six pairwise Euclidean RGB distances between the    */
/* four corner pixels of the node, on the 8-bit composited frame; a node     */
/* splits when D > tau_split and merges when D < tau_merge.  The comparison   */
/* is done on the sum of the six square roots against 6 tau.                 */

static int orc_bit(int l, int i, int j)
{
    if (l == 0) return 0;
    if (l == 1) return 1 + ((j & 1) << 1 | (i & 1));
    int c1 = ((j >> 1) & 1) << 1 | ((i >> 1) & 1);
    int c2 = (j & 1) << 1 | (i & 1);
    return 5 + 4 * c1 + c2;
}

static int orc_split(uint32_t m, int l, int i, int j)
{
    return l < 3 && ((m >> orc_bit(l, i, j)) & 1u);
}

static int orc_exists(uint32_t m, int l, int i, int j)
{
    for (int k = 1; k <= l; ++k)
        if (!orc_split(m, k - 1, i >> (l - k + 1), j >> (l - k + 1)))
            return 0;
    return 1;
}

static int orc_leaf(uint32_t m, int l, int i, int j)
{
    return orc_exists(m, l, i, j) && !orc_split(m, l, i, j);
}

static double orc_dsum(const uint32_t *img, int W, int H, int64_t x0, int64_t y0, int64_t S)
{
    int64_t xs[4] = {x0, x0 + S - 1, x0, x0 + S - 1};
    int64_t ys[4] = {y0, y0, y0 + S - 1, y0 + S - 1};
    int32_t c[4][3];
    for (int k = 0; k < 4; ++k) {
        int64_t x = xs[k] < 0 ? 0 : (xs[k] > W - 1 ? W - 1 : xs[k]);
        int64_t y = ys[k] < 0 ? 0 : (ys[k] > H - 1 ? H - 1 : ys[k]);
        uint32_t v = img[y * W + x];
        for (int q = 0; q < 3; ++q) c[k][q] = (int32_t)ch8(v, q);
    }
    static const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {1, 2, 3, 2, 3, 3};
    double s = 0.0;
    for (int e = 0; e < 6; ++e) {
        int64_t q = 0;
        for (int k = 0; k < 3; ++k) {
            int64_t d = c[pa[e]][k] - c[pb[e]][k];
            q += d * d;
        }
        s += sqrt((double)q);
    }
    return s;
}

/* level of the leaf covering cell (cx, cy) of a tile (cells are B/8 wide) */
static int orc_cell_level(uint32_t m, int cx, int cy)
{
    for (int l = 0; l < 3; ++l)
        if (!orc_split(m, l, cx >> (3 - l), cy >> (3 - l)))
            return l;
    return 3;
}

double orc_pass_scale(double wbar, double delta)
{
    double s = exp2(wbar - delta);
    return s < 0.25 ? 0.25 : (s > 1.0 ? 1.0 : s);
}

int32_t orc_pass_size(double s, int32_t n) { return (int32_t)ceil(s * (double)n); }

void orc_quadtree(const uint32_t *img, const int32_t *id1, int32_t W, int32_t H, int32_t B,
                  double tau_split, double tau_merge, int32_t relax_iters,
                  const uint32_t *mask_prev, uint32_t *mask_out, uint32_t *hist)
{
    int TX = (W + B - 1) / B, TY = (H + B - 1) / B;
    int64_t NT = (int64_t)TX * TY;
    /* 1. split and merge decisions, all taken on the previous mask */
    for (int64_t t = 0; t < NT; ++t) {
        int tx = (int)(t % TX), ty = (int)(t / TX);
        uint32_t m = mask_prev[t], add = 0, del = 0;
        int splits[3][4][4];
        memset(splits, 0, sizeof(splits));
        for (int l = 0; l < 3; ++l) {
            int n = 1 << l;
            int64_t S = B >> l;
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i)
                    if (orc_leaf(m, l, i, j) &&
                        orc_dsum(img, W, H, tx * (int64_t)B + i * S, ty * (int64_t)B + j * S, S) >
                            6.0 * tau_split) {
                        splits[l][i][j] = 1;
                        add |= 1u << orc_bit(l, i, j);
                    }
        }
        for (int l = 0; l < 3; ++l) {
            int n = 1 << l;
            int64_t S = B >> l;
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    if (!(orc_exists(m, l, i, j) && orc_split(m, l, i, j)))
                        continue;
                    int ok = 1;
                    for (int c = 0; c < 4; ++c) {
                        int ci = 2 * i + (c & 1), cj = 2 * j + (c >> 1);
                        if (l + 1 < 3 && (orc_split(m, l + 1, ci, cj) || splits[l + 1][ci][cj]))
                            ok = 0;
                    }
                    if (ok && orc_dsum(img, W, H, tx * (int64_t)B + i * S, ty * (int64_t)B + j * S, S) <
                                  6.0 * tau_merge)
                        del |= 1u << orc_bit(l, i, j);
                }
        }
        mask_out[t] = (m | add) & ~del;
    }
    /* 2. relaxation: a leaf splits while an edge neighbour leaf is two or
     *    more levels deeper (Jacobi iterations over the whole grid) */
    int CX = TX * 8, CY = TY * 8;
    uint8_t *lev = (uint8_t *)malloc((size_t)CX * CY);
    for (int it = 0; it < relax_iters; ++it) {
        for (int cy = 0; cy < CY; ++cy)
            for (int cx = 0; cx < CX; ++cx)
                lev[(int64_t)cy * CX + cx] = (uint8_t)orc_cell_level(mask_out[(cy / 8) * (int64_t)TX + cx / 8], cx % 8, cy % 8);
        for (int64_t t = 0; t < NT; ++t) {
            int tx = (int)(t % TX), ty = (int)(t / TX);
            uint32_t m = mask_out[t], add = 0;
            for (int l = 0; l < 3; ++l) {
                int n = 1 << l, span = 8 >> l;
                for (int j = 0; j < n; ++j)
                    for (int i = 0; i < n; ++i) {
                        if (!orc_leaf(m, l, i, j))
                            continue;
                        int cx0 = tx * 8 + i * span, cy0 = ty * 8 + j * span, deepest = 0;
                        for (int k = 0; k < span; ++k) {
                            int nb[4][2] = {{cx0 - 1, cy0 + k}, {cx0 + span, cy0 + k},
                                            {cx0 + k, cy0 - 1}, {cx0 + k, cy0 + span}};
                            for (int e = 0; e < 4; ++e) {
                                int qx = nb[e][0], qy = nb[e][1];
                                if (qx < 0 || qy < 0 || qx >= CX || qy >= CY)
                                    continue;
                                int lv = lev[(int64_t)qy * CX + qx];
                                if (lv > deepest) deepest = lv;
                            }
                        }
                        if (deepest >= l + 2)
                            add |= 1u << orc_bit(l, i, j);
                    }
            }
            mask_out[t] = m | add;
        }
    }
    free(lev);
    /* 3. histogram of occupied leaves per level */
    for (int l = 0; l < 4; ++l) hist[l] = 0;
    for (int64_t t = 0; t < NT; ++t) {
        int tx = (int)(t % TX), ty = (int)(t / TX);
        for (int l = 0; l < 4; ++l) {
            int n = 1 << l;
            int64_t S = B >> l;
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    if (!orc_leaf(mask_out[t], l, i, j))
                        continue;
                    int occ = 0;
                    for (int64_t y = ty * (int64_t)B + j * S; y < ty * (int64_t)B + (j + 1) * S && y < H; ++y)
                        for (int64_t x = tx * (int64_t)B + i * S; x < tx * (int64_t)B + (i + 1) * S && x < W; ++x)
                            if (id1[y * W + x] >= 0) occ = 1;
                    hist[l] += (uint32_t)occ;
                }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Depth-based reprojection of an interpolated frame (Sec. 3.3, last          */
/* paragraph): each pixel takes the first-fragment depth of the last real     */
/* frame at the same position, is unprojected with the current camera and     */
/* projected with the previous one; the previous frame is sampled there      */
/* bilinearly (clamp to edge).  A point behind the previous camera keeps the  */
/* previous colour of its own pixel.                                         */

int orc_inverse4(const double *a, double *inv)
{
    double m[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) m[i][j] = j < 4 ? a[4 * i + j] : (j - 4 == i ? 1.0 : 0.0);
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(m[r][c]) > fabs(m[piv][c])) piv = r;
        if (m[piv][c] == 0.0)
            return 0;
        for (int j = 0; j < 8; ++j) {
            double tmp = m[c][j];
            m[c][j] = m[piv][j];
            m[piv][j] = tmp;
        }
        double d = m[c][c];
        for (int j = 0; j < 8; ++j) m[c][j] /= d;
        for (int r = 0; r < 4; ++r) {
            if (r == c) continue;
            double f = m[r][c];
            for (int j = 0; j < 8; ++j) m[r][j] -= f * m[c][j];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) inv[4 * i + j] = m[i][4 + j];
    return 1;
}

void orc_reproject(const float *prev, const float *z1, const double *vp_prev, const double *vp_cur,
                   int32_t W, int32_t H, double *out)
{
    double inv[16];
    orc_inverse4(vp_cur, inv);
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            int64_t p = y * W + x;
            double ndc[4] = {(2.0 * x + 1.0) / W - 1.0, 1.0 - (2.0 * y + 1.0) / H, (double)z1[p], 1.0};
            double world[4], clip[4];
            for (int i = 0; i < 4; ++i) {
                world[i] = 0.0;
                for (int k = 0; k < 4; ++k) world[i] += inv[4 * i + k] * ndc[k];
            }
            for (int i = 0; i < 4; ++i) {
                clip[i] = 0.0;
                for (int k = 0; k < 4; ++k) clip[i] += vp_prev[4 * i + k] * world[k];
            }
            if (!(clip[3] > 0.0)) {
                for (int k = 0; k < 4; ++k) out[4 * p + k] = prev[4 * p + k];
                continue;
            }
            double u = clip[0] / clip[3], v = clip[1] / clip[3];
            double px = (u + 1.0) * 0.5 * W - 0.5, py = (1.0 - v) * 0.5 * H - 0.5;
            double fx0 = floor(px), fy0 = floor(py);
            double fx = px - fx0, fy = py - fy0;
            int64_t xs[2], ys[2];
            for (int k = 0; k < 2; ++k) {
                double xv = fx0 + k, yv = fy0 + k;
                xs[k] = xv < 0 ? 0 : (xv > W - 1 ? W - 1 : (int64_t)xv);
                ys[k] = yv < 0 ? 0 : (yv > H - 1 ? H - 1 : (int64_t)yv);
            }
            for (int c = 0; c < 4; ++c) {
                double v00 = prev[4 * (ys[0] * W + xs[0]) + c], v10 = prev[4 * (ys[0] * W + xs[1]) + c];
                double v01 = prev[4 * (ys[1] * W + xs[0]) + c], v11 = prev[4 * (ys[1] * W + xs[1]) + c];
                out[4 * p + c] = (1.0 - fy) * ((1.0 - fx) * v00 + fx * v10) + fy * ((1.0 - fx) * v01 + fx * v11);
            }
        }
}
