/*
 * ludvig_oracle.c -- plain CPU reference of LUDVIG's uplifting and graph
 * diffusion (arXiv 2410.14462).  TEST INFRASTRUCTURE ONLY: the library's
 * compute path never calls, links or loads this file; only the tests, the
 * smoke check and the benchmark's CPU-baseline leg do.
 *
 * What it computes, in the paper's notation:
 *   - rendering weights w_i(d,p) = alpha_i(d,p) * prod_{j<i} (1 - alpha_j(d,p))
 *     over the depth-ordered set S_{d,p} of a pixel (Sec. 3.1, Eq. 1), with
 *     alpha_i = opacity_i times the projected (EWA) 2D Gaussian at p;
 *   - uplifted features f_i = sum_{(d,p) in S_i} w_i(d,p) F_{d,p} / beta_i with
 *     beta_i = sum w_i(d,p)  (Sec. 3.2, Eq. 3; matrix form f = D^-1 W^T F, Eq. 5);
 *   - exact k-nearest neighbours of the Gaussian centres (Sec. 3.3).
 * The graph weights and the power iteration (Eq. 7, Eq. 8) are written in
 * numpy in oracle.py.
 *
 * The paper leaves the rasteriser rules to the original 3D Gaussian Splatting
 * implementation (Sec. 5).  The rules used here: alpha = min(0.99, o*G);
 * a Gaussian is skipped at a pixel when alpha < 1/255 or the exponent is
 * positive; the walk stops *before* the Gaussian that would bring the
 * transmittance below 1e-4; EWA covariance with +0.3 px^2 dilation and the
 * 1.3 x half-FOV clamp of the Jacobian; near plane z > 0.2; 3-sigma radius
 * from the larger eigenvalue (floored at 0.1 discriminant); 16x16 tiles and
 * tile-rectangle membership; order by (depth, index).
 *
 * Precision.  Values are float64.  Decisions that turn floating point into
 * integers (culling, tile rectangles, depth order, the 1/255 skip and the
 * 1e-4 stop) are taken, in the default "hybrid" mode, on a float32 track that
 * follows a fixed operation-by-operation specification (no contraction,
 * explicit fmaf where a fused op is meant, and an exponential defined below)
 * so that a float32 GPU implementation of the same specification takes the
 * same decisions.  Mode 64 takes every decision in float64 instead (the plain
 * definition, used by the closed-form pins).
 *
 * Compile with -ffp-contract=off (see oracle/__init__.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TILE 16

/* ------------------------------------------------------------------ */
/* float32 exponential used by the decision track.                     */
/* Cody & Waite style argument reduction x = n ln2 + r (ln2 split into  */
/* a float head and tail, |r| <= ln2/2) followed by the degree-7 Taylor */
/* polynomial of e^r in Horner form, then scaling by 2^n through the    */
/* exponent field.  Defined for x <= 0; returns 0 below -87.            */
/* ------------------------------------------------------------------ */
float orc_exp32(float x)
{
    if (x < -87.0f) return 0.0f;
    const float log2e = 0x1.715476p+0f;
    const float ln2_hi = 0x1.62e430p-1f;
    const float ln2_lo = -0x1.05c610p-29f;
    float t = x * log2e;
    float n = rintf(t);
    float r = fmaf(-n, ln2_hi, x);
    r = fmaf(-n, ln2_lo, r);
    float p = 0x1.a01a02p-13f;          /* 1/7! */
    p = fmaf(p, r, 0x1.6c16c2p-10f);    /* 1/6! */
    p = fmaf(p, r, 0x1.111112p-7f);     /* 1/5! */
    p = fmaf(p, r, 0x1.555556p-5f);     /* 1/4! */
    p = fmaf(p, r, 0x1.555556p-3f);     /* 1/3! */
    p = fmaf(p, r, 0x1.000000p-1f);     /* 1/2! */
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int32_t e = (int32_t)n + 127;
    uint32_t bits = (uint32_t)e << 23;
    float s;
    memcpy(&s, &bits, 4);
    return p * s;
}

/* ------------------------------------------------------------------ */
/* Projection of one Gaussian into one view.                            */
/* ------------------------------------------------------------------ */
typedef struct {
    int visible;
    float mx, my, z, ca, cb, cc, op;   /* float32 track */
    int32_t radius, x0, y0, x1, y1;     /* tile rectangle [x0,x1) x [y0,y1) */
    double mx64, my64, z64, ca64, cb64, cc64;
    int32_t radius64, x064, y064, x164, y164;
    int visible64;
} orc_proj;

static inline float clampf_(float v, float lo, float hi) { return v < lo ? lo : (v > hi ? hi : v); }
static inline double clampd_(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* float32 track: the operation-by-operation projection specification.
 * cam: R[9] row-major world->camera, t[3], fx, fy, cx, cy. */
static void project32(const float* m, const float* s, const float* q, float op,
                      const float* cam, int width, int height, orc_proj* o)
{
    o->visible = 0;
    const float* R = cam;
    const float* tc = cam + 9;
    const float fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    const int TX = (width + ORC_TILE - 1) / ORC_TILE;
    const int TY = (height + ORC_TILE - 1) / ORC_TILE;

    /* camera-space mean */
    float tx = ((R[0] * m[0] + R[1] * m[1]) + R[2] * m[2]) + tc[0];
    float ty = ((R[3] * m[0] + R[4] * m[1]) + R[5] * m[2]) + tc[1];
    float tz = ((R[6] * m[0] + R[7] * m[1]) + R[8] * m[2]) + tc[2];
    if (!(tz > 0.2f)) return;

    /* unit quaternion (w,x,y,z) -> rotation */
    float n2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    float inv = 1.0f / sqrtf(n2);
    float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float r[9];
    r[0] = 1.0f - 2.0f * (yy + zz); r[1] = 2.0f * (xy - wz);        r[2] = 2.0f * (xz + wy);
    r[3] = 2.0f * (xy + wz);        r[4] = 1.0f - 2.0f * (xx + zz); r[5] = 2.0f * (yz - wx);
    r[6] = 2.0f * (xz - wy);        r[7] = 2.0f * (yz + wx);        r[8] = 1.0f - 2.0f * (xx + yy);
    /* M = Rq diag(s); Sigma = M M^T */
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = r[3 * i + j] * s[j];
    float S[9];
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            float v = (M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1]) + M[3 * i + 2] * M[3 * j + 2];
            S[3 * i + j] = v;
            S[3 * j + i] = v;
        }
    /* Sigma_c = R Sigma R^T  (A = R Sigma first) */
    float A[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            A[3 * i + j] = (R[3 * i] * S[j] + R[3 * i + 1] * S[3 + j]) + R[3 * i + 2] * S[6 + j];
    float C[9];
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            float v = (A[3 * i] * R[3 * j] + A[3 * i + 1] * R[3 * j + 1]) + A[3 * i + 2] * R[3 * j + 2];
            C[3 * i + j] = v;
            C[3 * j + i] = v;
        }
    /* Jacobian of the perspective map at the (clamped) mean */
    float limx = 1.3f * ((0.5f * (float)width) / fx);
    float limy = 1.3f * ((0.5f * (float)height) / fy);
    float jx = clampf_(tx / tz, -limx, limx) * tz;
    float jy = clampf_(ty / tz, -limy, limy) * tz;
    float tz2 = tz * tz;
    float j00 = fx / tz, j11 = fy / tz;
    float j02 = -(fx * jx) / tz2;
    float j12 = -(fy * jy) / tz2;
    float u0 = j00 * C[0] + j02 * C[2];
    float u1 = j00 * C[1] + j02 * C[5];
    float u2 = j00 * C[2] + j02 * C[8];
    float v1 = j11 * C[4] + j12 * C[5];
    float v2 = j11 * C[5] + j12 * C[8];
    float a = (u0 * j00 + u2 * j02) + 0.3f;
    float b = u1 * j11 + u2 * j12;
    float c = (v1 * j11 + v2 * j12) + 0.3f;
    float det = a * c - b * b;
    if (!(det > 0.0f)) return;
    float ca, cb, cc;
    if (det < 1e-3f * (a * c)) {
        double dd = (double)a * (double)c - (double)b * (double)b;
        ca = (float)((double)c / dd);
        cb = (float)(-(double)b / dd);
        cc = (float)((double)a / dd);
    } else {
        float id = 1.0f / det;
        ca = c * id;
        cb = -b * id;
        cc = a * id;
    }
    float mid = 0.5f * (a + c);
    float disc = mid * mid - det;
    float lam = mid + sqrtf(disc > 0.1f ? disc : 0.1f);
    float rad = ceilf(3.0f * sqrtf(lam));
    float mx = (fx * tx) / tz + cx;
    float my = (fy * ty) / tz + cy;
    float fx0 = floorf((mx - rad) / 16.0f), fx1 = floorf((mx + rad) / 16.0f) + 1.0f;
    float fy0 = floorf((my - rad) / 16.0f), fy1 = floorf((my + rad) / 16.0f) + 1.0f;
    int x0 = (int)clampf_(fx0, 0.0f, (float)TX), x1 = (int)clampf_(fx1, 0.0f, (float)TX);
    int y0 = (int)clampf_(fy0, 0.0f, (float)TY), y1 = (int)clampf_(fy1, 0.0f, (float)TY);
    if (x0 >= x1 || y0 >= y1) return;
    o->visible = 1;
    o->mx = mx; o->my = my; o->z = tz; o->ca = ca; o->cb = cb; o->cc = cc; o->op = op;
    o->radius = (int32_t)rad;
    o->x0 = x0; o->y0 = y0; o->x1 = x1; o->y1 = y1;
}

/* float64 track: the same definition evaluated in double precision. */
static void project64(const float* mf, const float* sf, const float* qf, const float* camf,
                      int width, int height, orc_proj* o)
{
    o->visible64 = 0;
    double R[9], tc[3], m[3], s[3], q[4];
    for (int i = 0; i < 9; ++i) R[i] = camf[i];
    for (int i = 0; i < 3; ++i) { tc[i] = camf[9 + i]; m[i] = mf[i]; s[i] = sf[i]; }
    for (int i = 0; i < 4; ++i) q[i] = qf[i];
    const double fx = camf[12], fy = camf[13], cx = camf[14], cy = camf[15];
    const int TX = (width + ORC_TILE - 1) / ORC_TILE;
    const int TY = (height + ORC_TILE - 1) / ORC_TILE;
    double t[3];
    for (int i = 0; i < 3; ++i) t[i] = R[3 * i] * m[0] + R[3 * i + 1] * m[1] + R[3 * i + 2] * m[2] + tc[i];
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    double r[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                   2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                   2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    double S[9], A[9], C[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += r[3 * i + k] * s[k] * s[k] * r[3 * j + k];
            S[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * S[3 * k + j];
            A[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += A[3 * i + k] * R[3 * j + k];
            C[3 * i + j] = acc;
        }
    o->z64 = t[2];
    double limx = 1.3 * (0.5 * width / fx), limy = 1.3 * (0.5 * height / fy);
    double jx = clampd_(t[0] / t[2], -limx, limx) * t[2];
    double jy = clampd_(t[1] / t[2], -limy, limy) * t[2];
    double J[6] = {fx / t[2], 0.0, -fx * jx / (t[2] * t[2]), 0.0, fy / t[2], -fy * jy / (t[2] * t[2])};
    double cov[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += J[3 * i + k] * C[3 * k + l] * J[3 * j + l];
            cov[2 * i + j] = acc;
        }
    double a = cov[0] + 0.3, b = cov[1], c = cov[3] + 0.3;
    double det = a * c - b * b;
    o->mx64 = fx * t[0] / t[2] + cx;
    o->my64 = fy * t[1] / t[2] + cy;
    o->ca64 = c / det;
    o->cb64 = -b / det;
    o->cc64 = a / det;
    if (!(t[2] > 0.2) || !(det > 0.0)) return;
    double mid = 0.5 * (a + c);
    double disc = mid * mid - det;
    double lam = mid + sqrt(disc > 0.1 ? disc : 0.1);
    double rad = ceil(3.0 * sqrt(lam));
    int x0 = (int)clampd_(floor((o->mx64 - rad) / 16.0), 0, TX);
    int x1 = (int)clampd_(floor((o->mx64 + rad) / 16.0) + 1, 0, TX);
    int y0 = (int)clampd_(floor((o->my64 - rad) / 16.0), 0, TY);
    int y1 = (int)clampd_(floor((o->my64 + rad) / 16.0) + 1, 0, TY);
    if (x0 >= x1 || y0 >= y1) return;
    o->visible64 = 1;
    o->radius64 = (int32_t)rad;
    o->x064 = x0; o->y064 = y0; o->x164 = x1; o->y164 = y1;
}

static void project_all(int64_t n, const float* means, const float* scales, const float* quats,
                        const float* opac, const float* cam, int width, int height,
                        orc_proj* P, int nthreads)
{
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t i = 0; i < n; ++i) {
        memset(&P[i], 0, sizeof(orc_proj));
        project32(means + 3 * i, scales + 3 * i, quats + 4 * i, opac[i], cam, width, height, &P[i]);
        project64(means + 3 * i, scales + 3 * i, quats + 4 * i, cam, width, height, &P[i]);
    }
}

/* ------------------------------------------------------------------ */
/* Per-tile candidate lists, ordered by (depth, index).                 */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_proj* P;
    int mode;
} sort_ctx;

static sort_ctx g_sort;  /* qsort has no context argument; lists are sorted one view at a time */

static int cmp_depth32(const void* pa, const void* pb)
{
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    float za = g_sort.P[a].z, zb = g_sort.P[b].z;
    if (za < zb) return -1;
    if (za > zb) return 1;
    return (a > b) - (a < b);
}

static int cmp_depth64(const void* pa, const void* pb)
{
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    double za = g_sort.P[a].z64, zb = g_sort.P[b].z64;
    if (za < zb) return -1;
    if (za > zb) return 1;
    return (a > b) - (a < b);
}

static inline int vis_of(const orc_proj* p, int mode) { return mode == 64 ? p->visible64 : p->visible; }
static inline void rect_of(const orc_proj* p, int mode, int* x0, int* y0, int* x1, int* y1)
{
    if (mode == 64) { *x0 = p->x064; *y0 = p->y064; *x1 = p->x164; *y1 = p->y164; }
    else { *x0 = p->x0; *y0 = p->y0; *x1 = p->x1; *y1 = p->y1; }
}

/* Builds offsets[ntiles+1] and list[offsets[ntiles]] (caller frees).  Only
 * the tiles with sort_tile[t] != 0 are put in depth order (all of them when
 * sort_tile is NULL); the others keep index order and must not be walked. */
static int build_lists(int64_t n, const orc_proj* P, int mode, int TX, int TY, const uint8_t* sort_tile,
                       int64_t** offsets_out, int32_t** list_out)
{
    int64_t ntiles = (int64_t)TX * TY;
    int64_t* off = (int64_t*)calloc((size_t)ntiles + 1, sizeof(int64_t));
    if (!off) return -1;
    for (int64_t i = 0; i < n; ++i) {
        if (!vis_of(&P[i], mode)) continue;
        int x0, y0, x1, y1;
        rect_of(&P[i], mode, &x0, &y0, &x1, &y1);
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = x0; tx < x1; ++tx) off[(int64_t)ty * TX + tx + 1]++;
    }
    for (int64_t t = 0; t < ntiles; ++t) off[t + 1] += off[t];
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(off[ntiles] > 0 ? off[ntiles] : 1));
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)ntiles);
    if (!list || !cur) { free(off); free(list); free(cur); return -1; }
    memcpy(cur, off, sizeof(int64_t) * (size_t)ntiles);
    for (int64_t i = 0; i < n; ++i) {
        if (!vis_of(&P[i], mode)) continue;
        int x0, y0, x1, y1;
        rect_of(&P[i], mode, &x0, &y0, &x1, &y1);
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = x0; tx < x1; ++tx) list[cur[(int64_t)ty * TX + tx]++] = (int32_t)i;
    }
    free(cur);
    g_sort.P = P;
    g_sort.mode = mode;
    for (int64_t t = 0; t < ntiles; ++t) {
        int64_t len = off[t + 1] - off[t];
        if (sort_tile && !sort_tile[t]) continue;
        if (len > 1) qsort(list + off[t], (size_t)len, sizeof(int32_t), mode == 64 ? cmp_depth64 : cmp_depth32);
    }
    *offsets_out = off;
    *list_out = list;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Compositing of one pixel (Eq. 1).                                    */
/* ------------------------------------------------------------------ */
typedef struct { int32_t g; int32_t pix; double w64; float w32; } orc_contrib;

/* Walks the ordered candidates of pixel (u,v); writes contributors (w>0 by
 * the decision track) to out[] and returns their count; *t_final receives
 * the float64 transmittance left after the last contributor. */
static int64_t composite_pixel(const orc_proj* P, const int32_t* cand, int64_t ncand, int u, int v,
                               int mode, orc_contrib* out, double* t_final)
{
    float T32 = 1.0f;
    double T64 = 1.0;
    const float pxf = (float)u + 0.5f, pyf = (float)v + 0.5f;
    const double px = u + 0.5, py = v + 0.5;
    int64_t cnt = 0;
    for (int64_t k = 0; k < ncand; ++k) {
        const orc_proj* g = &P[cand[k]];
        float al32 = 0.0f;
        if (mode != 64) {
            /* decision track (float32 specification) */
            float ddx = g->mx - pxf, ddy = g->my - pyf;
            float pw = -0.5f * ((g->ca * (ddx * ddx)) + (g->cc * (ddy * ddy))) - (g->cb * (ddx * ddy));
            if (pw > 0.0f) continue;
            al32 = g->op * orc_exp32(pw);
            if (al32 > 0.99f) al32 = 0.99f;
            if (al32 < 0x1.010102p-8f) continue;          /* 1/255 */
            float Tn = T32 * (1.0f - al32);
            if (Tn < 0x1.a36e2ep-14f) break;              /* 1e-4 */
        }
        /* float64 values */
        double dx = g->mx64 - px, dy = g->my64 - py;
        double pw64 = -0.5 * (g->ca64 * dx * dx + g->cc64 * dy * dy) - g->cb64 * dx * dy;
        double al64 = (double)g->op * exp(pw64);
        if (al64 > 0.99) al64 = 0.99;
        if (mode == 64) {
            if (pw64 > 0.0) continue;
            if (al64 < 1.0 / 255.0) continue;
            if (T64 * (1.0 - al64) < 1e-4) break;
        }
        out[cnt].g = cand[k];
        out[cnt].w64 = al64 * T64;
        out[cnt].w32 = al32 * T32;
        ++cnt;
        T64 = T64 * (1.0 - al64);
        T32 = T32 * (1.0f - al32);
    }
    *t_final = T64;
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Public entry points (called through ctypes).                        */
/* ------------------------------------------------------------------ */

/* Projection dump.  out32[n*8]: mx,my,z,ca,cb,cc,opacity,radius (float32
 * track); rect[n*4]: x0,y0,x1,y1 (zeros when culled); out64[n*8]: mx,my,z,
 * ca,cb,cc,radius,visible (float64 track); visible[n] of the float32 track. */
int orc_project(int64_t n, const float* means, const float* scales, const float* quats,
                const float* opac, const float* cam, int32_t width, int32_t height,
                float* out32, int32_t* rect, double* out64, uint8_t* visible, int32_t nthreads)
{
    if (n < 0 || width <= 0 || height <= 0) return -1;
    orc_proj* P = (orc_proj*)malloc(sizeof(orc_proj) * (size_t)(n > 0 ? n : 1));
    if (!P) return -2;
    project_all(n, means, scales, quats, opac, cam, width, height, P, nthreads > 0 ? nthreads : 1);
    for (int64_t i = 0; i < n; ++i) {
        const orc_proj* p = &P[i];
        if (out32) {
            float* o = out32 + 8 * i;
            o[0] = p->mx; o[1] = p->my; o[2] = p->z; o[3] = p->ca; o[4] = p->cb; o[5] = p->cc;
            o[6] = p->op; o[7] = (float)p->radius;
        }
        if (rect) { rect[4 * i] = p->x0; rect[4 * i + 1] = p->y0; rect[4 * i + 2] = p->x1; rect[4 * i + 3] = p->y1; }
        if (out64) {
            double* o = out64 + 8 * i;
            o[0] = p->mx64; o[1] = p->my64; o[2] = p->z64; o[3] = p->ca64; o[4] = p->cb64; o[5] = p->cc64;
            o[6] = p->radius64; o[7] = p->visible64;
        }
        if (visible) visible[i] = (uint8_t)p->visible;
    }
    free(P);
    return 0;
}

/* Ordered tile lists of one view.  ranges[2*ntiles] = [start,end) into list;
 * returns the total list length (writes list only if it fits in cap). */
int64_t orc_tile_lists(int64_t n, const float* means, const float* scales, const float* quats,
                       const float* opac, const float* cam, int32_t width, int32_t height, int32_t mode,
                       int64_t* ranges, int64_t cap, int32_t* list, int32_t nthreads)
{
    if (n < 0 || width <= 0 || height <= 0) return -1;
    const int TX = (width + ORC_TILE - 1) / ORC_TILE, TY = (height + ORC_TILE - 1) / ORC_TILE;
    orc_proj* P = (orc_proj*)malloc(sizeof(orc_proj) * (size_t)(n > 0 ? n : 1));
    if (!P) return -2;
    project_all(n, means, scales, quats, opac, cam, width, height, P, nthreads > 0 ? nthreads : 1);
    int64_t* off;
    int32_t* lst;
    if (build_lists(n, P, mode, TX, TY, NULL, &off, &lst)) { free(P); return -2; }
    int64_t ntiles = (int64_t)TX * TY, total = off[ntiles];
    for (int64_t t = 0; t < ntiles; ++t) { ranges[2 * t] = off[t]; ranges[2 * t + 1] = off[t + 1]; }
    if (list && total <= cap) memcpy(list, lst, sizeof(int32_t) * (size_t)total);
    free(off); free(lst); free(P);
    return total;
}

/* One view's contribution to the uplift (Eq. 3 numerator and beta).
 *   feats: [H*W*d] float32 channels-last, or NULL (then only den / weights)
 *   want:  [n] 0/1 mask of Gaussians whose sums are wanted, or NULL for all;
 *          tiles that no wanted Gaussian touches are skipped
 *   num[n*d], den[n]: float64, ADDED to (caller zeroes)
 *   t_final[H*W] (optional): float64 transmittance after each pixel's walk
 *   trip_*: optional sparse W triplets (pixel, gaussian, w64, w32), at most cap
 * Returns the number of (pixel, Gaussian) contributions in the view. */
int64_t orc_view_uplift(int64_t n, const float* means, const float* scales, const float* quats,
                        const float* opac, const float* cam, int32_t width, int32_t height,
                        const float* feats, int32_t d, int32_t mode, const uint8_t* want,
                        double* num, double* den, double* t_final,
                        int64_t cap, int32_t* trip_pix, int32_t* trip_gid, double* trip_w64, float* trip_w32,
                        int32_t nthreads)
{
    if (n < 0 || width <= 0 || height <= 0 || d < 0) return -1;
    if (nthreads <= 0) nthreads = 1;
    const int TX = (width + ORC_TILE - 1) / ORC_TILE, TY = (height + ORC_TILE - 1) / ORC_TILE;
    const int64_t ntiles = (int64_t)TX * TY;
    orc_proj* P = (orc_proj*)malloc(sizeof(orc_proj) * (size_t)(n > 0 ? n : 1));
    if (!P) return -2;
    project_all(n, means, scales, quats, opac, cam, width, height, P, nthreads);
    int64_t* off;
    int32_t* lst;
    /* which tiles to composite: all, or those whose list holds a wanted Gaussian */
    uint8_t* tile_on = (uint8_t*)calloc((size_t)ntiles, 1);
    if (!want) {
        memset(tile_on, 1, (size_t)ntiles);
    } else {
        for (int64_t i = 0; i < n; ++i) {
            if (!want[i] || !vis_of(&P[i], mode)) continue;
            int x0, y0, x1, y1;
            rect_of(&P[i], mode, &x0, &y0, &x1, &y1);
            for (int ty = y0; ty < y1; ++ty)
                for (int tx = x0; tx < x1; ++tx) tile_on[(int64_t)ty * TX + tx] = 1;
        }
    }
    if (build_lists(n, P, mode, TX, TY, tile_on, &off, &lst)) { free(P); free(tile_on); return -2; }
    /* composite every pixel of every selected tile; contributions kept per
     * tile in pixel (row-major) then depth order */
    orc_contrib** tc = (orc_contrib**)calloc((size_t)ntiles, sizeof(orc_contrib*));
    int64_t* tcount = (int64_t*)calloc((size_t)ntiles, sizeof(int64_t));
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t t = 0; t < ntiles; ++t) {
        if (!tile_on[t]) continue;
        const int tx = (int)(t % TX), ty = (int)(t / TX);
        const int64_t len = off[t + 1] - off[t];
        int64_t cap_t = 64 * (len > 0 ? len : 1);
        orc_contrib* buf = (orc_contrib*)malloc(sizeof(orc_contrib) * (size_t)cap_t);
        orc_contrib* pix = (orc_contrib*)malloc(sizeof(orc_contrib) * (size_t)(len > 0 ? len : 1));
        int64_t used = 0;
        if (!buf || !pix) { failed = 1; free(buf); free(pix); continue; }
        for (int v = ty * ORC_TILE; v < ty * ORC_TILE + ORC_TILE && v < height; ++v)
            for (int u = tx * ORC_TILE; u < tx * ORC_TILE + ORC_TILE && u < width; ++u) {
                double tf;
                int64_t c = composite_pixel(P, lst + off[t], len, u, v, mode, pix, &tf);
                if (t_final) t_final[(int64_t)v * width + u] = tf;
                if (used + c > cap_t) {
                    while (used + c > cap_t) cap_t *= 2;
                    orc_contrib* nb = (orc_contrib*)realloc(buf, sizeof(orc_contrib) * (size_t)cap_t);
                    if (!nb) { failed = 1; break; }
                    buf = nb;
                }
                for (int64_t k = 0; k < c; ++k) {
                    buf[used] = pix[k];
                    buf[used].pix = v * width + u;
                    ++used;
                }
            }
        free(pix);
        tc[t] = buf;
        tcount[t] = used;
    }
    int64_t total = 0;
    for (int64_t t = 0; t < ntiles; ++t) total += tcount[t];
    if (failed) total = -2;

    /* accumulate in a fixed order; threads own disjoint channel ranges */
    if (!failed && (num || den)) {
        int nchunks = nthreads;
        if (d > 0 && nchunks > d) nchunks = d;
        if (nchunks < 1) nchunks = 1;
#pragma omp parallel for schedule(static, 1) num_threads(nthreads)
        for (int ch = 0; ch < nchunks; ++ch) {
            int c0 = (int)((int64_t)d * ch / nchunks), c1 = (int)((int64_t)d * (ch + 1) / nchunks);
            for (int64_t t = 0; t < ntiles; ++t) {
                const orc_contrib* b = tc[t];
                for (int64_t k = 0; k < tcount[t]; ++k) {
                    int32_t g = b[k].g;
                    if (want && !want[g]) continue;
                    double w = b[k].w64;
                    if (ch == 0 && den) den[g] += w;
                    if (num && feats) {
                        const float* F = feats + (int64_t)b[k].pix * d;
                        double* o = num + (int64_t)g * d;
                        for (int c = c0; c < c1; ++c) o[c] += w * (double)F[c];
                    }
                }
            }
        }
    }
    if (!failed && (trip_pix || trip_gid || trip_w64 || trip_w32)) {
        int64_t k2 = 0;
        for (int64_t t = 0; t < ntiles; ++t)
            for (int64_t k = 0; k < tcount[t] && k2 < cap; ++k, ++k2) {
                if (trip_pix) trip_pix[k2] = tc[t][k].pix;
                if (trip_gid) trip_gid[k2] = tc[t][k].g;
                if (trip_w64) trip_w64[k2] = tc[t][k].w64;
                if (trip_w32) trip_w32[k2] = tc[t][k].w32;
            }
    }
    for (int64_t t = 0; t < ntiles; ++t) free(tc[t]);
    free(tc); free(tcount); free(tile_on); free(off); free(lst); free(P);
    return total;
}

/* Rendering of per-Gaussian features into one view (Sec. 3.2, Eq. 4):
 *   out[p, :] = sum over the contributors i of pixel p of w_i(p) f_i
 * with the weights of Eq. 1 (the same walk as the uplift), no normalisation
 * and no background term.
 *   f:    [n*d] float64 features of the Gaussians
 *   tiles: [ntiles] 0/1 mask of the 16x16 tiles to render, or NULL for all
 *   out:  [H*W*d] float64; the selected tiles' pixels are OVERWRITTEN (zero
 *         where a pixel has no contributor), the others are left as they are
 * Returns the number of (pixel, Gaussian) contributions in the selected tiles. */
int64_t orc_view_render(int64_t n, const float* means, const float* scales, const float* quats,
                        const float* opac, const float* cam, int32_t width, int32_t height,
                        const double* f, int32_t d, int32_t mode, const uint8_t* tiles, double* out,
                        int32_t nthreads)
{
    if (n < 0 || width <= 0 || height <= 0 || d < 0 || (d > 0 && (!f || !out))) return -1;
    if (nthreads <= 0) nthreads = 1;
    const int TX = (width + ORC_TILE - 1) / ORC_TILE, TY = (height + ORC_TILE - 1) / ORC_TILE;
    const int64_t ntiles = (int64_t)TX * TY;
    orc_proj* P = (orc_proj*)malloc(sizeof(orc_proj) * (size_t)(n > 0 ? n : 1));
    if (!P) return -2;
    project_all(n, means, scales, quats, opac, cam, width, height, P, nthreads);
    uint8_t* tile_on = (uint8_t*)malloc((size_t)ntiles);
    if (tiles) memcpy(tile_on, tiles, (size_t)ntiles);
    else memset(tile_on, 1, (size_t)ntiles);
    int64_t* off;
    int32_t* lst;
    if (build_lists(n, P, mode, TX, TY, tile_on, &off, &lst)) { free(P); free(tile_on); return -2; }
    int64_t total = 0;
    int failed = 0;
    /* every pixel belongs to one tile, so tiles write disjoint parts of out */
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(+ : total)
    for (int64_t t = 0; t < ntiles; ++t) {
        if (!tile_on[t]) continue;
        const int tx = (int)(t % TX), ty = (int)(t / TX);
        const int64_t len = off[t + 1] - off[t];
        orc_contrib* pix = (orc_contrib*)malloc(sizeof(orc_contrib) * (size_t)(len > 0 ? len : 1));
        if (!pix) { failed = 1; continue; }
        for (int v = ty * ORC_TILE; v < ty * ORC_TILE + ORC_TILE && v < height; ++v)
            for (int u = tx * ORC_TILE; u < tx * ORC_TILE + ORC_TILE && u < width; ++u) {
                double tf;
                const int64_t c = composite_pixel(P, lst + off[t], len, u, v, mode, pix, &tf);
                double* o = out + ((int64_t)v * width + u) * d;
                for (int32_t ch = 0; ch < d; ++ch) o[ch] = 0.0;
                for (int64_t k = 0; k < c; ++k) {
                    const double w = pix[k].w64;
                    const double* fi = f + (int64_t)pix[k].g * d;
                    for (int32_t ch = 0; ch < d; ++ch) o[ch] += w * fi[ch];
                }
                total += c;
            }
        free(pix);
    }
    free(tile_on); free(off); free(lst); free(P);
    return failed ? -2 : total;
}

/* Normalisation (Eq. 3 / Eq. 5): f_i = num_i / beta_i, zero where beta_i = 0. */
void orc_normalise(int64_t n, int32_t d, const double* num, const double* den, double* out)
{
    for (int64_t i = 0; i < n; ++i)
        for (int32_t c = 0; c < d; ++c)
            out[i * d + c] = den[i] > 0.0 ? num[i * d + c] / den[i] : 0.0;
}

/* ------------------------------------------------------------------ */
/* Exact k nearest neighbours of Gaussian centres (Sec. 3.3).           */
/* Squared distance on a float32 track: d2 = (dx*dx + dy*dy) + dz*dz    */
/* with dx = m_j - m_i; order (d2, index); the query itself excluded.  */
/* Missing neighbours (n-1 < k) are -1.                                 */
/* ------------------------------------------------------------------ */
int orc_knn(int64_t n, const float* means, int32_t k, int64_t m, const int64_t* qidx,
            int32_t* out_idx, float* out_d2, int32_t nthreads)
{
    if (n < 0 || k <= 0 || m < 0) return -1;
    if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t qi = 0; qi < m; ++qi) {
        int64_t i = qidx ? qidx[qi] : qi;
        int32_t* bi = out_idx + qi * k;
        float* bd = out_d2 + qi * k;
        int32_t have = 0;
        const float xi = means[3 * i], yi = means[3 * i + 1], zi = means[3 * i + 2];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            float dx = means[3 * j] - xi, dy = means[3 * j + 1] - yi, dz = means[3 * j + 2] - zi;
            float d2 = (dx * dx + dy * dy) + dz * dz;
            if (have == k && !(d2 < bd[k - 1])) continue;   /* ties keep the lower index */
            int32_t pos = have < k ? have : k - 1;
            while (pos > 0 && (bd[pos - 1] > d2)) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = d2;
            bi[pos] = (int32_t)j;
            if (have < k) ++have;
        }
        for (int32_t t = have; t < k; ++t) { bi[t] = -1; bd[t] = INFINITY; }
    }
    return 0;
}
