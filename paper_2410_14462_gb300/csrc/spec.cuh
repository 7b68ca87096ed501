// Device-side rasteriser rules of the uplifting path, float32.
//
// Every rounding step is explicit (__fmul_rn, __fadd_rn, __fdiv_rn,
// __fsqrt_rn, __fmaf_rn) so that nvcc cannot contract or reorder them: the
// integer outcomes (culling, tile rectangles, depth order, the 1/255 skip and
// the 1e-4 stop) are then reproducible operation for operation on any IEEE
// float32 machine that follows the same written rules.
//
// The rules (3D Gaussian Splatting rasteriser, which the paper uses for its
// Eq. 1 weights, Sec. 3.1 and Sec. 5):
//   Sigma   = M M^T,  M = R(q) diag(s)
//   t       = R_c mu + t_c;  culled unless t.z > 0.2
//   Sigma_c = R_c Sigma R_c^T
//   J       = [[fx/z, 0, -fx x'/z^2], [0, fy/z, -fy y'/z^2]] with
//             x' = clamp(x/z, +-1.3 W/(2 fx)) z,  y' likewise
//   Sigma2D = J Sigma_c J^T + 0.3 I;  culled unless det > 0
//   conic   = Sigma2D^-1 (through float64 when det < 1e-3 a c)
//   radius  = ceil(3 sqrt(mid + sqrt(max(0.1, mid^2 - det)))),  mid = (a+c)/2
//   mean2D  = (fx x/z + cx, fy y/z + cy)
//   tiles   = [floor((m-r)/16), floor((m+r)/16)+1) clamped, culled when empty
//   alpha   = min(0.99, o exp(-0.5 (a dx^2 + c dy^2) - b dx dy)), dx = mean - pixel centre
#pragma once

#include <cstdint>

namespace ludvig {

constexpr int kTile = 16;

// Exponential for x <= 0: Cody-Waite reduction x = n ln2 + r with ln2 split in
// a float head and tail, the degree-7 Taylor polynomial of e^r (Horner, fused
// multiply-adds), and scaling by 2^n through the exponent field.  Below -87
// the result is flushed to 0.  Within 1 ulp of e^x on [-87, 0].
__device__ __forceinline__ float exp_neg(float x) {
    if (x < -87.0f) return 0.0f;
    float n = rintf(__fmul_rn(x, 0x1.715476p+0f));
    float r = __fmaf_rn(-n, 0x1.62e430p-1f, x);
    r = __fmaf_rn(-n, -0x1.05c610p-29f, r);
    float p = 0x1.a01a02p-13f;
    p = __fmaf_rn(p, r, 0x1.6c16c2p-10f);
    p = __fmaf_rn(p, r, 0x1.111112p-7f);
    p = __fmaf_rn(p, r, 0x1.555556p-5f);
    p = __fmaf_rn(p, r, 0x1.555556p-3f);
    p = __fmaf_rn(p, r, 0x1.000000p-1f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    const int e = static_cast<int>(n) + 127;
    return __fmul_rn(p, __int_as_float(e << 23));
}

constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 0x1.010102p-8f;   // 1/255 rounded to float
constexpr float kTransMin = 0x1.a36e2ep-14f;  // 1e-4 rounded to float

// Sigma = M M^T with M = R(q) diag(s); q = (w,x,y,z) normalised here.
// out6 = S00, S01, S02, S11, S12, S22.
__device__ __forceinline__ void covariance3d(const float* s, const float* q, float* out6) {
    float n2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(q[0], q[0]), __fmul_rn(q[1], q[1])),
                                   __fmul_rn(q[2], q[2])),
                         __fmul_rn(q[3], q[3]));
    float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
    float w = __fmul_rn(q[0], inv), x = __fmul_rn(q[1], inv), y = __fmul_rn(q[2], inv),
          z = __fmul_rn(q[3], inv);
    float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    float r[9];
    r[0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
    r[1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
    r[2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
    r[3] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
    r[4] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
    r[5] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
    r[6] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
    r[7] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
    r[8] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = __fmul_rn(r[3 * i + j], s[j]);
    auto dot3 = [&](int i, int j) {
        return __fadd_rn(__fadd_rn(__fmul_rn(M[3 * i], M[3 * j]), __fmul_rn(M[3 * i + 1], M[3 * j + 1])),
                         __fmul_rn(M[3 * i + 2], M[3 * j + 2]));
    };
    out6[0] = dot3(0, 0);
    out6[1] = dot3(0, 1);
    out6[2] = dot3(0, 2);
    out6[3] = dot3(1, 1);
    out6[4] = dot3(1, 2);
    out6[5] = dot3(2, 2);
}

struct Cam {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
};

struct Projected {
    float mx, my, z, ca, cb, cc, radius;
    int x0, y0, x1, y1;   // tile rectangle, half-open
    bool visible;
};

__device__ __forceinline__ float clampf_rule(float v, float lo, float hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

// Projection of one Gaussian (mean m, covariance S6) into one camera.
__device__ __forceinline__ Projected project_gaussian(const float* m, const float* S6, const Cam& c,
                                                      int width, int height) {
    Projected o;
    o.visible = false;
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    const float* R = c.R;
    float tx = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[0], m[0]), __fmul_rn(R[1], m[1])),
                                   __fmul_rn(R[2], m[2])), c.t[0]);
    float ty = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[3], m[0]), __fmul_rn(R[4], m[1])),
                                   __fmul_rn(R[5], m[2])), c.t[1]);
    float tz = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[6], m[0]), __fmul_rn(R[7], m[1])),
                                   __fmul_rn(R[8], m[2])), c.t[2]);
    o.z = tz;
    if (!(tz > 0.2f)) return o;
    float S[9] = {S6[0], S6[1], S6[2], S6[1], S6[3], S6[4], S6[2], S6[4], S6[5]};
    float A[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            A[3 * i + j] = __fadd_rn(__fadd_rn(__fmul_rn(R[3 * i], S[j]), __fmul_rn(R[3 * i + 1], S[3 + j])),
                                     __fmul_rn(R[3 * i + 2], S[6 + j]));
    auto cdot = [&](int i, int j) {
        return __fadd_rn(__fadd_rn(__fmul_rn(A[3 * i], R[3 * j]), __fmul_rn(A[3 * i + 1], R[3 * j + 1])),
                         __fmul_rn(A[3 * i + 2], R[3 * j + 2]));
    };
    const float C00 = cdot(0, 0), C01 = cdot(0, 1), C02 = cdot(0, 2);
    const float C11 = cdot(1, 1), C12 = cdot(1, 2), C22 = cdot(2, 2);
    const float limx = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, (float)width), c.fx));
    const float limy = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, (float)height), c.fy));
    const float jx = __fmul_rn(clampf_rule(__fdiv_rn(tx, tz), -limx, limx), tz);
    const float jy = __fmul_rn(clampf_rule(__fdiv_rn(ty, tz), -limy, limy), tz);
    const float tz2 = __fmul_rn(tz, tz);
    const float j00 = __fdiv_rn(c.fx, tz), j11 = __fdiv_rn(c.fy, tz);
    const float j02 = __fdiv_rn(-__fmul_rn(c.fx, jx), tz2);
    const float j12 = __fdiv_rn(-__fmul_rn(c.fy, jy), tz2);
    const float u0 = __fadd_rn(__fmul_rn(j00, C00), __fmul_rn(j02, C02));
    const float u1 = __fadd_rn(__fmul_rn(j00, C01), __fmul_rn(j02, C12));
    const float u2 = __fadd_rn(__fmul_rn(j00, C02), __fmul_rn(j02, C22));
    const float v1 = __fadd_rn(__fmul_rn(j11, C11), __fmul_rn(j12, C12));
    const float v2 = __fadd_rn(__fmul_rn(j11, C12), __fmul_rn(j12, C22));
    const float a = __fadd_rn(__fadd_rn(__fmul_rn(u0, j00), __fmul_rn(u2, j02)), 0.3f);
    const float b = __fadd_rn(__fmul_rn(u1, j11), __fmul_rn(u2, j12));
    const float cc = __fadd_rn(__fadd_rn(__fmul_rn(v1, j11), __fmul_rn(v2, j12)), 0.3f);
    const float det = __fsub_rn(__fmul_rn(a, cc), __fmul_rn(b, b));
    if (!(det > 0.0f)) return o;
    if (det < __fmul_rn(1e-3f, __fmul_rn(a, cc))) {
        const double dd = __dsub_rn(__dmul_rn((double)a, (double)cc), __dmul_rn((double)b, (double)b));
        o.ca = __double2float_rn(__ddiv_rn((double)cc, dd));
        o.cb = __double2float_rn(__ddiv_rn(-(double)b, dd));
        o.cc = __double2float_rn(__ddiv_rn((double)a, dd));
    } else {
        const float id = __fdiv_rn(1.0f, det);
        o.ca = __fmul_rn(cc, id);
        o.cb = __fmul_rn(-b, id);
        o.cc = __fmul_rn(a, id);
    }
    const float mid = __fmul_rn(0.5f, __fadd_rn(a, cc));
    const float disc = __fsub_rn(__fmul_rn(mid, mid), det);
    const float lam = __fadd_rn(mid, __fsqrt_rn(disc > 0.1f ? disc : 0.1f));
    const float rad = ceilf(__fmul_rn(3.0f, __fsqrt_rn(lam)));
    o.mx = __fadd_rn(__fdiv_rn(__fmul_rn(c.fx, tx), tz), c.cx);
    o.my = __fadd_rn(__fdiv_rn(__fmul_rn(c.fy, ty), tz), c.cy);
    o.radius = rad;
    // x / 16 and x * 2^-4 round the same exact value: identical results
    const float fx0 = floorf(__fmul_rn(__fsub_rn(o.mx, rad), 0.0625f));
    const float fx1 = __fadd_rn(floorf(__fmul_rn(__fadd_rn(o.mx, rad), 0.0625f)), 1.0f);
    const float fy0 = floorf(__fmul_rn(__fsub_rn(o.my, rad), 0.0625f));
    const float fy1 = __fadd_rn(floorf(__fmul_rn(__fadd_rn(o.my, rad), 0.0625f)), 1.0f);
    o.x0 = (int)clampf_rule(fx0, 0.0f, (float)TX);
    o.x1 = (int)clampf_rule(fx1, 0.0f, (float)TX);
    o.y0 = (int)clampf_rule(fy0, 0.0f, (float)TY);
    o.y1 = (int)clampf_rule(fy1, 0.0f, (float)TY);
    o.visible = (o.x0 < o.x1) && (o.y0 < o.y1);
    return o;
}

// alpha of a projected Gaussian at pixel centre (pxf, pyf); returns 0 when the
// Gaussian is skipped at this pixel (positive exponent or alpha < 1/255).
__device__ __forceinline__ float alpha_at(float mx, float my, float ca, float cb, float cc, float op,
                                          float pxf, float pyf) {
    const float dx = __fsub_rn(mx, pxf), dy = __fsub_rn(my, pyf);
    const float pw = __fsub_rn(
        __fmul_rn(-0.5f, __fadd_rn(__fmul_rn(ca, __fmul_rn(dx, dx)), __fmul_rn(cc, __fmul_rn(dy, dy)))),
        __fmul_rn(cb, __fmul_rn(dx, dy)));
    if (pw > 0.0f) return 0.0f;
    float al = __fmul_rn(op, exp_neg(pw));
    al = al > kAlphaMax ? kAlphaMax : al;
    return al < kAlphaMin ? 0.0f : al;
}

// alpha_at without branches (same roundings, same result), for evaluating
// several Gaussians side by side.
__device__ __forceinline__ float alpha_at_nb(float mx, float my, float ca, float cb, float cc, float op,
                                             float pxf, float pyf) {
    const float dx = __fsub_rn(mx, pxf), dy = __fsub_rn(my, pyf);
    const float pw = __fsub_rn(
        __fmul_rn(-0.5f, __fadd_rn(__fmul_rn(ca, __fmul_rn(dx, dx)), __fmul_rn(cc, __fmul_rn(dy, dy)))),
        __fmul_rn(cb, __fmul_rn(dx, dy)));
    float al = __fmul_rn(op, exp_neg(pw > 0.0f ? 0.0f : pw));
    al = al > kAlphaMax ? kAlphaMax : al;
    al = al < kAlphaMin ? 0.0f : al;
    return pw > 0.0f ? 0.0f : al;
}

// Conservative test: can a projected Gaussian reach alpha >= 1/255 at some
// pixel centre of the rectangle [xa, xb] x [ya, yb]?  It can only if
//   Q_min = min over the rectangle of  a dx^2 + 2 b dx dy + c dy^2  <=  2 ln(255 o)
// (d = mean - pixel centre); Q_min of a positive-definite form over a
// rectangle is 0 when the mean lies inside, otherwise the smallest of the
// four edge minima (each a clamped 1D minimisation).  The 0.1% + 1e-3 slack
// covers the float32 rounding of the per-pixel test, so a Gaussian this
// returns false for is skipped at every pixel of the rectangle anyway.  Every
// rounding is explicit: the projection and the pair emission evaluate the
// same decisions and must agree exactly.
struct Reach {
    float thr, inv_ca, inv_cc, cb2;
    bool possible;
};

__device__ __forceinline__ Reach reach_prep(float ca, float cb, float cc, float op) {
    Reach r;
    r.possible = !(op < kAlphaMin);   // alpha <= opacity < 1/255 everywhere otherwise
    r.thr = __fadd_rn(__fmul_rn(__fmul_rn(2.0f, __logf(__fmul_rn(255.0f, op))), 1.001f), 1e-3f);
    r.inv_ca = __frcp_rn(ca);
    r.inv_cc = __frcp_rn(cc);
    r.cb2 = __fmul_rn(2.0f, cb);
    return r;
}

__device__ __forceinline__ bool reaches_rect(const Reach& R, float mx, float my, float ca, float cb, float cc,
                                             float xa, float xb, float ya, float yb) {
    if (!R.possible) return false;
    const float dx1 = __fsub_rn(mx, xb), dx0 = __fsub_rn(mx, xa);
    const float dy1 = __fsub_rn(my, yb), dy0 = __fsub_rn(my, ya);
    if (dx1 <= 0.f && dx0 >= 0.f && dy1 <= 0.f && dy0 >= 0.f) return true;
    auto q = [&](float dx, float dy) {
        return __fadd_rn(__fadd_rn(__fmul_rn(ca, __fmul_rn(dx, dx)), __fmul_rn(R.cb2, __fmul_rn(dx, dy))),
                         __fmul_rn(cc, __fmul_rn(dy, dy)));
    };
    auto cl = [](float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); };
    float best = q(dx0, cl(__fmul_rn(-__fmul_rn(cb, dx0), R.inv_cc), dy1, dy0));
    best = fminf(best, q(dx1, cl(__fmul_rn(-__fmul_rn(cb, dx1), R.inv_cc), dy1, dy0)));
    best = fminf(best, q(cl(__fmul_rn(-__fmul_rn(cb, dy0), R.inv_ca), dx1, dx0), dy0));
    best = fminf(best, q(cl(__fmul_rn(-__fmul_rn(cb, dy1), R.inv_ca), dx1, dx0), dy1));
    return best <= R.thr;
}

__device__ __forceinline__ bool reaches_rect(float mx, float my, float ca, float cb, float cc, float op,
                                             float xa, float xb, float ya, float yb) {
    return reaches_rect(reach_prep(ca, cb, cc, op), mx, my, ca, cb, cc, xa, xb, ya, yb);
}

// The compositing kernels give each warp the 8x4 pixel block w of a 16x16
// tile, at offset ((w & 1) * 8, (w >> 1) * 4).  Bit w of block_mask is set
// when the Gaussian can reach alpha >= 1/255 somewhere in block w.
__device__ __forceinline__ float block_x0(int tx, int w) { return (float)(tx * kTile + (w & 1) * 8) + 0.5f; }
__device__ __forceinline__ float block_y0(int ty, int w) { return (float)(ty * kTile + (w >> 1) * 4) + 0.5f; }

// The pixel-centre x-range of the ellipse {Q <= thr} (Q = a dx^2 + 2 b dx dy
// + c dy^2, d = mean - pixel centre) over a band of pixel-centre rows, in
// closed form: for a fixed dy the dx-range is (-b dy -+ sqrt(thr a - det dy^2))
// / a (det = a c - b^2); over an interval of dy its largest dx is the
// ellipse's global one, sqrt(thr c / det) at dy = -b dx / c, if that lies
// inside, else an end point (the upper boundary is concave in dy), and likewise
// for the smallest.  Both ranges are widened for rounding (thr itself carries
// the slack of reach_prep), so a pixel that the float32 per-pixel test of
// Eq. 1 can give alpha >= 1/255 lies inside.  The square roots and quotients
// are the hardware approximations (a few ulp, far inside the widening); every
// product and sum is rounded explicitly, so that no call site fuses them
// differently: k_project (the count) and k_emit_pairs (the emission) must take
// the same tile decisions.
__device__ __forceinline__ float sqrt_fast(float x) { return x > 0.0f ? __fmul_rn(x, rsqrtf(x)) : 0.0f; }

struct EllipseX {
    float b, det, thra, umax, wmax, ws, inv_a, epsx;
    int state;   // 0: reaches nothing, 1: ranges valid, 2: degenerate (take everything)
};

__device__ __forceinline__ EllipseX ellipse_prep(const Reach& R, float a, float b, float c) {
    EllipseX E{};
    if (!R.possible) return E;
    const float thr = R.thr;
    E.b = b;
    E.det = __fsub_rn(__fmul_rn(a, c), __fmul_rn(b, b));
    if (!(E.det > 0.0f) || !(thr > 0.0f) || !(a > 0.0f) || !(c > 0.0f)) {
        E.state = 2;
        return E;
    }
    E.state = 1;
    E.inv_a = __fdividef(1.0f, a);
    E.umax = sqrt_fast(__fdividef(__fmul_rn(thr, c), E.det));
    E.wmax = __fadd_rn(__fmul_rn(sqrt_fast(__fdividef(__fmul_rn(thr, a), E.det)), 1.0002f), 0.05f);
    E.ws = __fdividef(__fmul_rn(-b, E.umax), c);
    E.thra = __fmul_rn(thr, a);
    E.epsx = __fadd_rn(__fmul_rn(2e-3f, __fadd_rn(E.umax, 1.0f)), 0.05f);
    return E;
}

// False when the rows [ylo, yhi] miss the ellipse (state 1 only).
__device__ __forceinline__ bool ellipse_x_range(const EllipseX& E, float mx, float my, float ylo, float yhi,
                                                float& xl, float& xr) {
    const float w0 = fmaxf(__fsub_rn(my, yhi), -E.wmax), w1 = fminf(__fsub_rn(my, ylo), E.wmax);
    if (w0 > w1) return false;
    const float s0 = sqrt_fast(__fsub_rn(E.thra, __fmul_rn(E.det, __fmul_rn(w0, w0))));
    const float s1 = sqrt_fast(__fsub_rn(E.thra, __fmul_rn(E.det, __fmul_rn(w1, w1))));
    const float bw0 = __fmul_rn(-E.b, w0), bw1 = __fmul_rn(-E.b, w1);
    const float hi = (E.ws >= w0 && E.ws <= w1)
                         ? E.umax
                         : fmaxf(__fmul_rn(__fadd_rn(bw0, s0), E.inv_a), __fmul_rn(__fadd_rn(bw1, s1), E.inv_a));
    const float lo = (-E.ws >= w0 && -E.ws <= w1)
                         ? -E.umax
                         : fminf(__fmul_rn(__fsub_rn(bw0, s0), E.inv_a), __fmul_rn(__fsub_rn(bw1, s1), E.inv_a));
    xl = __fsub_rn(__fsub_rn(mx, hi), E.epsx);   // pixel-centre x = mx - dx
    xr = __fadd_rn(__fsub_rn(mx, lo), E.epsx);
    return true;
}

// Bit w of block_mask: the Gaussian can reach alpha >= 1/255 in the 8x4 block
// w of tile (tx, ty) (per 4-row band, its x-range against the two halves).
__device__ __forceinline__ uint32_t block_mask(const Reach& R, float mx, float my, float a, float b, float c,
                                               int tx, int ty) {
    const EllipseX E = ellipse_prep(R, a, b, c);
    if (E.state != 1) return E.state == 2 ? 0xffu : 0u;
    const float xt = (float)(tx * kTile) + 0.5f, yt = (float)(ty * kTile) + 0.5f;
    uint32_t m = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float ylo = yt + (float)(4 * k);
        float xl, xr;
        if (!ellipse_x_range(E, mx, my, ylo, ylo + 3.0f, xl, xr)) continue;
        if (xr >= xt && xl <= xt + 7.0f) m |= 1u << (2 * k);
        if (xr >= xt + 8.0f && xl <= xt + 15.0f) m |= 1u << (2 * k + 1);
    }
    return m;
}

// A superset of block_mask's bits at a fraction of its cost, for the
// compositing kernels' per-batch skip test (it decides no weight: a block it
// keeps in vain costs only the per-pixel alpha test that then finds nothing).
// The same closed form with the hardware's approximate reciprocal and
// reciprocal square root in place of the correctly rounded division and
// square root; their relative error (a few ulp) is covered by widening the
// x-ranges by 2e-3 (|dx| + 1) + 0.05 px and the dy-range by 2e-4 relative +
// 0.05 px, well above what the exact form's own slack needs.
__device__ __forceinline__ float sqrt_approx(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

__device__ __forceinline__ uint32_t block_mask_fast(float mx, float my, float a, float b, float c, float op, int tx,
                                                    int ty) {
    if (op < kAlphaMin) return 0u;
    const float thr = 2.0f * __logf(255.0f * op) * 1.001f + 1e-3f;
    const float det = a * c - b * b;
    if (!(det > 0.0f) || !(thr > 0.0f) || !(a > 0.0f) || !(c > 0.0f)) return 0xffu;
    const float inv_a = __fdividef(1.0f, a), inv_det = __fdividef(1.0f, det);
    const float umax = sqrt_approx(thr * c * inv_det);
    const float wmax = sqrt_approx(thr * a * inv_det) * 1.0002f + 0.05f;
    const float ws = -b * umax * __fdividef(1.0f, c);
    const float thra = thr * a;
    const float epsx = 2e-3f * (umax + 1.0f) + 0.05f;
    const float xt = (float)(tx * kTile) + 0.5f, yt = (float)(ty * kTile) + 0.5f;
    uint32_t m = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float ylo = yt + (float)(4 * k);
        const float w0 = fmaxf(my - (ylo + 3.0f), -wmax), w1 = fminf(my - ylo, wmax);
        if (w0 > w1) continue;
        const float s0 = sqrt_approx(thra - det * w0 * w0), s1 = sqrt_approx(thra - det * w1 * w1);
        const float hi = (ws >= w0 && ws <= w1) ? umax : fmaxf((-b * w0 + s0) * inv_a, (-b * w1 + s1) * inv_a);
        const float lo = (-ws >= w0 && -ws <= w1) ? -umax : fminf((-b * w0 - s0) * inv_a, (-b * w1 - s1) * inv_a);
        const float xl = mx - hi - epsx, xr = mx - lo + epsx;
        if (xr >= xt && xl <= xt + 7.0f) m |= 1u << (2 * k);
        if (xr >= xt + 8.0f && xl <= xt + 15.0f) m |= 1u << (2 * k + 1);
    }
    return m;
}

// Tiles of row ty that the Gaussian reaches (a (Gaussian, tile) pair is kept
// when it can give alpha >= 1/255 at some pixel centre of the tile; leaving
// the others out of the tile lists changes no weight): columns [c0, c1) within
// the tile rectangle's [x0, x1).
__device__ __forceinline__ void tile_row_range(const EllipseX& E, float mx, float my, int ty, int x0, int x1,
                                               int& c0, int& c1) {
    c0 = x0;
    c1 = x1;
    if (E.state == 2) return;
    float xl = 0.f, xr = -1.f;
    const float ylo = (float)(ty * kTile) + 0.5f;
    if (E.state == 0 || !ellipse_x_range(E, mx, my, ylo, ylo + 15.0f, xl, xr)) {
        c1 = c0;
        return;
    }
    // tile tx holds pixel centres x in [16 tx + 0.5, 16 tx + 15.5]
    const float f0 = fmaxf(ceilf(__fmul_rn(__fsub_rn(xl, 15.5f), 0.0625f)), (float)x0);
    const float f1 = fminf(__fadd_rn(floorf(__fmul_rn(__fsub_rn(xr, 0.5f), 0.0625f)), 1.0f), (float)x1);
    c0 = (int)f0;
    c1 = f1 > f0 ? (int)f1 : c0;
}

// One entry of a tile's depth-ordered list as the compositing kernels read it:
// the projected Gaussian (mean, conic, opacity), its index and its block mask.
struct __align__(16) PairRec {
    float mx, my, ca, cb;
    float cc, op;
    uint32_t gid, mask;
};
static_assert(sizeof(PairRec) == 32, "PairRec is 32 bytes");

}  // namespace ludvig
