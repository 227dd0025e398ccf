// Device code shared by the evaluation kernels (exhaustive, broad phase, polar index, hulls):
// signed distances, crane kinematics, the spline at one checkpoint, the unit box of the
// broad phase and the per-unit reduction into a work item's sums.
#pragma once

#include <math_constants.h>

#include "cp_internal.cuh"

namespace cp {

// Square root for the exact distances: x rsqrt(x) on the special-function unit (the
// hardware reciprocal square root is within 2 ulp, so the product is within a few ulp,
// a relative error below 1e-6). At contact distances (under a metre) that is below 1e-6 m,
// far under the FP32 kinematics error of a 10 m lever arm, and it avoids the longer IEEE
// square root sequence in the hottest loop. x is clamped to 1e-30 so that 0 stays finite.
static __device__ __forceinline__ float sqrt_sfu(float x)
{
    const float y = fmaxf(x, 1e-30f);
    return y * rsqrtf(y);
}

static __device__ __forceinline__ float sdf_cylinder(float x, float y, float z, float cx, float cy,
                                              float4 e /* R, z_lo, z_hi */)
{
    const float dx = x - cx, dy = y - cy;
    const float rho = sqrt_sfu(fmaf(dx, dx, dy * dy));
    const float a = rho - e.x;
    const float b = fmaxf(e.y - z, z - e.z);
    const float ap = fmaxf(a, 0.f), bp = fmaxf(b, 0.f);
    return fminf(fmaxf(a, b), 0.f) + sqrt_sfu(fmaf(ap, ap, bp * bp));
}

static __device__ __forceinline__ float sdf_box(float x, float y, float z, float4 c, float4 h)
{
    const float qx = fabsf(x - c.x) - h.x;
    const float qy = fabsf(y - c.y) - h.y;
    const float qz = fabsf(z - c.z) - h.z;
    const float px = fmaxf(qx, 0.f), py = fmaxf(qy, 0.f), pz = fmaxf(qz, 0.f);
    return sqrt_sfu(fmaf(px, px, fmaf(py, py, pz * pz))) + fminf(fmaxf(qx, fmaxf(qy, qz)), 0.f);
}

// Gradient of the capped-cylinder SDF: radial on the side, axial on the caps, along (a, b)
// off the rim; inside, the nearer face.
static __device__ __forceinline__ float3 sdf_cylinder_grad(float x, float y, float z, float cx, float cy,
                                                    float4 e)
{
    const float dx = x - cx, dy = y - cy;
    const float rho = sqrtf(fmaf(dx, dx, dy * dy));
    const float a = rho - e.x;
    const float up = z - e.z, down = e.y - z;
    const float b = fmaxf(down, up);
    const float sz = up >= down ? 1.f : -1.f;
    const float ux = rho > 0.f ? dx / rho : 0.f, uy = rho > 0.f ? dy / rho : 0.f;
    if (a > 0.f && b > 0.f) {
        const float h = sqrtf(fmaf(a, a, b * b));
        return make_float3(a / h * ux, a / h * uy, b / h * sz);
    }
    if (a >= b) return make_float3(ux, uy, 0.f);
    return make_float3(0.f, 0.f, sz);
}

// Gradient of the box SDF: outside, along the clamped offset; inside, the face of the
// largest component.
static __device__ __forceinline__ float3 sdf_box_grad(float x, float y, float z, float4 c, float4 h)
{
    const float sx = x >= c.x ? 1.f : -1.f, sy = y >= c.y ? 1.f : -1.f, sz = z >= c.z ? 1.f : -1.f;
    const float qx = fabsf(x - c.x) - h.x, qy = fabsf(y - c.y) - h.y, qz = fabsf(z - c.z) - h.z;
    const float px = fmaxf(qx, 0.f), py = fmaxf(qy, 0.f), pz = fmaxf(qz, 0.f);
    const float out = fmaf(px, px, fmaf(py, py, pz * pz));
    if (out > 0.f) {
        const float inv = rsqrtf(out);
        return make_float3(px * inv * sx, py * inv * sy, pz * inv * sz);
    }
    if (qx >= qy && qx >= qz) return make_float3(sx, 0.f, 0.f);
    if (qy >= qz) return make_float3(0.f, sy, 0.f);
    return make_float3(0.f, 0.f, sz);
}

// Sine and cosine of an angle for the kinematics: the angle reduced to [-pi, pi] by 2 pi in
// two parts (Cody and Waite's additive reduction; 2 pi = 6.28318548202514648 - 1.7484555e-7,
// both parts exact in FP32, so the reduced angle is within a few 1e-7 rad of the true one for
// |x| < 2^14, far beyond any joint angle the search draws), then the hardware sine and cosine,
// whose absolute error on [-pi, pi] is below 2^-21.4 (3.6e-7). Over the crane's levers (at
// most about 10.5 m) that moves a sphere centre by under 1e-5 m, within the 2e-5 m to which
// the distances are checked against the FP64 oracle; the accurate library sincosf costs
// several times the instructions on this hottest path.
static __device__ __forceinline__ void sincos_reduced(float x, float *s, float *c)
{
    const float k = rintf(x * 0.159154943091895336f);
    const float r = fmaf(k, 1.7484555e-7f, fmaf(-k, 6.28318548202514648f, x));
    __sincosf(r, s, c);
}

// Sphere centres at configuration q (chain of Sec. 2 in the linear placement form), in
// polar form: every centre is (c1 h, s1 h, z) with (c1, s1) the cosine and sine of the slew
// angle and h the signed horizontal distance from the slew axis.
// kFastTrig: the reduced hardware sine and cosine above (the evaluation forms, which must all
// agree bit for bit); otherwise the accurate library sincosf (the forward-kinematics entry
// point and the smooth cost, whose softplus penalty is checked to 1e-4 relative).
template <int NSPH, bool kFastTrig = true>
static __device__ __forceinline__ void crane_fk_polar(const ModelDev &m, float4 q, float *h, float *z,
                                               float &s1, float &c1)
{
    float s2, c2, s23, c23;
    if (kFastTrig) {
        sincos_reduced(q.x, &s1, &c1);
        sincos_reduced(q.y, &s2, &c2);
        sincos_reduced(q.y + q.z, &s23, &c23);
    } else {
        sincosf(q.x, &s1, &c1);
        sincosf(q.y, &s2, &c2);
        sincosf(q.y + q.z, &s23, &c23);
    }
    // per sphere b = gamma q4 + beta, h = alpha c2 + b c23, z = base_z + (alpha s2 + (b s23 - delta)),
    // two spheres at a time in packed FP32x2 arithmetic (each lane the same IEEE operation as
    // the scalar form)
    const float2 q4 = make_float2(q.w, q.w), C2 = make_float2(c2, c2), C23 = make_float2(c23, c23);
    const float2 S2 = make_float2(s2, s2), S23 = make_float2(s23, s23), BZ = make_float2(m.base_z, m.base_z);
#pragma unroll
    for (int p = 0; p < NSPH / 2; ++p) {
        const float2 b = __ffma2_rn(m.pk_gamma[p], q4, m.pk_beta[p]);
        const float2 hh = __ffma2_rn(m.pk_alpha[p], C2, __fmul2_rn(b, C23));
        const float2 zz = __fadd2_rn(BZ, __ffma2_rn(m.pk_alpha[p], S2, __ffma2_rn(b, S23, m.pk_ndelta[p])));
        h[2 * p] = hh.x;
        h[2 * p + 1] = hh.y;
        z[2 * p] = zz.x;
        z[2 * p + 1] = zz.y;
    }
}

// The same centres in Cartesian form, x = c1 h and y = s1 h.
template <int NSPH, bool kFastTrig = true>
static __device__ __forceinline__ void crane_fk(const ModelDev &m, float4 q, float *x, float *y,
                                         float *z)
{
    float s1, c1;
    crane_fk_polar<NSPH, kFastTrig>(m, q, x, z, s1, c1);
#pragma unroll
    for (int s = 0; s < NSPH; ++s) {
        const float h = x[s];
        x[s] = __fmul_rn(c1, h);   // rounded products: the broad-phase form takes the same
        y[s] = __fmul_rn(s1, h);
    }
}

// w.x p0 + w.y p1 + w.z p2 + w.w p3 per component, innermost product first; the (x, y) and
// (z, w) components go through the packed FP32x2 FMA, each lane of which is the IEEE fmaf of
// the same operands, so the result equals four scalar chains bit for bit.
static __device__ __forceinline__ float4 combine4(float4 w, float4 p0, float4 p1, float4 p2, float4 p3)
{
    const float2 wx = make_float2(w.x, w.x), wy = make_float2(w.y, w.y);
    const float2 wz = make_float2(w.z, w.z), ww = make_float2(w.w, w.w);
    float2 a = __fmul2_rn(ww, make_float2(p3.x, p3.y));
    float2 b = __fmul2_rn(ww, make_float2(p3.z, p3.w));
    a = __ffma2_rn(wz, make_float2(p2.x, p2.y), a);
    b = __ffma2_rn(wz, make_float2(p2.z, p2.w), b);
    a = __ffma2_rn(wy, make_float2(p1.x, p1.y), a);
    b = __ffma2_rn(wy, make_float2(p1.z, p1.w), b);
    a = __ffma2_rn(wx, make_float2(p0.x, p0.y), a);
    b = __ffma2_rn(wx, make_float2(p0.z, p0.w), b);
    return make_float4(a.x, a.y, b.x, b.y);
}

static __device__ __forceinline__ float limit_excess(float v, float lo, float hi)
{
    const float a = fmaxf(0.f, v - hi), b = fmaxf(0.f, lo - v);
    return fmaf(a, a, b * b);
}

// 1 when g[s] < t[s] for some s of the 12: one chain of compares, each folding the
// running predicate in with setp's boolean OR, and one select at the end.
static __device__ __forceinline__ uint32_t any_below12(const float2 *g, const float *t)
{
    uint32_t r;
    asm("{\n\t.reg .pred p;\n\t"
        "setp.lt.f32 p, %1, %13;\n\t"
        "setp.lt.or.f32 p, %2, %14, p;\n\t"
        "setp.lt.or.f32 p, %3, %15, p;\n\t"
        "setp.lt.or.f32 p, %4, %16, p;\n\t"
        "setp.lt.or.f32 p, %5, %17, p;\n\t"
        "setp.lt.or.f32 p, %6, %18, p;\n\t"
        "setp.lt.or.f32 p, %7, %19, p;\n\t"
        "setp.lt.or.f32 p, %8, %20, p;\n\t"
        "setp.lt.or.f32 p, %9, %21, p;\n\t"
        "setp.lt.or.f32 p, %10, %22, p;\n\t"
        "setp.lt.or.f32 p, %11, %23, p;\n\t"
        "setp.lt.or.f32 p, %12, %24, p;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "f"(g[0].x), "f"(g[0].y), "f"(g[1].x), "f"(g[1].y), "f"(g[2].x), "f"(g[2].y),
          "f"(g[3].x), "f"(g[3].y), "f"(g[4].x), "f"(g[4].y), "f"(g[5].x), "f"(g[5].y),
          "f"(t[0]), "f"(t[1]), "f"(t[2]), "f"(t[3]), "f"(t[4]), "f"(t[5]),
          "f"(t[6]), "f"(t[7]), "f"(t[8]), "f"(t[9]), "f"(t[10]), "f"(t[11]));
    return r;
}

// 1 when some value of the packed filter t (NSPH values of the form dh^2 - rhs) is below zero:
// the OR of their sign bits. Such a value is never -0 (an exact cancellation rounds to +0) nor
// NaN (its terms are finite or +inf), so a set sign bit means exactly t < 0.
template <int NSPH>
static __device__ __forceinline__ uint32_t any_negative(const float2 *t)
{
    uint32_t bits = 0u;
#pragma unroll
    for (int q = 0; q < NSPH / 2; ++q) bits |= __float_as_uint(t[q].x) | __float_as_uint(t[q].y);
    return bits >> 31;
}

template <int NSPH>
static __device__ __forceinline__ uint32_t any_below(const float2 *g, const float *t)
{
    uint32_t r = 0;
#pragma unroll
    for (int q = 0; q < NSPH / 12; ++q) r |= any_below12(g + 6 * q, t + 12 * q);
#pragma unroll
    for (int s = 12 * (NSPH / 12); s < NSPH; s += 2)
        r |= (uint32_t)((g[s / 2].x < t[s]) | (g[s / 2].y < t[s + 1]));
    return r;
}

// Broad phase of one work unit (32 checkpoints of one candidate). All spheres of one
// configuration lie on the vertical plane at its slew angle, at signed horizontal distances
// h from the slew axis. The unit's centres are bounded by a box in a frame turned to the
// slew angle of lane 16: a sphere at h on the plane at angle phi has frame coordinates
// h (cos, sin)(phi - phi_16), so the box follows from each lane's smallest and largest h.
// An obstacle whose centre lies farther than its reach (the `w` of its record) from that
// box cannot pass the per-sphere filter for any lane; the reach carries 1 cm of slack over
// the filter's own bound, far above the FP32 rounding of either test.
// Minimum and maximum of a float over the full warp in one warp-wide reduction (the
// hardware's float min / max reduce, NaN ignored as by fminf / fmaxf).
static __device__ __forceinline__ float warp_min(float v)
{
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

static __device__ __forceinline__ float warp_max(float v)
{
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

struct UnitFrame {
    float c0, s0;     // frame axes
    float uc, uh;     // box centre and half extent along the slew direction
    float vc, vh;     // and across it
};

template <int NSPH>
static __device__ __forceinline__ UnitFrame unit_frame(float s1, float c1, const float *H)
{
    UnitFrame f;
    f.s0 = __shfl_sync(0xffffffffu, s1, 16);
    f.c0 = __shfl_sync(0xffffffffu, c1, 16);
    float hmin = H[0], hmax = H[0];
#pragma unroll
    for (int s = 1; s < NSPH; ++s) {
        hmin = fminf(hmin, H[s]);
        hmax = fmaxf(hmax, H[s]);
    }
    const float cd = fmaf(f.c0, c1, f.s0 * s1), sd = fmaf(f.c0, s1, -f.s0 * c1);
    const float umin = warp_min(fminf(hmin * cd, hmax * cd)), umax = warp_max(fmaxf(hmin * cd, hmax * cd));
    const float vmin = warp_min(fminf(hmin * sd, hmax * sd)), vmax = warp_max(fmaxf(hmin * sd, hmax * sd));
    f.uc = 0.5f * (umin + umax);
    f.uh = 0.5f * (umax - umin);
    f.vc = 0.5f * (vmin + vmax);
    f.vh = 0.5f * (vmax - vmin);
    return f;
}

// The unit box of unit_frame over the spheres whose centre height lies in (zlo, zhi), the
// band in which some obstacle can be penetrated at all; a lane with no such sphere adds
// its first sphere (a larger box is still a bound).
// The extent [hmin, hmax] of h over this lane's spheres whose centre height lies in
// (zlo, zhi); hmin > hmax when there is none.
template <int NSPH>
static __device__ __forceinline__ void band_extent(const float *H, const float *Z, float zlo, float zhi,
                                                   float &hmin, float &hmax)
{
    hmin = CUDART_INF_F;
    hmax = -CUDART_INF_F;
#pragma unroll
    for (int s = 0; s < NSPH; ++s) {
        const bool in = Z[s] > zlo && Z[s] < zhi;
        hmin = in ? fminf(hmin, H[s]) : hmin;
        hmax = in ? fmaxf(hmax, H[s]) : hmax;
    }
}

// The in-band extent [hmin, hmax] of h over the lane's spheres (hmin > hmax when there is
// none) and their heights packed for the filter, spheres outside the band at 1e30 so that no
// filter passes them. When every centre lies inside the band (the common case) it is one
// min / max pass over all spheres with nothing masked, which gives the same values.
template <int NSPH>
static __device__ __forceinline__ void band_pack(const float *H, const float *Z, float zlo, float zhi, float &hmin,
                                                 float &hmax, float2 *H2)
{
    float zmn = Z[0], zmx = Z[0];
#pragma unroll
    for (int s = 1; s < NSPH; ++s) {
        zmn = fminf(zmn, Z[s]);
        zmx = fmaxf(zmx, Z[s]);
    }
    if (zmn > zlo && zmx < zhi) {
        hmin = H[0];
        hmax = H[0];
#pragma unroll
        for (int s = 1; s < NSPH; ++s) {
            hmin = fminf(hmin, H[s]);
            hmax = fmaxf(hmax, H[s]);
        }
#pragma unroll
        for (int q = 0; q < NSPH / 2; ++q) H2[q] = make_float2(H[2 * q], H[2 * q + 1]);
    } else {
        band_extent<NSPH>(H, Z, zlo, zhi, hmin, hmax);
#pragma unroll
        for (int q = 0; q < NSPH / 2; ++q)
            H2[q] = make_float2(Z[2 * q] > zlo && Z[2 * q] < zhi ? H[2 * q] : 1e30f,
                                Z[2 * q + 1] > zlo && Z[2 * q + 1] < zhi ? H[2 * q + 1] : 1e30f);
    }
}

template <int NSPH>
static __device__ __forceinline__ UnitFrame unit_frame_band(float s1, float c1, const float *H, const float *Z,
                                                            float zlo, float zhi)
{
    float hmin, hmax;
    band_extent<NSPH>(H, Z, zlo, zhi, hmin, hmax);
    if (hmin > hmax) hmin = hmax = H[0];
    const float hb[2] = {hmin, hmax};
    return unit_frame<2>(s1, c1, hb);
}

// True when the obstacle record r = {cx, cy, ., reach} may come within reach (plus
// `extra`, a further dilation for longer-range terms) of the unit.
static __device__ __forceinline__ bool unit_near(const UnitFrame &f, float4 r, float extra = 0.f)
{
    const float u = fmaf(f.c0, r.x, f.s0 * r.y);
    const float v = fmaf(f.c0, r.y, -f.s0 * r.x);
    const float w = r.w + extra;
    return (fabsf(u - f.uc) <= f.uh + w) & (fabsf(v - f.vc) <= f.vh + w);
}

// Per lane: the checkpoint k = 32 chunk + lane + 1 of a candidate whose control points
// [q0 x4, xi (K), qd x4] are staged in s_ctrl, its configuration q(s_k), the squared and plain
// length of the increment q(s_k) - q(s_{k-1}) and the joint-limit excess (Eq. path opt).
// Lanes past n_s evaluate the last checkpoint and are marked invalid.
struct Checkpoint {
    float4 q;
    float jp, len, jl;
    int k;
    bool valid;
};

// The control points of candidate `cand` into this warp's s_ctrl[K + 8]. The warp syncs
// before (the previous item's reads are done) and after (every lane sees them).
static __device__ __forceinline__ void stage_controls(float4 *s_ctrl, const EvalArgs &a, int cand, int lane)
{
    __syncwarp();
    const float4 q0 = a.ends != nullptr ? __ldg(a.ends) : a.q0;
    const float4 qd = a.ends != nullptr ? __ldg(a.ends + 1) : a.qd;
    const float4 *xi = a.xi + (size_t)cand * a.K;
    for (int i = lane; i < a.K + 8; i += 32) s_ctrl[i] = i < 4 ? q0 : (i >= a.K + 4 ? qd : __ldg(xi + (i - 4)));
    __syncwarp();
}

static __device__ __forceinline__ Checkpoint checkpoint_at(const ModelDev &m, const EvalArgs &a,
                                                           const float4 *s_basis, const float4 *s_ctrl,
                                                           int chunk, int lane)
{
    Checkpoint c;
    c.k = chunk * 32 + lane + 1;
    c.valid = c.k <= a.n_s;
    const int kc = c.valid ? c.k : a.n_s;
    const int span = (int)fdiv((uint32_t)(kc - 1), a.div_S);   // moving span - 1, 0..K+2
    const int mstep = kc - span * a.S;                           // 1..S within the span
    const float4 *P = s_ctrl + span + 1;                         // P_{span+1..span+4}
    const float4 P0 = P[0], P1 = P[1], P2 = P[2], P3 = P[3];
    const float4 bw = s_basis[2 * (mstep - 1)];
    const float4 dbw = s_basis[2 * (mstep - 1) + 1];
    c.q = combine4(bw, P0, P1, P2, P3);
    const float4 dq = combine4(dbw, P0, P1, P2, P3);   // q(s_k) - q(s_{k-1})
    c.jp = fmaf(dq.x, dq.x, fmaf(dq.y, dq.y, fmaf(dq.z, dq.z, dq.w * dq.w)));
    c.len = sqrtf(c.jp);
    // limit excess per joint: only one of v - q_max and q_min - v can be positive (q_min <
    // q_max), so max(0, v - q_max)^2 + max(0, q_min - v)^2 is e^2 with e the larger of the two
    // clamped at 0, the same rounding as the two-term form; the differences and squares packed
    const float2 qa = make_float2(c.q.x, c.q.y), qb = make_float2(c.q.z, c.q.w), m1 = make_float2(-1.f, -1.f);
    const float2 hi_a = __fadd2_rn(qa, m.pk_nqmax[0]), hi_b = __fadd2_rn(qb, m.pk_nqmax[1]);   // v - q_max
    const float2 lo_a = __ffma2_rn(m1, qa, m.pk_qmin[0]), lo_b = __ffma2_rn(m1, qb, m.pk_qmin[1]);   // q_min - v
    const float2 ea = make_float2(fmaxf(fmaxf(hi_a.x, lo_a.x), 0.f), fmaxf(fmaxf(hi_a.y, lo_a.y), 0.f));
    const float2 eb = make_float2(fmaxf(fmaxf(hi_b.x, lo_b.x), 0.f), fmaxf(fmaxf(hi_b.y, lo_b.y), 0.f));
    const float2 sa = __fmul2_rn(ea, ea), sb = __fmul2_rn(eb, eb);
    c.jl = sa.x + sa.y + sb.x + sb.y;
    return c;
}

// Candidate and unit range [c0, c1) of work item `item`.
struct ItemRange {
    int cand, c0, c1;
};

static __device__ __forceinline__ ItemRange item_range(const EvalArgs &a, int item)
{
    ItemRange r;
    r.cand = (int)fdiv((uint32_t)item, a.div_P);
    r.c0 = (item - r.cand * a.P) * a.G;
    r.c1 = min(a.chunks, r.c0 + a.G);
    return r;
}

// The unit's four sums (J_p, penetration, J_l, length) in FP32 over its lanes, added to the
// item's FP64 sums, and its collision count. The four sums share one transposing butterfly:
// across lanes 16 apart each lane keeps two of the values and hands the other two to its
// partner, across lanes 8 apart one of the two, and three more steps finish the sum of that
// one value, so lane 8 j ends with the sum of value j (6 shuffles instead of 20); lane 8 j
// keeps the item's FP64 sum of value j. The ballot word of checkpoints in collision and the
// per-checkpoint penalty are written when asked for; a kernel compiled with kExtras false
// (launched only when neither is asked for) leaves out their tests.
template <bool kExtras = true>
static __device__ __forceinline__ void unit_accumulate(const EvalArgs &a, const Checkpoint &c, float dmin,
                                                       int cand, int chunk, int lane, double &acc,
                                                       uint32_t &count)
{
    const float pen = fmaxf(0.f, -dmin);
    const bool hit = c.valid && (dmin < 0.f);
    const float v0 = c.valid ? c.jp : 0.f, v1 = c.valid ? pen : 0.f;
    const float v2 = c.valid ? c.jl : 0.f, v3 = c.valid ? c.len : 0.f;
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    const float r0 = __shfl_xor_sync(0xffffffffu, hi16 ? v0 : v2, 16);
    const float r1 = __shfl_xor_sync(0xffffffffu, hi16 ? v1 : v3, 16);
    const float w0 = (hi16 ? v2 : v0) + r0, w1 = (hi16 ? v3 : v1) + r1;   // values 2 hi16, 2 hi16 + 1
    float x = (hi8 ? w1 : w0) + __shfl_xor_sync(0xffffffffu, hi8 ? w0 : w1, 8);   // value 2 hi16 + hi8
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    acc += (double)x;
    const uint32_t word = __ballot_sync(0xffffffffu, hit);
    count += (uint32_t)__popc(word);
    if (kExtras) {
        if (a.words_out != nullptr && lane == 0) a.words_out[(size_t)cand * a.chunks + chunk] = word;
        if (a.pen_out != nullptr && c.valid) a.pen_out[(size_t)cand * a.n_s + (c.k - 1)] = pen;
    }
}

static __device__ __forceinline__ void item_flush(const EvalArgs &a, int item, double acc, uint32_t count,
                                                  int lane)
{
    if ((lane & 7) == 0) a.item_sum[(size_t)item * 4 + (lane >> 3)] = acc;
    if (lane == 0) a.item_count[item] = count;
}

}  // namespace cp
