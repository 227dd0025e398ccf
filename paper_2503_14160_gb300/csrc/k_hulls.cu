// Convex-hull collision checking (arXiv 2503.14160, Sec. 3.1: the crane's links as convex
// hulls against the obstacles, by the separating axis theorem), batched over configurations.
//
// Hulls: the boom, jib and telescope as oriented boxes along their axes (axes e, n, e x n
// with n the normal of the crane's vertical plane; the telescope box spans the extension
// max(q4, 0)), and the grapple as an upright box below the tip. Obstacles: axis-aligned
// boxes, and each vertical cylinder as the regular octagonal prism that circumscribes it.
// For centrally symmetric convex polytopes A and B the overlap along a unit axis L is
//     o(L) = r_A(L) + r_B(L) - |(c_B - c_A) . L|,
// they are disjoint when o(L) < 0 for a face normal of either or a cross product of their
// edge directions, and otherwise the smallest o over those axes is the penetration depth.
// Every configuration's result is the largest depth over links and obstacles (0 when
// collision-free).
//
// One thread per configuration. All threads scan the obstacles in the same order (the
// loads are warp-wide broadcasts); an obstacle whose horizontal reach stays farther from
// the crane's vertical plane than the widest hull is skipped, and so is a pair whose
// bounding spheres (the link box's and the obstacle's) do not meet. A pair's axes are
// tried with the cheap obstacle axes first and stop at the first separating one.
#include <math_constants.h>

#include "cp_internal.cuh"

namespace cp {
namespace {

constexpr float kOctCos = 0.92387953251128674f;   // cos(pi / 8): apothem / circumradius
constexpr float kSqrtHalf = 0.70710678118654752f;
constexpr int kHullThreads = 128;

struct Obb {
    float3 c;        // centre
    float3 u[3];     // unit axes
    float h[3];      // half extents
    float rb;        // bounding-sphere radius
};

__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }

__device__ __forceinline__ float3 cross3(float3 a, float3 b)
{
    return make_float3(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x));
}

__device__ __forceinline__ float obb_support(const Obb &a, float3 L)
{
    return fmaf(a.h[0], fabsf(dot3(a.u[0], L)), fmaf(a.h[1], fabsf(dot3(a.u[1], L)), a.h[2] * fabsf(dot3(a.u[2], L))));
}

// Support of the octagonal prism (circumradius rc, half height hz) along a unit axis: the
// largest |v . L| over the four vertex directions at (k + 1/2) 45 degrees, times rc, plus
// hz |L_z|.
__device__ __forceinline__ float prism_support(float rc, float hz, float3 L)
{
    // vertex directions (cos, sin) of 22.5 and 67.5 degrees; the other two are their mirrors
    const float a = 0.92387953251128674f, b = 0.38268343236508977f;
    const float v0 = fabsf(fmaf(a, L.x, b * L.y)), v1 = fabsf(fmaf(b, L.x, a * L.y));
    const float v2 = fabsf(fmaf(-b, L.x, a * L.y)), v3 = fabsf(fmaf(-a, L.x, b * L.y));
    return fmaf(rc, fmaxf(fmaxf(v0, v1), fmaxf(v2, v3)), hz * fabsf(L.z));
}

// Smallest overlap over the axes of (box a, prism at centre pc) or (box a, axis-aligned box
// with half extents bh); negative as soon as one axis separates.
__device__ __forceinline__ float sat_prism(const Obb &a, float3 pc, float rc, float hz)
{
    const float3 d = make_float3(pc.x - a.c.x, pc.y - a.c.y, pc.z - a.c.z);
    float best = CUDART_INF_F;
    // prism faces: z, then the four side normals at multiples of 45 degrees
    const float3 dirs[5] = {make_float3(0.f, 0.f, 1.f), make_float3(1.f, 0.f, 0.f),
                            make_float3(kSqrtHalf, kSqrtHalf, 0.f), make_float3(0.f, 1.f, 0.f),
                            make_float3(-kSqrtHalf, kSqrtHalf, 0.f)};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float3 L = dirs[k];
        const float o = obb_support(a, L) + prism_support(rc, hz, L) - fabsf(dot3(d, L));
        best = fminf(best, o);
    }
    if (best < 0.f) return best;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float3 L = a.u[k];
        best = fminf(best, a.h[k] + prism_support(rc, hz, L) - fabsf(dot3(d, L)));
    }
    if (best < 0.f) return best;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int e = 0; e < 5; ++e) {
            float3 L = cross3(a.u[k], dirs[e]);
            const float n2 = dot3(L, L);
            if (n2 < 1e-12f) continue;   // parallel edges: no axis
            const float inv = rsqrtf(n2);
            L = make_float3(L.x * inv, L.y * inv, L.z * inv);
            best = fminf(best, obb_support(a, L) + prism_support(rc, hz, L) - fabsf(dot3(d, L)));
        }
    }
    return best;
}

__device__ __forceinline__ float sat_box(const Obb &a, float3 bc, float3 bh)
{
    const float3 d = make_float3(bc.x - a.c.x, bc.y - a.c.y, bc.z - a.c.z);
    float best = CUDART_INF_F;
    const float3 e[3] = {make_float3(1.f, 0.f, 0.f), make_float3(0.f, 1.f, 0.f), make_float3(0.f, 0.f, 1.f)};
    const float hb[3] = {bh.x, bh.y, bh.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float3 L = e[k];
        best = fminf(best, obb_support(a, L) + hb[k] - fabsf(dot3(d, L)));
    }
    if (best < 0.f) return best;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float3 L = a.u[k];
        const float rb = fmaf(bh.x, fabsf(L.x), fmaf(bh.y, fabsf(L.y), bh.z * fabsf(L.z)));
        best = fminf(best, a.h[k] + rb - fabsf(dot3(d, L)));
    }
    if (best < 0.f) return best;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float3 L = cross3(a.u[k], e[j]);
            const float n2 = dot3(L, L);
            if (n2 < 1e-12f) continue;
            const float inv = rsqrtf(n2);
            L = make_float3(L.x * inv, L.y * inv, L.z * inv);
            const float rb = fmaf(bh.x, fabsf(L.x), fmaf(bh.y, fabsf(L.y), bh.z * fabsf(L.z)));
            best = fminf(best, obb_support(a, L) + rb - fabsf(dot3(d, L)));
        }
    }
    return best;
}

struct HullArgs {
    const float4 *q;
    int n;
    float w[3], hh[3], pad, gw, glen;
    float *pen;
};

__device__ __forceinline__ void make_box(Obb &b, float3 c, float3 e, float3 n, float hl, float w, float h)
{
    b.c = c;
    b.u[0] = e;
    b.u[1] = n;
    b.u[2] = cross3(e, n);
    b.h[0] = hl;
    b.h[1] = w;
    b.h[2] = h;
    b.rb = sqrtf(fmaf(hl, hl, fmaf(w, w, h * h)));
}

__global__ void __launch_bounds__(kHullThreads)
k_hull_penetration(const ModelDev m, const SceneDev sc, const HullArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < a.n;
    const float4 q = a.q[live ? i : 0];
    float s1, c1, s2, c2, s23, c23;
    sincosf(q.x, &s1, &c1);
    sincosf(q.y, &s2, &c2);
    sincosf(q.y + q.z, &s23, &c23);
    const float3 eb = make_float3(c2 * c1, c2 * s1, s2), ej = make_float3(c23 * c1, c23 * s1, s23);
    const float3 n = make_float3(-s1, c1, 0.f);
    const float3 O = make_float3(0.f, 0.f, m.base_z);
    const float3 J = make_float3(fmaf(m.boom_len, eb.x, O.x), fmaf(m.boom_len, eb.y, O.y), fmaf(m.boom_len, eb.z, O.z));
    const float tl = m.jib_len + q.w;
    const float3 T = make_float3(fmaf(tl, ej.x, J.x), fmaf(tl, ej.y, J.y), fmaf(tl, ej.z, J.z));
    const float q4p = fmaxf(q.w, 0.f);
    Obb box[4];
    make_box(box[0], make_float3(fmaf(0.5f * m.boom_len, eb.x, O.x), fmaf(0.5f * m.boom_len, eb.y, O.y),
                                 fmaf(0.5f * m.boom_len, eb.z, O.z)),
             eb, n, 0.5f * m.boom_len + a.pad, a.w[0], a.hh[0]);
    make_box(box[1], make_float3(fmaf(0.5f * m.jib_len, ej.x, J.x), fmaf(0.5f * m.jib_len, ej.y, J.y),
                                 fmaf(0.5f * m.jib_len, ej.z, J.z)),
             ej, n, 0.5f * m.jib_len + a.pad, a.w[1], a.hh[1]);
    const float tc = fmaf(0.5f, q4p, m.jib_len);
    make_box(box[2], make_float3(fmaf(tc, ej.x, J.x), fmaf(tc, ej.y, J.y), fmaf(tc, ej.z, J.z)), ej, n,
             fmaf(0.5f, q4p, a.pad), a.w[2], a.hh[2]);
    make_box(box[3], make_float3(T.x, T.y, T.z - 0.5f * a.glen), make_float3(c1, s1, 0.f), n, a.gw, a.gw,
             0.5f * a.glen);
    // every hull point lies within wmax of the crane's vertical plane
    const float wmax = fmaxf(fmaxf(a.w[0], a.w[1]), fmaxf(a.w[2], a.gw));
    float pen = 0.f;
    for (int o = 0; o < sc.n_cyl; ++o) {
        const float4 f = __ldg(sc.cyl_filt + o), e = __ldg(sc.cyl_exact + o);
        const float rc = e.x / kOctCos;
        const float v = fmaf(-s1, f.x, c1 * f.y);
        if (fabsf(v) > rc + wmax + 1e-3f) continue;
        const float3 pc = make_float3(f.x, f.y, 0.5f * (e.y + e.z));
        const float hz = 0.5f * (e.z - e.y);
        const float rbo = sqrtf(fmaf(rc, rc, hz * hz));
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const float3 d = make_float3(pc.x - box[l].c.x, pc.y - box[l].c.y, pc.z - box[l].c.z);
            const float rr = box[l].rb + rbo;
            if (dot3(d, d) > rr * rr) continue;   // bounding spheres apart
            pen = fmaxf(pen, sat_prism(box[l], pc, rc, hz));
        }
    }
    for (int b = 0; b < sc.n_box; ++b) {
        const float4 c = __ldg(sc.box_c + b), h = __ldg(sc.box_h + b);
        const float reach = sqrtf(fmaf(h.x, h.x, h.y * h.y));
        const float v = fmaf(-s1, c.x, c1 * c.y);
        if (fabsf(v) > reach + wmax + 1e-3f) continue;
        const float rbo = sqrtf(fmaf(h.x, h.x, fmaf(h.y, h.y, h.z * h.z)));
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const float3 d = make_float3(c.x - box[l].c.x, c.y - box[l].c.y, c.z - box[l].c.z);
            const float rr = box[l].rb + rbo;
            if (dot3(d, d) > rr * rr) continue;
            pen = fmaxf(pen, sat_box(box[l], make_float3(c.x, c.y, c.z), make_float3(h.x, h.y, h.z)));
        }
    }
    if (live) a.pen[i] = pen;
}

}  // namespace

int launch_hull_penetration(const ModelDev &m, const SceneDev &sc, const float *q, int n, const float w[3],
                            const float hh[3], float pad, float gw, float glen, float *pen, cudaStream_t st)
{
    if (n == 0) return CP_OK;
    HullArgs a{};
    a.q = (const float4 *)q;
    a.n = n;
    for (int k = 0; k < 3; ++k) {
        a.w[k] = w[k];
        a.hh[k] = hh[k];
    }
    a.pad = pad;
    a.gw = gw;
    a.glen = glen;
    a.pen = pen;
    k_hull_penetration<<<(n + kHullThreads - 1) / kHullThreads, kHullThreads, 0, st>>>(m, sc, a);
    CP_LAUNCHED("k_hull_penetration");
    return CP_OK;
}

}  // namespace cp
