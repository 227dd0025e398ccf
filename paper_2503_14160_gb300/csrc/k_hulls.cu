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
// One thread per configuration scans the obstacles (all threads in the same order, so the
// loads are warp-wide broadcasts); an obstacle whose horizontal reach stays farther from the
// crane's vertical plane than the widest hull, or beyond the arm's extent along it, is
// skipped. The pairs left go through a queue per warp and are worked 32 at a time, one per
// lane; a pair whose bounding spheres (the link box's and the obstacle's) do not meet is
// skipped, and a pair's axes are tried with the cheap obstacle axes first and stop at the
// first separating one.
#include "eval_common.cuh"
#include "item_queue.cuh"

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
    HullDims d;
    float *pen;
};

constexpr int kHullWarps = kHullThreads / 32;
constexpr int kBoxFloats = 16;   // centre, three axes, half extents, bounding radius

__device__ __forceinline__ void store_box(float *r, float3 c, float3 e, float3 n, float hl, float w, float h)
{
    const float3 u2 = cross3(e, n);
    const float v[kBoxFloats] = {c.x, c.y, c.z, e.x, e.y, e.z, n.x, n.y, n.z, u2.x, u2.y, u2.z, hl, w, h,
                                 sqrtf(fmaf(hl, hl, fmaf(w, w, h * h)))};
#pragma unroll
    for (int k = 0; k < kBoxFloats; ++k) r[k] = v[k];
}

__device__ __forceinline__ Obb load_box(const float *r)
{
    Obb b;
    b.c = make_float3(r[0], r[1], r[2]);
    b.u[0] = make_float3(r[3], r[4], r[5]);
    b.u[1] = make_float3(r[6], r[7], r[8]);
    b.u[2] = make_float3(r[9], r[10], r[11]);
    b.h[0] = r[12];
    b.h[1] = r[13];
    b.h[2] = r[14];
    b.rb = r[15];
    return b;
}

// Depth of the four link boxes of one configuration against obstacle `ob` (cylinders
// first, then boxes), 0 when disjoint.
__device__ __forceinline__ float pair_depth(const SceneDev &sc, const float *boxes, int ob)
{
    float pen = 0.f;
    if (ob < sc.n_cyl) {
        const float4 f = __ldg(sc.cyl_filt + ob), e = __ldg(sc.cyl_exact + ob);
        const float rc = e.x / kOctCos, hz = 0.5f * (e.z - e.y);
        const float3 pc = make_float3(f.x, f.y, 0.5f * (e.y + e.z));
        const float rbo = sqrtf(fmaf(rc, rc, hz * hz));
#pragma unroll 1
        for (int l = 0; l < 4; ++l) {
            const Obb b = load_box(boxes + l * kBoxFloats);
            const float3 d = make_float3(pc.x - b.c.x, pc.y - b.c.y, pc.z - b.c.z);
            const float rr = b.rb + rbo;
            if (dot3(d, d) > rr * rr) continue;   // bounding spheres apart
            pen = fmaxf(pen, sat_prism(b, pc, rc, hz));
        }
    } else {
        const int bi = ob - sc.n_cyl;
        const float4 c = __ldg(sc.box_c + bi), h = __ldg(sc.box_h + bi);
        const float rbo = sqrtf(fmaf(h.x, h.x, fmaf(h.y, h.y, h.z * h.z)));
#pragma unroll 1
        for (int l = 0; l < 4; ++l) {
            const Obb b = load_box(boxes + l * kBoxFloats);
            const float3 d = make_float3(c.x - b.c.x, c.y - b.c.y, c.z - b.c.z);
            const float rr = b.rb + rbo;
            if (dot3(d, d) > rr * rr) continue;
            pen = fmaxf(pen, sat_box(b, make_float3(c.x, c.y, c.z), make_float3(h.x, h.y, h.z)));
        }
    }
    return pen;
}

// Entries 0..count-1 of the warp's queue, one per lane: (configuration lane, obstacle); the
// depth goes to the owning lane's running maximum (non-negative floats order as their bits).
__device__ __forceinline__ void run_queue(const SceneDev &sc, const float *s_boxes, const int *queue, int count,
                                          int *s_pen, int lane)
{
    if (lane < count) {
        const int e = queue[lane];
        const int owner = e & 31, ob = e >> 5;
        const float pen = pair_depth(sc, s_boxes + owner * 4 * kBoxFloats, ob);
        if (pen > 0.f) atomicMax(s_pen + owner, __float_as_int(pen));
    }
    __syncwarp();
}

// The hull penetration of configuration q on this lane, the warp working together: one
// lane per configuration for the kinematics and the obstacle scan; the (configuration,
// obstacle) pairs that pass the scan's plane and range tests join the warp's queue, and the
// warp works through them 32 at a time, one pair per lane, so that the separating-axis work
// runs on full warps whatever pairs each configuration has. s_box (32 x 4 boxes), s_pen (32)
// and queue (64) are the warp's shared memory. Every lane of the warp must call it. With
// BROAD (the lanes' configurations are neighbours on a path), the obstacles first go
// through the broad phase of the sphere forms: the box, in the slew frame of lane 16, that
// holds every lane's arm extent [h_lo, h_hi] on its plane, against the Morton-ordered groups
// of eight cylinders and then their members, dilated by the hulls' half width and by how
// far a prism reaches beyond the records' sphere reach.
template <bool BROAD>
__device__ __forceinline__ float hull_pen_warp(const ModelDev &m, const SceneDev &sc, const HullDims &hd, float4 q,
                                               bool live, float *s_box, int *s_pen, int *queue, int lane)
{
    float s1, c1, s2, c2, s23, c23;
    sincosf(q.x, &s1, &c1);
    sincosf(q.y, &s2, &c2);
    sincosf(q.y + q.z, &s23, &c23);
    const float3 eb = make_float3(c2 * c1, c2 * s1, s2), ej = make_float3(c23 * c1, c23 * s1, s23);
    const float3 n = make_float3(-s1, c1, 0.f);
    const float3 J = make_float3(m.boom_len * eb.x, m.boom_len * eb.y, fmaf(m.boom_len, eb.z, m.base_z));
    const float tl = m.jib_len + q.w;
    const float3 T = make_float3(fmaf(tl, ej.x, J.x), fmaf(tl, ej.y, J.y), fmaf(tl, ej.z, J.z));
    const float q4p = fmaxf(q.w, 0.f);
    float *mine = s_box + lane * 4 * kBoxFloats;
    const float hb = 0.5f * m.boom_len, hj = 0.5f * m.jib_len, tc = fmaf(0.5f, q4p, m.jib_len);
    store_box(mine, make_float3(hb * eb.x, hb * eb.y, fmaf(hb, eb.z, m.base_z)), eb, n, hb + hd.pad, hd.w[0],
              hd.hh[0]);
    store_box(mine + kBoxFloats, make_float3(fmaf(hj, ej.x, J.x), fmaf(hj, ej.y, J.y), fmaf(hj, ej.z, J.z)), ej, n,
              hj + hd.pad, hd.w[1], hd.hh[1]);
    store_box(mine + 2 * kBoxFloats, make_float3(fmaf(tc, ej.x, J.x), fmaf(tc, ej.y, J.y), fmaf(tc, ej.z, J.z)), ej,
              n, fmaf(0.5f, q4p, hd.pad), hd.w[2], hd.hh[2]);
    store_box(mine + 3 * kBoxFloats, make_float3(T.x, T.y, T.z - 0.5f * hd.glen), make_float3(c1, s1, 0.f), n,
              hd.gw, hd.gw, 0.5f * hd.glen);
    s_pen[lane] = 0;
    // every hull point lies within wmax of the crane's vertical plane, and its coordinate
    // along the slew direction within [h_lo, h_hi]: the arm's joints O, J, the jib's end and
    // T, widened by an arm box's end pad plus its in-plane half extent, or the grapple's
    // half width
    const float wmax = fmaxf(fmaxf(hd.w[0], hd.w[1]), fmaxf(hd.w[2], hd.gw));
    const float ext = fmaxf(hd.pad + fmaxf(fmaxf(hd.hh[0], hd.hh[1]), hd.hh[2]), hd.gw);
    const float hJ = m.boom_len * c2, hT = fmaf(tl, c23, hJ), hE = fmaf(m.jib_len, c23, hJ);
    const float h_lo = fminf(fminf(0.f, hJ), fminf(hT, hE)) - ext, h_hi = fmaxf(fmaxf(0.f, hJ), fmaxf(hT, hE)) + ext;
    __syncwarp();
    int count = 0;
    // one obstacle for every lane: its plane and range test, the queue, and a full round of
    // pairs whenever 32 are waiting (warp-uniform)
    auto scan_one = [&](int o) {
        float cx, cy, reach;
        if (o < sc.n_cyl) {
            const float4 f = __ldg(sc.cyl_filt + o);
            cx = f.x;
            cy = f.y;
            reach = __ldg(&sc.cyl_exact[o].x) / kOctCos;
        } else {
            const float4 c = __ldg(sc.box_c + o - sc.n_cyl), h = __ldg(sc.box_h + o - sc.n_cyl);
            cx = c.x;
            cy = c.y;
            reach = sqrtf(fmaf(h.x, h.x, h.y * h.y));
        }
        const float v = fmaf(-s1, cx, c1 * cy), u = fmaf(c1, cx, s1 * cy);
        const bool pass = live && fabsf(v) <= reach + wmax + 1e-3f && u >= h_lo - reach - 1e-3f &&
                          u <= h_hi + reach + 1e-3f;
        const uint32_t mask = __ballot_sync(0xffffffffu, pass);
        if (pass) queue[count + __popc(mask & ((1u << lane) - 1u))] = lane | (o << 5);
        count += __popc(mask);
        __syncwarp();
        if (count >= 32) {
            run_queue(sc, s_box, queue, 32, s_pen, lane);
            const int rest = count - 32;
            const int moved = lane < rest ? queue[32 + lane] : 0;
            __syncwarp();
            if (lane < rest) queue[lane] = moved;
            count = rest;
            __syncwarp();
        }
    };
    if (BROAD) {
        const float hbnd[2] = {h_lo, h_hi};
        const UnitFrame fr = unit_frame<2>(s1, c1, hbnd);
        const float extra = wmax + hd.reach_extra + 1e-3f;
        const int n_grp = n_groups(sc.n_cyl);
        for (int gbase = 0; gbase < n_grp; gbase += 32) {
            uint32_t gmask = __ballot_sync(0xffffffffu, gbase + lane < n_grp &&
                                                            unit_near(fr, __ldg(sc.cyl_group + gbase + lane), extra));
            while (gmask) {
                // lane l takes member l % 8 of the (l / 8)-th remaining group
                uint32_t g = gmask;
                const int slot = lane >> 3;
                g = slot >= 1 ? g & (g - 1) : g;
                g = slot >= 2 ? g & (g - 1) : g;
                g = slot >= 3 ? g & (g - 1) : g;
                const int o = g ? (gbase + __ffs(g) - 1) * kGroup + (lane & (kGroup - 1)) : sc.n_cyl;
#pragma unroll
                for (int k = 0; k < 4; ++k) gmask &= gmask - 1;
                uint32_t mmask = __ballot_sync(0xffffffffu, o < sc.n_cyl && unit_near(fr, __ldg(sc.cyl_filt + o), extra));
                while (mmask) {
                    const int ob = __shfl_sync(0xffffffffu, o, __ffs(mmask) - 1);
                    mmask &= mmask - 1;
                    scan_one(ob);
                }
            }
        }
        for (int b = 0; b < sc.n_box; ++b) scan_one(sc.n_cyl + b);
    } else {
        for (int o = 0; o < sc.n_cyl + sc.n_box; ++o) scan_one(o);
    }
    if (count > 0) run_queue(sc, s_box, queue, count, s_pen, lane);
    return __int_as_float(s_pen[lane]);
}

__global__ void __launch_bounds__(kHullThreads)
k_hull_penetration(const ModelDev m, const SceneDev sc, const HullArgs a)
{
    __shared__ float s_box[kHullWarps][32 * 4 * kBoxFloats];
    __shared__ int s_pen[kHullWarps][32];
    __shared__ int s_queue[kHullWarps][64];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < a.n;
    const float pen =
        hull_pen_warp<false>(m, sc, a.d, a.q[live ? i : 0], live, s_box[wib], s_pen[wib], s_queue[wib], lane);
    if (live) a.pen[i] = pen;
}

// The path evaluation with the hull model: a warp per (candidate, 32 checkpoints), the
// checkpoint's configuration and costs as in the sphere forms, its collision term the hull
// penetration (d = -depth where the hulls meet an obstacle, +inf elsewhere: only the
// penetration enters J_c and the flags).
__global__ void __launch_bounds__(kHullThreads)
k_eval_hulls(const ModelDev m, const SceneDev sc, const HullDims hd, const EvalArgs a)
{
    extern __shared__ __align__(16) float4 s_basis[];
    __shared__ float s_box[kHullWarps][32 * 4 * kBoxFloats];
    __shared__ int s_pen[kHullWarps][32];
    __shared__ int s_queue[kHullWarps][64];
    __shared__ float4 s_ctrl_all[kHullWarps][CP_MAX_WAYPOINTS + 8];
    for (int i = threadIdx.x; i < 2 * a.S; i += blockDim.x) s_basis[i] = a.basis[i];
    __syncthreads();
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int n_warps = (int)((gridDim.x * blockDim.x) >> 5);
    float4 *s_ctrl = s_ctrl_all[wib];
    for (int it = queue_first(a, warp, lane); it < a.n * a.P; it = queue_next(a, it, n_warps, lane)) {
        const ItemRange ir = item_range(a, it);
        stage_controls(s_ctrl, a, ir.cand, lane);
        double acc = 0.0;
        uint32_t count = 0;
        for (int chunk = ir.c0; chunk < ir.c1; ++chunk) {
            const Checkpoint c = checkpoint_at(m, a, s_basis, s_ctrl, chunk, lane);
            const float pen = hull_pen_warp<true>(m, sc, hd, c.q, true, s_box[wib], s_pen[wib], s_queue[wib], lane);
            __syncwarp();
            unit_accumulate(a, c, pen > 0.f ? -pen : CUDART_INF_F, ir.cand, chunk, lane, acc, count);
        }
        item_flush(a, it, acc, count, lane);
    }
}

}  // namespace

int launch_hull_penetration(const ModelDev &m, const SceneDev &sc, const HullDims &d, const float *q, int n, float *pen,
                            cudaStream_t st)
{
    if (n == 0) return CP_OK;
    HullArgs a{};
    a.q = (const float4 *)q;
    a.n = n;
    a.d = d;
    a.pen = pen;
    k_hull_penetration<<<(n + kHullThreads - 1) / kHullThreads, kHullThreads, 0, st>>>(m, sc, a);
    CP_LAUNCHED("k_hull_penetration");
    return CP_OK;
}

int launch_eval_hulls(const ModelDev &m, const SceneDev &sc, const HullDims &d, const EvalArgs &a, int num_sms,
                      cudaStream_t st)
{
    const size_t smem = sizeof(float4) * 2 * (size_t)a.S;
    CP_CUDA(cudaFuncSetAttribute(k_eval_hulls, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eval_hulls, kHullThreads, smem));
    if (per_sm < 1) per_sm = 1;
    const long long items = (long long)a.n * a.P;
    long long blocks = (items + kHullWarps - 1) / kHullWarps;
    if (blocks > (long long)num_sms * per_sm) blocks = (long long)num_sms * per_sm;
    if (a.queue != nullptr) CP_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(int), st));
    k_eval_hulls<<<(unsigned)blocks, kHullThreads, smem, st>>>(m, sc, d, a);
    CP_LAUNCHED("k_eval_hulls");
    return CP_OK;
}

}  // namespace cp
