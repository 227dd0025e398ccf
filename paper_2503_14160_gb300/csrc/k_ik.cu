// Collision-free inverse kinematics (arXiv 2503.14160, Sec. 3.2, Eq. IK opt): for every
// target pose (x, y, z, psi), the configuration q minimising |r|^2 with
//   r = [p_g - p_d, lambda_q Log(R_d^T R_g), lambda_c max(0, -d(q))],
// p_g the grapple centre (grapple_len below the tip, plumb) and R_g = Rz(q1); the passive
// joints' equilibrium residual is zero by the chain's reading. Damped Gauss-Newton
// (Levenberg-Marquardt) from several starting points per target, the best kept.
//
// One thread per (target, start): the lanes of a warp take the starts of one to 32 targets
// (a group of G lanes per target, G the power of two >= min(starts, 32); more starts loop
// over the group's lanes), so a warp instruction advances up to 32 solves. Each thread
// scans the obstacles in the same order (the loads are warp-wide broadcasts) and evaluates
// sphere distances only for obstacles that pass a plane test. The best start of a target
// is found by shuffles within its group; a NaN cost (a NaN target) ranks as +inf there.
#include "eval_common.cuh"
#include "philox.cuh"

namespace cp {
namespace {

constexpr int kIKThreads = 128;
constexpr int kIKMinBlocks = 7;            // 28 warps per SM: 72 registers a thread
constexpr int kIKStagedObstacles = 1024;   // up to this many obstacles, plane-test records in
                                           // shared memory (16 KB; 7 CTAs fit an SM)
constexpr uint32_t kIKTag = 0x494B5354u;   // third Philox counter word of the starting points

struct IKArgs {
    const float4 *targets;   // [n] {x, y, z, psi}
    const float4 *q_init;    // [n] or null: start of restart 0
    int n, restarts, iters;
    int group;               // lanes per target (power of two, <= 32)
    float lambda_q, lambda_c, grapple_len, mu0;
    uint32_t k0, k1, query;
    float4 *q_out;           // [n]
    float *f_out;            // [n]
    int *restart_out;        // [n] or null
    float *r_out;            // [n][5] or null: residual at q_out
};

// One evaluation in the form the step needs: the residual, |r|^2 and the normal equations
// H = J^T J (upper triangle, row-major: 00 01 02 03 11 12 13 22 23 33) and g = J^T r.
struct Eval {
    float r[5];
    float f;
    float H[10];
    float g[4];
};

// H += j^T j, g += j^T rk for one residual row j.
__device__ __forceinline__ void add_row(Eval &ev, float j0, float j1, float j2, float j3, float rk)
{
    ev.H[0] = fmaf(j0, j0, ev.H[0]);
    ev.H[1] = fmaf(j0, j1, ev.H[1]);
    ev.H[2] = fmaf(j0, j2, ev.H[2]);
    ev.H[3] = fmaf(j0, j3, ev.H[3]);
    ev.H[4] = fmaf(j1, j1, ev.H[4]);
    ev.H[5] = fmaf(j1, j2, ev.H[5]);
    ev.H[6] = fmaf(j1, j3, ev.H[6]);
    ev.H[7] = fmaf(j2, j2, ev.H[7]);
    ev.H[8] = fmaf(j2, j3, ev.H[8]);
    ev.H[9] = fmaf(j3, j3, ev.H[9]);
    ev.g[0] = fmaf(j0, rk, ev.g[0]);
    ev.g[1] = fmaf(j1, rk, ev.g[1]);
    ev.g[2] = fmaf(j2, rk, ev.g[2]);
    ev.g[3] = fmaf(j3, rk, ev.g[3]);
}

// x - 2 pi round(x / 2 pi), the remainder of x by 2 pi in [-pi, pi]; 2 pi is split into a
// float head and tail (Cody and Waite) so that n 2 pi is subtracted to ~1e-7 rad for the
// small n met here (|x| within a few turns).
__device__ __forceinline__ float wrap_angle(float x)
{
    const float n = rintf(x * 0.159154943091895336f);
    return fmaf(-n, -1.74845553e-7f, fmaf(-n, 6.28318548202514648f, x));
}

// Kinematic quantities of one configuration shared by the residual and the Jacobian.
struct Pose {
    float s1, c1, s2, c2, s23, c23, q4;
};

// Shared-memory records of a CTA: the sphere table, and per thread the sphere centres of
// the configuration being evaluated (h and z of sphere s at [s][thread]), so that the
// obstacle loop reads them instead of holding them in registers.
template <int NSPH>
struct IKShared {
    SphereLin sph[NSPH];
    float h[NSPH][kIKThreads];
    float z[NSPH][kIKThreads];
};

// Centre of sphere s at the pose, in polar form (h along the slew direction, z).
__device__ __forceinline__ void sphere_polar(const ModelDev &m, const Pose &p, int s, float &h, float &z, float &L)
{
    const SphereLin sp = m.sph[s];
    L = fmaf(sp.gamma, p.q4, sp.beta);
    h = fmaf(sp.alpha, p.c2, L * p.c23);
    z = m.base_z + fmaf(sp.alpha, p.s2, fmaf(L, p.s23, -sp.delta));
}

// The most negative sphere-obstacle distance and its pair (key s (n_cyl + n_box) + o,
// cylinders first, the lower key kept on ties). Only negative distances enter the
// residual, so pairs that cannot be negative are skipped. Every centre is (c1 h, s1 h, z):
// at squared horizontal distance (h - u)^2 + v^2 from a point with plane coordinates
// (u, v) (u along the slew direction, v across). A cylinder is skipped when v^2 is above
// (R + r_max)^2 plus the filter margin (its bound .w) or u lies beyond the spheres' range
// of h by more than its reach (a bound above R + r_max); a sphere of a kept cylinder when
// (h - u)^2 + v^2 is above the same bound. A box is skipped when its footprint circle
// (radius .w, which includes r_max) is that far from the plane or the range. Every skipped
// pair has a distance >= 0. d = +inf when no pair is negative.
template <int NSPH, bool STAGED>
__device__ __forceinline__ void scan_distance(const ModelDev &m, const SceneDev &sc, const Pose &p,
                                              IKShared<NSPH> &sm, const float4 *s_obs, float &d, int &key)
{
    const int n_obs = sc.n_cyl + sc.n_box;
    const int tid = threadIdx.x;
    float h_lo = CUDART_INF_F, h_hi = -CUDART_INF_F;
#pragma unroll
    for (int s = 0; s < NSPH; ++s) {
        float h, z, L;
        sphere_polar(m, p, s, h, z, L);
        sm.h[s][tid] = h;
        sm.z[s][tid] = z;
        h_lo = fminf(h_lo, h);
        h_hi = fmaxf(h_hi, h);
    }
    d = 0.f;
    key = 0x7fffffff;
    for (int o = 0; o < sc.n_cyl; ++o) {
        // plane test on {cx, cy, reach, (R + r_max)^2 + margin}; the exact record on a pass
        float4 f;
        if (STAGED) {
            f = s_obs[o];
        } else {
            f = __ldg(sc.cyl_filt + o);
            f.z = __ldg(&sc.cyl_exact[o].w);
            const float r = f.w;
            f.w = f.z;
            f.z = r;
        }
        const float u = fmaf(p.c1, f.x, p.s1 * f.y), v = fmaf(-p.s1, f.x, p.c1 * f.y);
        if (v * v >= f.w || u < h_lo - f.z || u > h_hi + f.z) continue;
        const float4 e = __ldg(sc.cyl_exact + o);
#pragma unroll 1
        for (int s = 0; s < NSPH; ++s) {
            const float h = sm.h[s][tid];
            const float dx = h - u;
            if (fmaf(dx, dx, v * v) >= e.w) continue;
            const float t = sdf_cylinder(__fmul_rn(p.c1, h), __fmul_rn(p.s1, h), sm.z[s][tid], f.x, f.y, e) -
                            sm.sph[s].radius;
            const int k = s * n_obs + o;
            if (t < d || (t == d && d < 0.f && k < key)) {
                d = t;
                key = k;
            }
        }
    }
    for (int b = 0; b < sc.n_box; ++b) {
        const float4 cb = STAGED ? s_obs[sc.n_cyl + b] : __ldg(sc.box_c + b);
        const float u = fmaf(p.c1, cb.x, p.s1 * cb.y), v = fmaf(-p.s1, cb.x, p.c1 * cb.y);
        if (fabsf(v) >= cb.w || u < h_lo - cb.w || u > h_hi + cb.w) continue;
        const float4 c = __ldg(sc.box_c + b), hb = __ldg(sc.box_h + b);
#pragma unroll 1
        for (int s = 0; s < NSPH; ++s) {
            const float h = sm.h[s][tid];
            const float t = sdf_box(__fmul_rn(p.c1, h), __fmul_rn(p.s1, h), sm.z[s][tid], c, hb) - sm.sph[s].radius;
            const int k = s * n_obs + sc.n_cyl + b;
            if (t < d || (t == d && d < 0.f && k < key)) {
                d = t;
                key = k;
            }
        }
    }
    if (key == 0x7fffffff) d = CUDART_INF_F;
}

// r(q) and dr/dq for the target.
template <int NSPH, bool STAGED>
__device__ __forceinline__ void evaluate(const ModelDev &m, const SceneDev &sc, const IKArgs &a, float4 q,
                                         float4 tg, IKShared<NSPH> &sm, const float4 *s_obs, Eval &ev)
{
    Pose p;
    sincosf(q.x, &p.s1, &p.c1);
    sincosf(q.y, &p.s2, &p.c2);
    sincosf(q.y + q.z, &p.s23, &p.c23);
    p.q4 = q.w;
    // the tip: boom L_b along e_b, (L_j + q4) along e_j
    const float Lb = m.boom_len, Lt = m.jib_len + q.w;
    const float ht = fmaf(Lb, p.c2, Lt * p.c23), zt = m.base_z + fmaf(Lb, p.s2, Lt * p.s23);
    // explicit fused forms: every instance of this function rounds the residual alike
    ev.r[0] = fmaf(p.c1, ht, -tg.x);
    ev.r[1] = fmaf(p.s1, ht, -tg.y);
    ev.r[2] = zt - a.grapple_len - tg.z;
    ev.r[3] = a.lambda_q * wrap_angle(q.x - tg.w);
    float d;
    int key;
    scan_distance<NSPH, STAGED>(m, sc, p, sm, s_obs, d, key);
    ev.r[4] = a.lambda_c * fmaxf(0.f, -d);
    // Jacobian rows (tip, yaw, collision: the gradient of the attaining pair) folded into
    // the normal equations as they are formed
#pragma unroll
    for (int i = 0; i < 10; ++i) ev.H[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) ev.g[i] = 0.f;
    const float dh2 = -fmaf(Lb, p.s2, Lt * p.s23), dh3 = -Lt * p.s23, dh4 = p.c23;
    const float dz2 = fmaf(Lb, p.c2, Lt * p.c23), dz3 = Lt * p.c23, dz4 = p.s23;
    add_row(ev, -p.s1 * ht, p.c1 * dh2, p.c1 * dh3, p.c1 * dh4, ev.r[0]);
    add_row(ev, p.c1 * ht, p.s1 * dh2, p.s1 * dh3, p.s1 * dh4, ev.r[1]);
    add_row(ev, 0.f, dz2, dz3, dz4, ev.r[2]);
    add_row(ev, a.lambda_q, 0.f, 0.f, 0.f, ev.r[3]);
    if (d < 0.f) {
        const int n_obs = sc.n_cyl + sc.n_box;
        const int s = key / n_obs, o = key - s * n_obs;
        const SphereLin sp = sm.sph[s];
        const float h = sm.h[s][threadIdx.x], pz = sm.z[s][threadIdx.x];
        const float L = fmaf(sp.gamma, p.q4, sp.beta);
        const float px = __fmul_rn(p.c1, h), py = __fmul_rn(p.s1, h);
        float3 g;
        if (o < sc.n_cyl) {
            const float4 f = __ldg(sc.cyl_filt + o), e = __ldg(sc.cyl_exact + o);
            g = sdf_cylinder_grad(px, py, pz, f.x, f.y, e);
        } else {
            g = sdf_box_grad(px, py, pz, __ldg(sc.box_c + o - sc.n_cyl), __ldg(sc.box_h + o - sc.n_cyl));
        }
        const float ph2 = -fmaf(sp.alpha, p.s2, L * p.s23), ph3 = -L * p.s23, ph4 = sp.gamma * p.c23;
        const float pz2 = fmaf(sp.alpha, p.c2, L * p.c23), pz3 = L * p.c23, pz4 = sp.gamma * p.s23;
        // d(centre)/dq: slew turns (x, y) = (c1 h, s1 h); the others move h and z
        const float gh = fmaf(g.x, p.c1, g.y * p.s1);   // gradient along the slew direction
        const float k = -a.lambda_c;
        add_row(ev, k * h * fmaf(-g.x, p.s1, g.y * p.c1), k * fmaf(gh, ph2, g.z * pz2),
                k * fmaf(gh, ph3, g.z * pz3), k * fmaf(gh, ph4, g.z * pz4), ev.r[4]);
    }
    float f = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) f = fmaf(ev.r[i], ev.r[i], f);
    ev.f = f;
}

__device__ __forceinline__ float4 clamp_q(const ModelDev &m, float4 q)
{
    return make_float4(fminf(fmaxf(q.x, m.q_min[0]), m.q_max[0]), fminf(fmaxf(q.y, m.q_min[1]), m.q_max[1]),
                       fminf(fmaxf(q.z, m.q_min[2]), m.q_max[2]), fminf(fmaxf(q.w, m.q_min[3]), m.q_max[3]));
}

// Solves (H + mu (diag H + 1e-6)) s = -g by Cholesky, L L^T with the reciprocal pivots
// from the hardware reciprocal square root (within 2 ulp) so that no division is needed.
__device__ __forceinline__ float4 damped_step(const Eval &ev, float mu)
{
    const float a00 = fmaf(mu, ev.H[0] + 1e-6f, ev.H[0]), a11 = fmaf(mu, ev.H[4] + 1e-6f, ev.H[4]);
    const float a22 = fmaf(mu, ev.H[7] + 1e-6f, ev.H[7]), a33 = fmaf(mu, ev.H[9] + 1e-6f, ev.H[9]);
    const float i0 = rsqrtf(fmaxf(a00, 1e-30f));
    const float l10 = ev.H[1] * i0, l20 = ev.H[2] * i0, l30 = ev.H[3] * i0;
    const float i1 = rsqrtf(fmaxf(fmaf(-l10, l10, a11), 1e-30f));
    const float l21 = fmaf(-l20, l10, ev.H[5]) * i1, l31 = fmaf(-l30, l10, ev.H[6]) * i1;
    const float i2 = rsqrtf(fmaxf(fmaf(-l21, l21, fmaf(-l20, l20, a22)), 1e-30f));
    const float l32 = fmaf(-l31, l21, fmaf(-l30, l20, ev.H[8])) * i2;
    const float i3 = rsqrtf(fmaxf(fmaf(-l32, l32, fmaf(-l31, l31, fmaf(-l30, l30, a33))), 1e-30f));
    // L y = -g, then L^T x = y
    const float y0 = -ev.g[0] * i0;
    const float y1 = fmaf(-l10, y0, -ev.g[1]) * i1;
    const float y2 = fmaf(-l21, y1, fmaf(-l20, y0, -ev.g[2])) * i2;
    const float y3 = fmaf(-l32, y2, fmaf(-l31, y1, fmaf(-l30, y0, -ev.g[3]))) * i3;
    const float x3 = y3 * i3;
    const float x2 = fmaf(-l32, x3, y2) * i2;
    const float x1 = fmaf(-l31, x3, fmaf(-l21, x2, y1)) * i1;
    const float x0 = fmaf(-l30, x3, fmaf(-l20, x2, fmaf(-l10, x1, y0))) * i0;
    return make_float4(x0, x1, x2, x3);
}

__device__ __forceinline__ float rank_cost(float f) { return f == f ? f : CUDART_INF_F; }

template <int NSPH>
__device__ __forceinline__ float4 ik_start(const ModelDev &m, const IKArgs &a, int t, int restart)
{
    if (restart == 0 && a.q_init != nullptr) return a.q_init[t];
    const uint4 x = philox4x32_10(make_uint4((uint32_t)restart, (uint32_t)t, kIKTag, a.query), a.k0, a.k1);
    const float u0 = (float)(x.x >> 8) * 0x1p-24f, u1 = (float)(x.y >> 8) * 0x1p-24f;
    const float u2 = (float)(x.z >> 8) * 0x1p-24f, u3 = (float)(x.w >> 8) * 0x1p-24f;
    return make_float4(fmaf(u0, m.q_max[0] - m.q_min[0], m.q_min[0]), fmaf(u1, m.q_max[1] - m.q_min[1], m.q_min[1]),
                       fmaf(u2, m.q_max[2] - m.q_min[2], m.q_min[2]), fmaf(u3, m.q_max[3] - m.q_min[3], m.q_min[3]));
}

// Thread (target t, lane j of its group) solves the starts j, j + G, ... of t and keeps
// its best (the lowest |r|^2, the lower start on ties); the group then agrees on the best.
template <int NSPH, bool STAGED>
__global__ void __launch_bounds__(kIKThreads, kIKMinBlocks)
k_ik(const ModelDev m, const SceneDev sc, const IKArgs a)
{
    __shared__ IKShared<NSPH> sm;
    extern __shared__ float4 s_obs[];   // STAGED: the plane-test records of every obstacle
    if (threadIdx.x < NSPH) sm.sph[threadIdx.x] = m.sph[threadIdx.x];
    if (STAGED) {
        for (int o = threadIdx.x; o < sc.n_cyl; o += kIKThreads) {
            const float4 f = sc.cyl_filt[o];
            s_obs[o] = make_float4(f.x, f.y, f.w, sc.cyl_exact[o].w);
        }
        for (int b = threadIdx.x; b < sc.n_box; b += kIKThreads) s_obs[sc.n_cyl + b] = sc.box_c[b];
    }
    __syncthreads();
    const int G = a.group;
    const long long gid = (long long)blockIdx.x * kIKThreads + threadIdx.x;
    const int j = threadIdx.x & (G - 1);
    const bool live = gid / G < a.n;
    const int t = live ? (int)(gid / G) : a.n - 1;
    const float4 tg = a.targets[t];
    float best_f = CUDART_INF_F;
    int best_k = -1;
    float4 best_q = make_float4(0.f, 0.f, 0.f, 0.f);
    Eval ev, en;
    for (int k = j; k < a.restarts; k += G) {
        float4 q = clamp_q(m, ik_start<NSPH>(m, a, t, k));
        float mu = a.mu0;
        evaluate<NSPH, STAGED>(m, sc, a, q, tg, sm, s_obs, ev);
        for (int it = 0; it < a.iters; ++it) {
            const float4 st = damped_step(ev, mu);
            const float4 qn = clamp_q(m, make_float4(q.x + st.x, q.y + st.y, q.z + st.z, q.w + st.w));
            if (qn.x == q.x && qn.y == q.y && qn.z == q.z && qn.w == q.w) {
                // the step vanished in rounding: the trial is q itself, whose cost is not
                // below its own, so the step is rejected without evaluating it again
                mu = fminf(mu * 4.f, 1e12f);
                continue;
            }
            evaluate<NSPH, STAGED>(m, sc, a, qn, tg, sm, s_obs, en);
            if (en.f < ev.f) {
                q = qn;
                ev = en;
                mu = fmaxf(mu * (1.f / 3.f), 1e-12f);
            } else {
                mu = fminf(mu * 4.f, 1e12f);
            }
        }
        if (best_k < 0 || rank_cost(ev.f) < rank_cost(best_f)) {
            best_f = ev.f;
            best_k = k;
            best_q = q;
        }
    }
    // best over the group: (f, start) in lexicographic order; lanes without a start rank last
    float fr = best_k >= 0 ? rank_cost(best_f) : CUDART_INF_F;
    int kr = best_k >= 0 ? best_k : 0x7fffffff;
    for (int off = G >> 1; off > 0; off >>= 1) {
        const float f2 = __shfl_xor_sync(0xffffffffu, fr, off);
        const int k2 = __shfl_xor_sync(0xffffffffu, kr, off);
        if (f2 < fr || (f2 == fr && k2 < kr)) {
            fr = f2;
            kr = k2;
        }
    }
    const int owner = ((int)threadIdx.x & 31 & ~(G - 1)) | (kr & (G - 1));   // the lane that solved start kr
    const float4 qb = make_float4(__shfl_sync(0xffffffffu, best_q.x, owner), __shfl_sync(0xffffffffu, best_q.y, owner),
                                  __shfl_sync(0xffffffffu, best_q.z, owner), __shfl_sync(0xffffffffu, best_q.w, owner));
    const float fb = __shfl_sync(0xffffffffu, best_f, owner);
    if (live && j == 0) {
        a.q_out[t] = qb;
        a.f_out[t] = fb;
        if (a.restart_out != nullptr) a.restart_out[t] = kr;
    }
    if (a.r_out != nullptr) {
        // the residual at the answer, evaluated once more (the same arithmetic as the solve)
        evaluate<NSPH, STAGED>(m, sc, a, qb, tg, sm, s_obs, en);
        if (live && j == 0)
            for (int i = 0; i < 5; ++i) a.r_out[(size_t)t * 5 + i] = en.r[i];
    }
}

// Sphere centres and tip for single configurations (Sec. 2 kinematics in the linear
// placement form), one thread per configuration.
template <int NSPH>
__global__ void k_forward_kinematics(const ModelDev m, const float4 *__restrict__ q, int n,
                                     float *centres, float *tip)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 qi = q[i];
    float x[NSPH], y[NSPH], z[NSPH];
    crane_fk<NSPH, false>(m, qi, x, y, z);
    if (centres != nullptr) {
        float *c = centres + (size_t)i * m.n_spheres * 3;
#pragma unroll
        for (int s = 0; s < NSPH; ++s) {
            if (s < m.n_spheres) {
                c[3 * s] = x[s];
                c[3 * s + 1] = y[s];
                c[3 * s + 2] = z[s];
            }
        }
    }
    if (tip != nullptr) {
        float s1, c1, s2, c2, s23, c23;
        sincosf(qi.x, &s1, &c1);
        sincosf(qi.y, &s2, &c2);
        sincosf(qi.y + qi.z, &s23, &c23);
        const float Lt = m.jib_len + qi.w;
        const float h = fmaf(m.boom_len, c2, Lt * c23);
        tip[3 * (size_t)i] = c1 * h;
        tip[3 * (size_t)i + 1] = s1 * h;
        tip[3 * (size_t)i + 2] = m.base_z + fmaf(m.boom_len, s2, Lt * s23);
    }
}

}  // namespace

int launch_ik(const ModelDev &m, const SceneDev &sc, const float *targets, const float *q_init, int n,
              int restarts, int iters, float lambda_q, float lambda_c, float grapple_len, float mu0,
              uint64_t seed, uint32_t query, float *q_out, float *f_out, int *restart_out, float *r_out,
              cudaStream_t st)
{
    if (n == 0) return CP_OK;
    IKArgs a{};
    a.targets = (const float4 *)targets;
    a.q_init = (const float4 *)q_init;
    a.n = n;
    a.restarts = restarts;
    a.iters = iters;
    a.lambda_q = lambda_q;
    a.lambda_c = lambda_c;
    a.grapple_len = grapple_len;
    a.mu0 = mu0;
    a.k0 = (uint32_t)seed;
    a.k1 = (uint32_t)(seed >> 32);
    a.query = query;
    a.q_out = (float4 *)q_out;
    a.f_out = f_out;
    a.restart_out = restart_out;
    a.r_out = r_out;
    int G = 1;
    while (G < restarts && G < 32) G <<= 1;
    a.group = G;
    const long long blocks = ((long long)n * G + kIKThreads - 1) / kIKThreads;
    const int n_obs = sc.n_cyl + sc.n_box;
    const bool staged = n_obs <= kIKStagedObstacles;
    const size_t smem = staged ? sizeof(float4) * (size_t)n_obs : 0;
    if (m.n_spheres == 12) {
        if (staged) k_ik<12, true><<<(unsigned)blocks, kIKThreads, smem, st>>>(m, sc, a);
        else k_ik<12, false><<<(unsigned)blocks, kIKThreads, 0, st>>>(m, sc, a);
    } else {
        if (staged) k_ik<16, true><<<(unsigned)blocks, kIKThreads, smem, st>>>(m, sc, a);
        else k_ik<16, false><<<(unsigned)blocks, kIKThreads, 0, st>>>(m, sc, a);
    }
    CP_LAUNCHED("k_ik");
    return CP_OK;
}

int launch_forward_kinematics(const ModelDev &m, const float *q, int n, float *centres, float *tip,
                              cudaStream_t st)
{
    if (n == 0) return CP_OK;
    const int threads = 128;
    const int blocks = (n + threads - 1) / threads;
    if (m.n_spheres == 12)
        k_forward_kinematics<12><<<blocks, threads, 0, st>>>(m, (const float4 *)q, n, centres, tip);
    else
        k_forward_kinematics<16><<<blocks, threads, 0, st>>>(m, (const float4 *)q, n, centres, tip);
    CP_LAUNCHED("k_forward_kinematics");
    return CP_OK;
}

}  // namespace cp
