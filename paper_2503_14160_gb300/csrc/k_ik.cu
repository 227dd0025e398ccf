// Collision-free inverse kinematics (arXiv 2503.14160, Sec. 3.2, Eq. IK opt): for every
// target pose (x, y, z, psi), the configuration q minimising |r|^2 with
//   r = [p_g - p_d, lambda_q Log(R_d^T R_g), lambda_c max(0, -d(q))],
// p_g the grapple centre (grapple_len below the tip, plumb) and R_g = Rz(q1); the passive
// joints' equilibrium residual is zero by the chain's reading. Damped Gauss-Newton
// (Levenberg-Marquardt) from several starting points per target, the best kept.
//
// One CTA per target, one warp per starting point (up to 8 warps; more starts loop over
// the warps). Each evaluation of r and its Jacobian
// takes the kinematics on every lane and spreads the obstacles over the lanes for d(q) and
// its attaining pair; the 4x4 damped normal equations are solved by every lane (a Cholesky
// in FP32, identical on all lanes), so the warp stays converged. The best start of each
// target is chosen through shared memory at the end; a NaN cost (a NaN target) ranks as
// +inf there, so every lane agrees on the choice.
#include "eval_common.cuh"
#include "philox.cuh"

namespace cp {
namespace {

constexpr int kIKMaxWarps = 8;             // warps per target; more starts loop
constexpr uint32_t kIKTag = 0x494B5354u;   // third Philox counter word of the starting points

struct IKArgs {
    const float4 *targets;   // [n] {x, y, z, psi}
    const float4 *q_init;    // [n] or null: start of restart 0
    int n, restarts, iters;
    float lambda_q, lambda_c, grapple_len, mu0;
    uint32_t k0, k1, query;
    float4 *q_out;           // [n]
    float *f_out;            // [n]
    int *restart_out;        // [n] or null
    float *r_out;            // [n][5] or null: residual at q_out
};

struct Eval {
    float r[5];
    float J[5][4];
    float f;
};

// The most negative sphere-obstacle distance and its pair, spread over the warp's lanes;
// the pair key is s (n_cyl + n_box) + o (cylinders first), the lower key kept on ties.
// Only negative distances enter the residual, so an obstacle whose axis (cylinder) or
// bounding circle (box) lies farther from the crane's vertical plane than it can reach a
// sphere is skipped: every centre is (c1 h, s1 h, z), at squared horizontal distance
// (h - u)^2 + v^2 from a point whose plane coordinates are (u, v), so v^2 above
// (R + r_max)^2 (plus the filter margin) leaves every pair at a distance >= 0. When no pair
// is negative d is returned as +inf.
template <int NSPH>
__device__ __forceinline__ void warp_distance(const ModelDev &m, const SceneDev &sc, float s1, float c1,
                                              const float *x, const float *y, const float *z, int lane,
                                              float &d, int &key)
{
    const int n_obs = sc.n_cyl + sc.n_box;
    d = CUDART_INF_F;
    key = 0x7fffffff;
    for (int o = lane; o < sc.n_cyl; o += 32) {
        const float4 f = __ldg(sc.cyl_filt + o), e = __ldg(sc.cyl_exact + o);
        const float v = fmaf(-s1, f.x, c1 * f.y);
        if (v * v >= e.w) continue;
#pragma unroll
        for (int s = 0; s < NSPH; ++s) {
            const float t = sdf_cylinder(x[s], y[s], z[s], f.x, f.y, e) - m.sph[s].radius;
            const int k = s * n_obs + o;
            if (t < d || (t == d && k < key)) {
                d = t;
                key = k;
            }
        }
    }
    for (int b = lane; b < sc.n_box; b += 32) {
        const float4 c = __ldg(sc.box_c + b), h = __ldg(sc.box_h + b);
        const float v = fmaf(-s1, c.x, c1 * c.y);
        if (fabsf(v) >= c.w) continue;
#pragma unroll
        for (int s = 0; s < NSPH; ++s) {
            const float t = sdf_box(x[s], y[s], z[s], c, h) - m.sph[s].radius;
            const int k = s * n_obs + sc.n_cyl + b;
            if (t < d || (t == d && k < key)) {
                d = t;
                key = k;
            }
        }
    }
    if (!(d < 0.f)) {
        d = CUDART_INF_F;
        key = 0x7fffffff;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float d2 = __shfl_xor_sync(0xffffffffu, d, off);
        const int k2 = __shfl_xor_sync(0xffffffffu, key, off);
        if (d2 < d || (d2 == d && k2 < key)) {
            d = d2;
            key = k2;
        }
    }
}

// r(q) and dr/dq for the target; every lane returns the same values.
template <int NSPH>
__device__ __forceinline__ void evaluate(const ModelDev &m, const SceneDev &sc, const IKArgs &a, float4 q,
                                         float4 tg, int lane, Eval &ev)
{
    float H[NSPH], Z[NSPH], s1, c1;
    crane_fk_polar<NSPH>(m, q, H, Z, s1, c1);
    float X[NSPH], Y[NSPH];
#pragma unroll
    for (int s = 0; s < NSPH; ++s) {
        X[s] = __fmul_rn(c1, H[s]);
        Y[s] = __fmul_rn(s1, H[s]);
    }
    float s2, c2, s23, c23;
    sincosf(q.y, &s2, &c2);
    sincosf(q.y + q.z, &s23, &c23);
    // the tip: boom L_b along e_b, (L_j + q4) along e_j
    const float Lb = m.boom_len, Lt = m.jib_len + q.w;
    const float ht = fmaf(Lb, c2, Lt * c23), zt = m.base_z + fmaf(Lb, s2, Lt * s23);
    ev.r[0] = c1 * ht - tg.x;
    ev.r[1] = s1 * ht - tg.y;
    ev.r[2] = zt - a.grapple_len - tg.z;
    ev.r[3] = a.lambda_q * remainderf(q.x - tg.w, 6.28318530717958648f);
    float d;
    int key;
    warp_distance<NSPH>(m, sc, s1, c1, X, Y, Z, lane, d, key);
    ev.r[4] = a.lambda_c * fmaxf(0.f, -d);
    // Jacobian: tip rows, yaw row, collision row (gradient of the attaining pair)
    const float dh2 = -fmaf(Lb, s2, Lt * s23), dh3 = -Lt * s23, dh4 = c23;
    const float dz2 = fmaf(Lb, c2, Lt * c23), dz3 = Lt * c23, dz4 = s23;
    ev.J[0][0] = -s1 * ht; ev.J[0][1] = c1 * dh2; ev.J[0][2] = c1 * dh3; ev.J[0][3] = c1 * dh4;
    ev.J[1][0] = c1 * ht;  ev.J[1][1] = s1 * dh2; ev.J[1][2] = s1 * dh3; ev.J[1][3] = s1 * dh4;
    ev.J[2][0] = 0.f;      ev.J[2][1] = dz2;      ev.J[2][2] = dz3;      ev.J[2][3] = dz4;
    ev.J[3][0] = a.lambda_q; ev.J[3][1] = 0.f; ev.J[3][2] = 0.f; ev.J[3][3] = 0.f;
    ev.J[4][0] = ev.J[4][1] = ev.J[4][2] = ev.J[4][3] = 0.f;
    if (d < 0.f) {
        const int n_obs = sc.n_cyl + sc.n_box;
        const int s = key / n_obs, o = key - s * n_obs;
        const SphereLin sp = m.sph[s];
        const float L = fmaf(sp.gamma, q.w, sp.beta);
        const float h = fmaf(sp.alpha, c2, L * c23);
        const float px = __fmul_rn(c1, h), py = __fmul_rn(s1, h);
        const float pz = m.base_z + fmaf(sp.alpha, s2, fmaf(L, s23, -sp.delta));
        float3 g;
        if (o < sc.n_cyl) {
            const float4 f = __ldg(sc.cyl_filt + o), e = __ldg(sc.cyl_exact + o);
            g = sdf_cylinder_grad(px, py, pz, f.x, f.y, e);
        } else {
            g = sdf_box_grad(px, py, pz, __ldg(sc.box_c + o - sc.n_cyl), __ldg(sc.box_h + o - sc.n_cyl));
        }
        const float ph2 = -fmaf(sp.alpha, s2, L * s23), ph3 = -L * s23, ph4 = sp.gamma * c23;
        const float pz2 = fmaf(sp.alpha, c2, L * c23), pz3 = L * c23, pz4 = sp.gamma * s23;
        const float k = -a.lambda_c;
        ev.J[4][0] = k * (g.x * (-s1 * h) + g.y * (c1 * h));
        ev.J[4][1] = k * (g.x * c1 * ph2 + g.y * s1 * ph2 + g.z * pz2);
        ev.J[4][2] = k * (g.x * c1 * ph3 + g.y * s1 * ph3 + g.z * pz3);
        ev.J[4][3] = k * (g.x * c1 * ph4 + g.y * s1 * ph4 + g.z * pz4);
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

// Solves (H + mu (diag H + 1e-6)) s = -g for the 4x4 symmetric H by Cholesky.
__device__ __forceinline__ float4 damped_step(const Eval &ev, float mu)
{
    float A[4][4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float g = 0.f;
#pragma unroll
        for (int k = 0; k < 5; ++k) g = fmaf(ev.J[k][i], ev.r[k], g);
        b[i] = -g;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float h = 0.f;
#pragma unroll
            for (int k = 0; k < 5; ++k) h = fmaf(ev.J[k][i], ev.J[k][j], h);
            A[i][j] = h;
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) A[i][i] = fmaf(mu, A[i][i] + 1e-6f, A[i][i]);
    // A = L L^T in place (lower), then forward and back substitution
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float dj = A[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) dj = fmaf(-A[j][k], A[j][k], dj);
        dj = sqrtf(fmaxf(dj, 1e-30f));
        A[j][j] = dj;
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
            float v = A[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) v = fmaf(-A[i][k], A[j][k], v);
            A[i][j] = v / dj;
        }
    }
    float y[4], x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float v = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) v = fmaf(-A[i][k], y[k], v);
        y[i] = v / A[i][i];
    }
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        float v = y[i];
#pragma unroll
        for (int k = i + 1; k < 4; ++k) v = fmaf(-A[k][i], x[k], v);
        x[i] = v / A[i][i];
    }
    return make_float4(x[0], x[1], x[2], x[3]);
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

// One CTA per target; warp w solves the starts w, w + warps, ... and keeps its best (the
// lowest |r|^2, the lower start on ties).
template <int NSPH>
__global__ void __launch_bounds__(kIKMaxWarps * 32)
k_ik(const ModelDev m, const SceneDev sc, const IKArgs a)
{
    __shared__ float s_f[kIKMaxWarps];
    __shared__ int s_k[kIKMaxWarps];
    __shared__ float4 s_q[kIKMaxWarps];
    __shared__ float s_r[kIKMaxWarps][5];
    const int t = blockIdx.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    const float4 tg = a.targets[t];
    float best_f = CUDART_INF_F;
    int best_k = -1;
    float4 best_q = make_float4(0.f, 0.f, 0.f, 0.f);
    float best_r[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    Eval ev, en;
    for (int k = w; k < a.restarts; k += warps) {
        float4 q = clamp_q(m, ik_start<NSPH>(m, a, t, k));
        float mu = a.mu0;
        evaluate<NSPH>(m, sc, a, q, tg, lane, ev);
        for (int it = 0; it < a.iters; ++it) {
            const float4 st = damped_step(ev, mu);
            const float4 qn = clamp_q(m, make_float4(q.x + st.x, q.y + st.y, q.z + st.z, q.w + st.w));
            evaluate<NSPH>(m, sc, a, qn, tg, lane, en);
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
#pragma unroll
            for (int i = 0; i < 5; ++i) best_r[i] = ev.r[i];
        }
    }
    if (lane == 0) {
        s_f[w] = best_f;
        s_k[w] = best_k;
        s_q[w] = best_q;
#pragma unroll
        for (int i = 0; i < 5; ++i) s_r[w][i] = best_r[i];
    }
    __syncthreads();
    if (w == 0) {
        // best over the warps: (f, start) in lexicographic order
        float f = lane < warps ? rank_cost(s_f[lane]) : CUDART_INF_F;
        int k = lane < warps ? s_k[lane] : 0x7fffffff;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float f2 = __shfl_xor_sync(0xffffffffu, f, off);
            const int k2 = __shfl_xor_sync(0xffffffffu, k, off);
            if (f2 < f || (f2 == f && k2 < k)) {
                f = f2;
                k = k2;
            }
        }
        if (lane == 0) {
            const int wb = k % warps;   // the warp that solved start k
            a.q_out[t] = s_q[wb];
            a.f_out[t] = s_f[wb];
            if (a.restart_out != nullptr) a.restart_out[t] = k;
        }
        if (a.r_out != nullptr && lane < 5) a.r_out[(size_t)t * 5 + lane] = s_r[k % warps][lane];
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
    crane_fk<NSPH>(m, qi, x, y, z);
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
    const int threads = 32 * (restarts < kIKMaxWarps ? restarts : kIKMaxWarps);
    if (m.n_spheres == 12)
        k_ik<12><<<n, threads, 0, st>>>(m, sc, a);
    else
        k_ik<16><<<n, threads, 0, st>>>(m, sc, a);
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
