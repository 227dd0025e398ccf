// Differentiable form of the cost and its adjoint (the smooth surrogate of Eq. path opt,
// arXiv 2503.14160 Sec. 4.1, used to polish candidates before trajectory optimisation):
//   J_s = sum_k |q(s_k) - q(s_{k-1})|^2 + w_c lambda_c sum_k sum_pairs beta softplus((m - sd)/beta)
//         + w_l sum_k sum_j (max(0, q - q_max)^2 + max(0, q_min - q)^2)
// q(s_k) is linear in the control points, so with r_k = dJ/dq(s_k) the gradient is
//   dJ/dP_g = sum_k [2 (q_k - q_{k-1}) (b_g(s_k) - b_g(s_{k-1})) + r_k^pen b_g(s_k)],
// r_k^pen chaining the softplus derivative through the signed-distance gradient and the
// kinematic Jacobian. One warp per candidate walks its checkpoints 32 at a time (one per
// lane), recomputing the forward pass (no tape); the per-control-point sums of a chunk are
// reduced in a fixed lane order into a per-warp accumulator, so results are deterministic.
#include "eval_common.cuh"

namespace cp {
namespace {

constexpr int kSmoothMaxThreads = 512;  // up to 16 warps per CTA, one candidate per warp
constexpr float kSmoothCut = 30.f;      // pairs with sd > m + 30 beta are skipped

struct SmoothArgs {
    const float4 *xi;
    int n, K, S, n_s, chunks;
    float4 q0, qd;
    const float4 *basis;     // [S][2] as in EvalArgs
    float margin, beta;      // softplus margin m and width beta
    float wc_lc, w_l;        // w_c lambda_c and w_l
    const double *gJ;        // [n] or nullptr (ones)
    double *J;               // [n] or nullptr
    float *dxi;              // [n][K][4] or nullptr
    int groups;              // warps per candidate (chunk groups); > 1 writes partials
    int chunks_per_group;
    float *part_g;           // [n groups][4K] when groups > 1
    double *part_J;          // [n groups] when groups > 1
    int *queue;              // the next unit to take (zeroed before the launch), or null: a
                             // fixed stride of units over the warps
};

__device__ __forceinline__ float softplus_f(float x)
{
    return x > 0.f ? x + log1pf(expf(-x)) : log1pf(expf(x));
}

__device__ __forceinline__ float logistic_f(float x)
{
    return x >= 0.f ? 1.f / (1.f + expf(-x)) : expf(x) / (1.f + expf(x));
}

// Softplus term of one pair and (GRAD) its contribution to d penalty / d centre.
template <bool GRAD>
__device__ __forceinline__ void pair_term(float sd, float3 grad_sdf, float m, float beta,
                                          float &pen, float3 &dp)
{
    const float x = (m - sd) / beta;
    pen = fmaf(beta, softplus_f(x), pen);
    if (GRAD) {
        const float w = -logistic_f(x);
        dp.x = fmaf(w, grad_sdf.x, dp.x);
        dp.y = fmaf(w, grad_sdf.y, dp.y);
        dp.z = fmaf(w, grad_sdf.z, dp.z);
    }
}

// Shared floats of one warp: the lane sums of the gradient ([32][4 control points][4]),
// the lanes' spans, the candidate's accumulator [K][4], and per sphere and lane h, z and the
// three components of d penalty / d centre.
__host__ __device__ inline int smooth_warp_floats(int K, int nsph) { return 32 * 16 + 32 + 4 * K + 5 * nsph * 32; }

template <int NSPH, bool GRAD>
__global__ void __launch_bounds__(kSmoothMaxThreads)
k_smooth(const ModelDev m, const SceneDev sc, const SmoothArgs a)
{
    extern __shared__ __align__(16) float4 smem[];
    float4 *s_filt = smem;                      // {cx, cy, W_s, reach}
    float4 *s_exact = s_filt + sc.n_cyl;        // {R, z_lo, z_hi, 0}
    float4 *s_bc = s_exact + sc.n_cyl;
    float4 *s_bh = s_bc + sc.n_box;
    float4 *s_basis = s_bh + sc.n_box;
    float4 *s_group = s_basis + 2 * a.S;
    float *s_warp = reinterpret_cast<float *>(s_group + n_groups(sc.n_cyl));
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per_warp = smooth_warp_floats(a.K, NSPH);
    float *s_contrib = s_warp + wib * per_warp;              // [32][4 control points][4]
    int *s_span = reinterpret_cast<int *>(s_contrib + 32 * 16);
    float *s_acc = s_contrib + 32 * 16 + 32;                 // [K][4]
    // per sphere s the lane's entries sit at [s * 32 + lane] (no bank conflicts)
    float *s_h = s_acc + 4 * a.K + lane;
    float *s_z = s_h + NSPH * 32, *s_dx = s_z + NSPH * 32, *s_dy = s_dx + NSPH * 32, *s_dz = s_dy + NSPH * 32;
    const double reach = (double)m.r_max + (double)a.margin + (double)kSmoothCut * a.beta;
    for (int i = threadIdx.x; i < sc.n_cyl; i += blockDim.x) {
        const float4 f = sc.cyl_filt[i], e = sc.cyl_exact[i];
        const double R = (double)e.x + reach;
        const double W = (double)f.x * f.x + (double)f.y * f.y - R * R;
        s_filt[i] = make_float4(f.x, f.y, (float)W, f.w);   // w: broad-phase reach
        s_exact[i] = e;
    }
    for (int i = threadIdx.x; i < n_groups(sc.n_cyl); i += blockDim.x) s_group[i] = sc.cyl_group[i];
    for (int i = threadIdx.x; i < sc.n_box; i += blockDim.x) {
        s_bc[i] = sc.box_c[i];
        s_bh[i] = sc.box_h[i];
    }
    for (int i = threadIdx.x; i < 2 * a.S; i += blockDim.x) s_basis[i] = a.basis[i];
    __syncthreads();

    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int n_warps = (int)((gridDim.x * blockDim.x) >> 5);
    // A unit is (candidate, group of consecutive chunks); with few candidates several
    // warps share one candidate and write partial sums that k_smooth_reduce combines. A warp
    // takes its next unit from the queue when it has one (candidates in contact cost more),
    // else the units go round the warps in a fixed stride.
    auto next_unit = [&](int u) {
        if (a.queue == nullptr) return u + n_warps;
        int v = 0;
        if (lane == 0) v = atomicAdd(a.queue, 1);
        return __shfl_sync(0xffffffffu, v, 0);
    };
    for (int unit = a.queue == nullptr ? warp : next_unit(0); unit < a.n * a.groups; unit = next_unit(unit)) {
        const int cand = unit / a.groups, group = unit - cand * a.groups;
        const int c_begin = group * a.chunks_per_group;
        const int c_end = min(a.chunks, c_begin + a.chunks_per_group);
        if (GRAD)
            for (int t = lane; t < 4 * a.K; t += 32) s_acc[t] = 0.f;
        double J = 0.0;
        const float4 *xi = a.xi + (size_t)cand * a.K;
        for (int chunk = c_begin; chunk < c_end; ++chunk) {
            const int k = chunk * 32 + lane + 1;
            const bool valid = k <= a.n_s;
            const int kc = valid ? k : a.n_s;
            const int span = (kc - 1) / a.S;
            const int mstep = kc - span * a.S;
            float4 P[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int g = span + 1 + i;
                P[i] = g < 4 ? a.q0 : (g >= a.K + 4 ? a.qd : __ldg(xi + (g - 4)));
            }
            const float4 bw = s_basis[2 * (mstep - 1)], dbw = s_basis[2 * (mstep - 1) + 1];
            const float4 q = combine4(bw, P[0], P[1], P[2], P[3]);
            const float4 dq = combine4(dbw, P[0], P[1], P[2], P[3]);
            const float jp = fmaf(dq.x, dq.x, fmaf(dq.y, dq.y, fmaf(dq.z, dq.z, dq.w * dq.w)));
            const float jl = limit_excess(q.x, m.q_min[0], m.q_max[0]) + limit_excess(q.y, m.q_min[1], m.q_max[1]) +
                             limit_excess(q.z, m.q_min[2], m.q_max[2]) + limit_excess(q.w, m.q_min[3], m.q_max[3]);

            float X[NSPH], Y[NSPH], Z[NSPH], T[NSPH], s1, c1;
            crane_fk_polar<NSPH, false>(m, q, X, Z, s1, c1);
            // broad phase of the chunk: the box of its spheres in the slew frame, dilated by
            // the softplus range m + cut beta beyond the obstacles' contact reach
            // spheres farther below or above every obstacle than the softplus range reaches
            // (r_max + m + cut beta) add nothing: left out of the box and of the filter
            const float extra = a.margin + kSmoothCut * a.beta;
            const float zreach = m.r_max + extra + kZGate;
            const float zlo = sc.z_lo_all - zreach, zhi = sc.z_hi_all + zreach;
            const UnitFrame fr = unit_frame_band<NSPH>(s1, c1, X, Z, zlo, zhi);
#pragma unroll
            for (int s = 0; s < NSPH; ++s) {
                const float h = X[s];
                s_h[s * 32] = h;
                s_z[s * 32] = Z[s];
                s_dx[s * 32] = 0.f;
                s_dy[s * 32] = 0.f;
                s_dz[s * 32] = 0.f;
                X[s] = __fmul_rn(c1, h);
                Y[s] = __fmul_rn(s1, h);
            }
            // Registers feed the unrolled filter; the shared per-lane entries (h, z, d pen / d
            // centre) feed the rolled exact path, so that one copy of the distance, gradient
            // and softplus code serves every sphere (unrolled it outgrows the instruction
            // cache) without per-thread local arrays.
#pragma unroll
            for (int s = 0; s < NSPH; ++s)
                T[s] = Z[s] > zlo && Z[s] < zhi ? kFilterMargin - fmaf(X[s], X[s], Y[s] * Y[s]) : -1e30f;
            float2 X2[NSPH / 2], Y2[NSPH / 2];
#pragma unroll
            for (int p = 0; p < NSPH / 2; ++p) {
                X2[p] = make_float2(-2.f * X[2 * p], -2.f * X[2 * p + 1]);
                Y2[p] = make_float2(-2.f * Y[2 * p], -2.f * Y[2 * p + 1]);
            }
            float pen = 0.f;
            const int n_grp = n_groups(sc.n_cyl);
            for (int gbase = 0; gbase < n_grp; gbase += 32) {
                uint32_t gmask = __ballot_sync(0xffffffffu, gbase + lane < n_grp &&
                                                                unit_near(fr, s_group[gbase + lane], extra));
                while (gmask) {
                    uint32_t gg = gmask;
                    const int slot = lane >> 3;
                    gg = slot >= 1 ? gg & (gg - 1) : gg;
                    gg = slot >= 2 ? gg & (gg - 1) : gg;
                    gg = slot >= 3 ? gg & (gg - 1) : gg;
                    const int oc = gg ? (gbase + __ffs(gg) - 1) * kGroup + (lane & (kGroup - 1)) : sc.n_cyl;
#pragma unroll
                    for (int k = 0; k < 4; ++k) gmask &= gmask - 1;
                    uint32_t omask = __ballot_sync(0xffffffffu, oc < sc.n_cyl && unit_near(fr, s_filt[oc], extra));
                    while (omask) {
                const int o = __shfl_sync(0xffffffffu, oc, __ffs(omask) - 1);
                omask &= omask - 1;
                const float4 f = s_filt[o];
                float2 g[NSPH / 2];
#pragma unroll
                for (int p = 0; p < NSPH / 2; ++p)
                    g[p] = __ffma2_rn(X2[p], make_float2(f.x, f.x),
                                      __ffma2_rn(Y2[p], make_float2(f.y, f.y), make_float2(f.z, f.z)));
                if (any_below<NSPH>(g, T)) {
                    const float4 e = s_exact[o];
#pragma unroll 1
                    for (int s = 0; s < m.n_spheres; ++s) {
                        const float h = s_h[s * 32];
                        const float cx = __fmul_rn(c1, h), cy = __fmul_rn(s1, h);
                        const float cw = kFilterMargin - fmaf(cx, cx, cy * cy);
                        const float cz = s_z[s * 32];
                        if (fmaf(-2.f * cx, f.x, fmaf(-2.f * cy, f.y, f.z)) < cw && cz > e.y - zreach &&
                            cz < e.z + zreach) {
                            const float sd = sdf_cylinder(cx, cy, cz, f.x, f.y, e) - m.sph[s].radius;
                            const float3 gr = GRAD ? sdf_cylinder_grad(cx, cy, cz, f.x, f.y, e)
                                                   : make_float3(0.f, 0.f, 0.f);
                            float3 d = make_float3(0.f, 0.f, 0.f);
                            if (GRAD) d = make_float3(s_dx[s * 32], s_dy[s * 32], s_dz[s * 32]);
                            pair_term<GRAD>(sd, gr, a.margin, a.beta, pen, d);
                            if (GRAD) {
                                s_dx[s * 32] = d.x;
                                s_dy[s * 32] = d.y;
                                s_dz[s * 32] = d.z;
                            }
                        }
                    }
                }
                    }
                }
            }
            for (int bbase = 0; bbase < sc.n_box; bbase += 32) {
                uint32_t bmask = __ballot_sync(0xffffffffu, bbase + lane < sc.n_box &&
                                                                unit_near(fr, s_bc[bbase + lane], extra));
                while (bmask) {
                const int o = bbase + __ffs(bmask) - 1;
                bmask &= bmask - 1;
                const float4 cb = s_bc[o], hb = s_bh[o];
#pragma unroll 1
                for (int s = 0; s < m.n_spheres; ++s) {
                    const float h = s_h[s * 32];
                    const float cx = __fmul_rn(c1, h), cy = __fmul_rn(s1, h), cz = s_z[s * 32];
                    const float sd = sdf_box(cx, cy, cz, cb, hb) - m.sph[s].radius;
                    if (sd < a.margin + kSmoothCut * a.beta) {
                        const float3 gr = GRAD ? sdf_box_grad(cx, cy, cz, cb, hb)
                                               : make_float3(0.f, 0.f, 0.f);
                        float3 d = make_float3(0.f, 0.f, 0.f);
                        if (GRAD) d = make_float3(s_dx[s * 32], s_dy[s * 32], s_dz[s * 32]);
                        pair_term<GRAD>(sd, gr, a.margin, a.beta, pen, d);
                        if (GRAD) {
                            s_dx[s * 32] = d.x;
                            s_dy[s * 32] = d.y;
                            s_dz[s * 32] = d.z;
                        }
                    }
                }
                }
            }

            float v = valid ? jp + a.wc_lc * pen + a.w_l * jl : 0.f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            J += (double)v;   // every lane holds the same sum; lane 0 writes it

            if (GRAD) {
                // r = d(terms at s_k)/dq: penalty through the kinematic Jacobian, and limits
                float s1, c1, s2, c2, s23, c23;
                sincosf(q.x, &s1, &c1);
                sincosf(q.y, &s2, &c2);
                sincosf(q.y + q.z, &s23, &c23);
                float r0 = 0.f, r1 = 0.f, r2 = 0.f, r3 = 0.f;
#pragma unroll
                for (int s = 0; s < NSPH; ++s) {
                    const SphereLin sp = m.sph[s];
                    const float L = fmaf(sp.gamma, q.w, sp.beta);
                    const float u = fmaf(sp.alpha, s2, L * s23);     // d h / d q2 = -u
                    const float hz = fmaf(sp.alpha, c2, L * c23);    // horizontal reach
                    const float3 d = make_float3(s_dx[s * 32], s_dy[s * 32], s_dz[s * 32]);
                    r0 += fmaf(-d.x, Y[s], d.y * X[s]);
                    r1 += fmaf(d.x, -c1 * u, fmaf(d.y, -s1 * u, d.z * hz));
                    r2 += L * fmaf(d.x, -c1 * s23, fmaf(d.y, -s1 * s23, d.z * c23));
                    r3 += sp.gamma * fmaf(d.x, c1 * c23, fmaf(d.y, s1 * c23, d.z * s23));
                }
                const float4 lim2 = make_float4(
                    2.f * (fmaxf(0.f, q.x - m.q_max[0]) - fmaxf(0.f, m.q_min[0] - q.x)),
                    2.f * (fmaxf(0.f, q.y - m.q_max[1]) - fmaxf(0.f, m.q_min[1] - q.y)),
                    2.f * (fmaxf(0.f, q.z - m.q_max[2]) - fmaxf(0.f, m.q_min[2] - q.z)),
                    2.f * (fmaxf(0.f, q.w - m.q_max[3]) - fmaxf(0.f, m.q_min[3] - q.w)));
                const float4 r = make_float4(fmaf(a.wc_lc, r0, a.w_l * lim2.x), fmaf(a.wc_lc, r1, a.w_l * lim2.y),
                                             fmaf(a.wc_lc, r2, a.w_l * lim2.z), fmaf(a.wc_lc, r3, a.w_l * lim2.w));
                // contribution to control point span+1+i: 2 dq db_i + r b_i
                const float bi[4] = {bw.x, bw.y, bw.z, bw.w}, dbi[4] = {dbw.x, dbw.y, dbw.z, dbw.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float wd = valid ? 2.f * dbi[i] : 0.f, wb = valid ? bi[i] : 0.f;
                    s_contrib[lane * 16 + 4 * i + 0] = fmaf(wd, dq.x, wb * r.x);
                    s_contrib[lane * 16 + 4 * i + 1] = fmaf(wd, dq.y, wb * r.y);
                    s_contrib[lane * 16 + 4 * i + 2] = fmaf(wd, dq.z, wb * r.z);
                    s_contrib[lane * 16 + 4 * i + 3] = fmaf(wd, dq.w, wb * r.w);
                }
                s_span[lane] = span;
                __syncwarp();
                // fixed-order sums over the lanes for every (control point, joint) touched
                const int g_lo = s_span[0] + 1, g_hi = s_span[31] + 4;
                for (int t = lane; t < 4 * (g_hi - g_lo + 1); t += 32) {
                    const int G = g_lo + (t >> 2), j = t & 3;
                    float acc = 0.f;
                    for (int l = 0; l < 32; ++l) {
                        const int i = G - s_span[l] - 1;
                        if (i >= 0 && i < 4) acc += s_contrib[l * 16 + 4 * i + j];
                    }
                    if (G >= 4 && G < a.K + 4) s_acc[(G - 4) * 4 + j] += acc;
                }
                __syncwarp();
            }
        }
        if (a.groups == 1) {
            if (lane == 0 && a.J != nullptr) a.J[cand] = J;
            if (GRAD) {
                const float gj = a.gJ != nullptr ? (float)a.gJ[cand] : 1.f;
                for (int t = lane; t < 4 * a.K; t += 32) a.dxi[(size_t)cand * 4 * a.K + t] = gj * s_acc[t];
            }
        } else {
            if (lane == 0) a.part_J[unit] = J;
            if (GRAD)
                for (int t = lane; t < 4 * a.K; t += 32) a.part_g[(size_t)unit * 4 * a.K + t] = s_acc[t];
        }
        __syncwarp();
    }
}

// Sums the groups' partials of each candidate in group order (one warp per candidate).
__global__ void k_smooth_reduce(int n, int groups, int K, const double *part_J, const float *part_g,
                                const double *gJ, double *J, float *dxi)
{
    const int cand = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (cand >= n) return;
    if (lane == 0 && J != nullptr) {
        double acc = 0.0;
        for (int g = 0; g < groups; ++g) acc += part_J[(size_t)cand * groups + g];
        J[cand] = acc;
    }
    if (dxi == nullptr) return;
    const float gj = gJ != nullptr ? (float)gJ[cand] : 1.f;
    for (int t = lane; t < 4 * K; t += 32) {
        float acc = 0.f;
        for (int g = 0; g < groups; ++g) acc += part_g[((size_t)cand * groups + g) * 4 * K + t];
        dxi[(size_t)cand * 4 * K + t] = gj * acc;
    }
}

__global__ void k_axpy(float *x, const float *y, float alpha, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = fmaf(-alpha, y[i], x[i]);
}

size_t smooth_smem(int n_cyl, int n_box, int S, int K, int nsph, int threads)
{
    return sizeof(float4) * (2 * (size_t)n_cyl + 2 * (size_t)n_box + 2 * (size_t)S +
                             (size_t)n_groups(n_cyl)) +
           sizeof(float) * (size_t)(threads / 32) * (size_t)smooth_warp_floats(K, nsph);
}

template <bool GRAD>
int launch_smooth_t(const ModelDev &m, const SceneDev &sc, const SmoothArgs &a, int num_sms,
                    cudaStream_t st)
{
    const int nsph = m.n_spheres == 12 ? 12 : 16;
    int dev = 0, optin = 0;
    CP_CUDA(cudaGetDevice(&dev));
    CP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    // the largest CTA (512, 256 or 128 threads) whose shared memory fits: the obstacle
    // tables are staged once per CTA, so larger CTAs leave room for more warps per SM
    int threads = kSmoothMaxThreads;
    while (threads > 128 && smooth_smem(sc.n_cyl, sc.n_box, a.S, a.K, nsph, threads) > (size_t)optin)
        threads /= 2;
    const size_t smem = smooth_smem(sc.n_cyl, sc.n_box, a.S, a.K, nsph, threads);
    auto kern = m.n_spheres == 12 ? k_smooth<12, GRAD> : k_smooth<16, GRAD>;
    CP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    const int units = a.n * a.groups;
    int grid = (units + threads / 32 - 1) / (threads / 32);
    if (grid > num_sms * per_sm) grid = num_sms * per_sm;
    if (a.queue != nullptr) CP_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(int), st));
    kern<<<grid, threads, smem, st>>>(m, sc, a);
    CP_LAUNCHED("k_smooth");
    if (a.groups > 1) {
        k_smooth_reduce<<<(a.n * 32 + 255) / 256, 256, 0, st>>>(a.n, a.groups, a.K, a.part_J, a.part_g,
                                                                a.gJ, a.J, a.dxi);
        CP_LAUNCHED("k_smooth_reduce");
    }
    return CP_OK;
}

}  // namespace

// Shared memory of the smallest launch (128 threads, 16 spheres): the scene fits if this does.
size_t smooth_smem_bytes(int n_cyl, int n_box, int S, int K) { return smooth_smem(n_cyl, n_box, S, K, 16, 128); }

// Chunk groups per candidate: enough units for about 32 warps per SM when candidates are
// few, at most the number of chunks; the partial buffers hold smooth_partial_units() units.
int smooth_groups(int n, int chunks, int num_sms)
{
    const int target = 32 * num_sms;
    if (n <= 0 || n >= target) return 1;
    int g = (target + n - 1) / n;
    return g < chunks ? g : chunks;
}

int64_t smooth_partial_units(int num_sms) { return 2 * 32 * (int64_t)num_sms; }

int launch_smooth(const ModelDev &m, const SceneDev &sc, const float *xi, int n, int K, int S,
                  float4 q0, float4 qd, const float4 *basis, double margin, double beta,
                  double wc_lc, double w_l, const double *gJ, double *J, float *dxi, float *part_g,
                  double *part_J, int *queue, int num_sms, cudaStream_t st)
{
    if (n == 0) return CP_OK;
    SmoothArgs a{};
    a.queue = queue;
    a.xi = (const float4 *)xi;
    a.n = n;
    a.K = K;
    a.S = S;
    a.n_s = (K + 3) * S;
    a.chunks = (a.n_s + 31) / 32;
    a.q0 = q0;
    a.qd = qd;
    a.basis = basis;
    a.margin = (float)margin;
    a.beta = (float)beta;
    a.wc_lc = (float)wc_lc;
    a.w_l = (float)w_l;
    a.gJ = gJ;
    a.J = J;
    a.dxi = dxi;
    a.groups = smooth_groups(n, a.chunks, num_sms);
    a.chunks_per_group = (a.chunks + a.groups - 1) / a.groups;
    a.groups = (a.chunks + a.chunks_per_group - 1) / a.chunks_per_group;   // no empty group
    a.part_g = part_g;
    a.part_J = part_J;
    return dxi != nullptr ? launch_smooth_t<true>(m, sc, a, num_sms, st)
                          : launch_smooth_t<false>(m, sc, a, num_sms, st);
}

int launch_axpy(float *x, const float *y, double alpha, int64_t n, cudaStream_t st)
{
    if (n == 0) return CP_OK;
    k_axpy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, (float)alpha, n);
    CP_LAUNCHED("k_axpy");
    return CP_OK;
}

}  // namespace cp
