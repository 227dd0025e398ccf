// Algorithm 1 step (2) on the GPU: for every candidate path, the cubic B-spline at the
// n_s checkpoints, the crane kinematics, the link-sphere vs obstacle signed distance and
// the three cost terms of Eq. path opt (arXiv 2503.14160, Sec. 4.1; d(q) of Sec. 3.1).
//
// Work decomposition: a work unit is (candidate, chunk of 32 consecutive checkpoints), one
// checkpoint per lane; a warp takes one work item (candidate, G consecutive units) at a time,
// stages the candidate's control points in its slice of shared memory, and adds the units'
// FP32 lane sums (warp shuffles) into FP64 sums in unit order. All obstacles are staged once
// per CTA in shared memory by bulk copies (TMA, no multicast) completing on an mbarrier with
// a bounded wait. Per checkpoint and link sphere the obstacle loop is a 2-FMA power test
// against every cylinder; only pairs that pass it (sphere within reach of the cylinder) take
// the exact capped-cylinder distance. A second kernel adds each candidate's item sums in a
// fixed order in FP64.
#include "eval_common.cuh"
#include "item_queue.cuh"

namespace cp {
namespace {

constexpr int kEvalThreads = 256;
#ifndef CP_EVAL_MIN_BLOCKS
#define CP_EVAL_MIN_BLOCKS 3   // CTAs of 8 warps resident per SM (3: at most 85 registers)
#endif
constexpr int kEvalMinBlocks = CP_EVAL_MIN_BLOCKS;
#ifndef CP_EVAL_BROAD_MIN_BLOCKS
#define CP_EVAL_BROAD_MIN_BLOCKS 3   // broad-phase form: at most 80 registers
#endif
constexpr int kEvalBroadMinBlocks = CP_EVAL_BROAD_MIN_BLOCKS;
constexpr int kObstaclesPerBranch = 2;   // obstacles tested between two branches
constexpr long long kStagingWaitCycles = 2000000000ll;   // about one second at 2 GHz
constexpr int kCtrlSlots = CP_MAX_WAYPOINTS + 8;         // control points per warp, float4

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Bulk copy (TMA, no multicast) of `bytes` from global memory into this CTA's shared
// memory; both addresses 16-byte aligned, bytes a multiple of 16. Completes on `bar`.
__device__ __forceinline__ void bulk_copy_to_smem(void *dst, const void *src, uint32_t bytes,
                                                  uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbarrier_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Stages the obstacle records, box records, spline table and cylinder groups into shared memory with bulk
// copies completing on one mbarrier. Every thread waits at most kStagingWaitCycles; when
// the wait runs out in any thread the CTA records DEV_ERR_TIMEOUT and returns false (a
// uniform decision). `withhold` issues no copy, so that the wait runs out on purpose (the
// test of this path); nothing is then in flight when the CTA leaves.
__device__ __noinline__ bool stage_bulk(uint64_t *bar, float4 *s_filt, float4 *s_exact, float4 *s_bc,
                           float4 *s_bh, float4 *s_basis, float4 *s_group, const SceneDev &sc,
                           const EvalArgs &a)
{
    const uint32_t b_cyl = 16u * (uint32_t)sc.n_cyl, b_box = 16u * (uint32_t)sc.n_box;
    const uint32_t b_basis = 32u * (uint32_t)a.S, b_group = 16u * (uint32_t)n_groups(sc.n_cyl);
    const uint32_t total = 2 * b_cyl + 2 * b_box + b_basis + b_group;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(smem_u32(bar)), "r"(total) : "memory");
        if (!a.withhold_staging) {
            if (b_cyl) {
                bulk_copy_to_smem(s_filt, sc.cyl_filt, b_cyl, bar);
                bulk_copy_to_smem(s_exact, sc.cyl_exact, b_cyl, bar);
                bulk_copy_to_smem(s_group, sc.cyl_group, b_group, bar);
            }
            if (b_box) {
                bulk_copy_to_smem(s_bc, sc.box_c, b_box, bar);
                bulk_copy_to_smem(s_bh, sc.box_h, b_box, bar);
            }
            bulk_copy_to_smem(s_basis, a.basis, b_basis, bar);
        }
    }
    const long long t0 = clock64();
    bool done = mbarrier_try_wait(bar, 0);
    while (!done && clock64() - t0 < kStagingWaitCycles) done = mbarrier_try_wait(bar, 0);
    if (__syncthreads_or(!done)) {
        if (threadIdx.x == 0 && a.status != nullptr) atomicOr(a.status, DEV_ERR_TIMEOUT);
        return false;
    }
    return true;
}

// Exact signed distance of every sphere whose filter test and vertical gate pass against
// one cylinder (f = {cx, cy, W}, e = {R, z_lo, z_hi}); +inf when none passes.
template <int NSPH>
__device__ __forceinline__ float exact_cylinders(const ModelDev &m, const float *X, const float *Y,
                                              const float *Z, const float *T, float4 f, float4 e)
{
    float d = CUDART_INF_F;
    const float zlo = e.y - m.r_max - kZGate, zhi = e.z + m.r_max + kZGate;
#pragma unroll
    for (int s = 0; s < NSPH; ++s) {
        const float g = fmaf(X[s], f.x, fmaf(Y[s], f.y, f.z));
        if (g < T[s] && Z[s] > zlo && Z[s] < zhi)
            d = fminf(d, sdf_cylinder(-0.5f * X[s], -0.5f * Y[s], Z[s], f.x, f.y, e) - m.sph[s].radius);
    }
    return d;
}

// Exact distance of every sphere whose polar filter passes against one cylinder: with the
// obstacle centre at p along the lane's plane and q across it, sphere s passes when
// (h_s - p)^2 < (R + r_max)^2 + margin - q^2 = rhs and its centre is within the cylinder's
// height range widened by r_max and the gate. The distance itself is taken from the
// Cartesian centre (c1 h, s1 h, z), rounded products (no contraction into the distance's
// differences), the same values the exhaustive form uses.
template <int NSPH>
__device__ __forceinline__ float exact_polar(const ModelDev &m, const float *H, const float *Z,
                                             float c1, float s1, float p, float rhs, float4 f,
                                             float4 e)
{
    float d = CUDART_INF_F;
    const float zlo = e.y - m.r_max - kZGate, zhi = e.z + m.r_max + kZGate;
#pragma unroll
    for (int s = 0; s < NSPH; ++s) {
        const float dh = H[s] - p;
        if (fmaf(dh, dh, -rhs) < 0.f && Z[s] > zlo && Z[s] < zhi)
            d = fminf(d, sdf_cylinder(__fmul_rn(c1, H[s]), __fmul_rn(s1, H[s]), Z[s], f.x, f.y, e) -
                             m.sph[s].radius);
    }
    return d;
}

// A surviving cylinder (filter record f = {cx, cy, W, reach}, exact record e = {R, z_lo,
// z_hi, (R + r_max)^2 + margin}) against the unit's spheres at one lane: its centre at p
// along the lane's plane and q across it; sphere s passes the polar filter when
// (h_s - p)^2 < e.w - q^2 (two packed FP32x2 operations per sphere pair, H2 holding the
// in-band h and 1e30 for the others), and the passing spheres take the exact distance.
template <int NSPH>
__device__ __forceinline__ float survivor_cylinder(const ModelDev &m, const float *H, const float *Z,
                                                   const float2 *H2, float c1, float s1, float4 f, float4 e,
                                                   const float *zero)
{
    const float p = fmaf(c1, f.x, s1 * f.y);
    const float q = fmaf(c1, f.y, -(s1 * f.x));
    const float rhs = fmaf(-q, q, e.w);
    const float2 mp2 = make_float2(-p, -p), mr2 = make_float2(-rhs, -rhs);
    float2 t[NSPH / 2];
#pragma unroll
    for (int k = 0; k < NSPH / 2; ++k) {
        const float2 dh = __fadd2_rn(H2[k], mp2);
        t[k] = __ffma2_rn(dh, dh, mr2);
    }
    return any_negative<NSPH>(t) ? exact_polar<NSPH>(m, H, Z, c1, s1, p, rhs, f, e) : CUDART_INF_F;
}

// A surviving box (centre c, half extent hb) against every sphere of the lane.
template <int NSPH>
__device__ __forceinline__ float survivor_box(const ModelDev &m, const float *H, const float *Z, float c1,
                                              float s1, float4 c, float4 hb)
{
    float d = CUDART_INF_F;
#pragma unroll
    for (int s = 0; s < NSPH; ++s)
        d = fminf(d, sdf_box(__fmul_rn(c1, H[s]), __fmul_rn(s1, H[s]), Z[s], c, hb) - m.sph[s].radius);
    return d;
}

// The evaluation with the broad phase (the default form). Per unit: the checkpoints and
// the kinematics in polar form, the unit box, then rounds of 32 obstacles: each lane tests
// one obstacle against the box, and the warp takes the survivors one by one (a uniform
// loop) through the per-sphere polar filter, two packed FP32x2 operations per sphere pair,
// and the exact distance where it passes. Boxes take the same broad phase and then the
// exact distance for every sphere. Its distances are those of the exhaustive form for
// every pair that can be in contact, so both forms give the same results bit for bit.
template <int NSPH>
__global__ void __launch_bounds__(kEvalThreads, kEvalBroadMinBlocks)
k_eval_broad(const ModelDev m, const SceneDev sc, const EvalArgs a)
{
    extern __shared__ __align__(16) float4 smem[];
    float4 *s_filt = smem;
    float4 *s_exact = s_filt + sc.n_cyl;
    float4 *s_bc = s_exact + sc.n_cyl;
    float4 *s_bh = s_bc + sc.n_box;
    float4 *s_basis = s_bh + sc.n_box;
    float4 *s_group = s_basis + 2 * a.S;
    float4 *s_ctrl = s_group + n_groups(sc.n_cyl) + (threadIdx.x >> 5) * kCtrlSlots;
    __shared__ __align__(8) uint64_t staging_bar;
    if (!stage_bulk(&staging_bar, s_filt, s_exact, s_bc, s_bh, s_basis, s_group, sc, a)) return;

    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int n_warps = (int)((gridDim.x * blockDim.x) >> 5);
    const int items = a.n * a.P;
    uint32_t tested = 0;   // broad-phase survivors of this warp's units
    const float zero[NSPH] = {};
    const float zlo = sc.z_lo_all - m.r_max - kZGate, zhi = sc.z_hi_all + m.r_max + kZGate;

    for (int it = queue_first(a, warp, lane); it < items; it = queue_next(a, it, n_warps, lane)) {
        const ItemRange ir = item_range(a, it);
        stage_controls(s_ctrl, a, ir.cand, lane);
        double acc = 0.0;
        uint32_t count = 0;
        for (int chunk = ir.c0; chunk < ir.c1; ++chunk) {
            const Checkpoint c = checkpoint_at(m, a, s_basis, s_ctrl, chunk, lane);
            float H[NSPH], Z[NSPH], s1, c1;
            crane_fk_polar<NSPH>(m, c.q, H, Z, s1, c1);
            // Spheres above or below every obstacle by more than r_max (the vertical gate over
            // the whole scene) can penetrate nothing: they leave the unit box, and their packed
            // h is pushed far away so that no polar filter passes them.
            const UnitFrame fr = unit_frame_band<NSPH>(s1, c1, H, Z, zlo, zhi);
            float2 H2[NSPH / 2];
#pragma unroll
            for (int q = 0; q < NSPH / 2; ++q)
                H2[q] = make_float2(Z[2 * q] > zlo && Z[2 * q] < zhi ? H[2 * q] : 1e30f,
                                    Z[2 * q + 1] > zlo && Z[2 * q + 1] < zhi ? H[2 * q + 1] : 1e30f);

            float dmin = CUDART_INF_F;
            const int n_grp = n_groups(sc.n_cyl);
            for (int gbase = 0; gbase < n_grp; gbase += 32) {
                // groups whose circle meets the unit box, then their members four groups at a
                // time: lane l takes member l % 8 of the (l / 8)-th remaining group
                uint32_t gmask = __ballot_sync(0xffffffffu, gbase + lane < n_grp && unit_near(fr, s_group[gbase + lane]));
                while (gmask) {
                    uint32_t g = gmask;
                    const int slot = lane >> 3;
                    g = slot >= 1 ? g & (g - 1) : g;
                    g = slot >= 2 ? g & (g - 1) : g;
                    g = slot >= 3 ? g & (g - 1) : g;
                    const int o = g ? (gbase + __ffs(g) - 1) * kGroup + (lane & (kGroup - 1)) : sc.n_cyl;
#pragma unroll
                    for (int k = 0; k < 4; ++k) gmask &= gmask - 1;
                    uint32_t mask = __ballot_sync(0xffffffffu, o < sc.n_cyl && unit_near(fr, s_filt[o]));
                    tested += __popc(mask);
                    while (mask) {
                        const int ob = __shfl_sync(0xffffffffu, o, __ffs(mask) - 1);
                        mask &= mask - 1;
                        dmin = fminf(dmin, survivor_cylinder<NSPH>(m, H, Z, H2, c1, s1, s_filt[ob], s_exact[ob], zero));
                    }
                }
            }
            for (int base = 0; base < sc.n_box; base += 32) {
                const int o = base + lane;
                uint32_t mask = __ballot_sync(0xffffffffu, o < sc.n_box && unit_near(fr, s_bc[o]));
                tested += __popc(mask);
                while (mask) {
                    const int ob = base + __ffs(mask) - 1;
                    mask &= mask - 1;
                    dmin = fminf(dmin, survivor_box<NSPH>(m, H, Z, c1, s1, s_bc[ob], s_bh[ob]));
                }
            }
            unit_accumulate(a, c, dmin, ir.cand, chunk, lane, acc, count);
        }
        item_flush(a, it, acc, count, lane);
    }
    if (a.work != nullptr && lane == 0 && tested != 0) atomicAdd(a.work, (unsigned long long)tested);
}

// The exhaustive evaluation: every sphere against every obstacle.
template <int NSPH>
__global__ void __launch_bounds__(kEvalThreads, kEvalMinBlocks)
k_eval(const ModelDev m, const SceneDev sc, const EvalArgs a)
{
    // Shared memory: per cylinder the filter record {cx, cy, W, reach} and the exact record
    // {R, z_lo, z_hi, bound}; per box its centre and half extent; the spline basis table.
    extern __shared__ __align__(16) float4 smem[];
    float4 *s_filt = smem;
    float4 *s_exact = s_filt + sc.n_cyl;
    float4 *s_bc = s_exact + sc.n_cyl;
    float4 *s_bh = s_bc + sc.n_box;
    float4 *s_basis = s_bh + sc.n_box;
    float4 *s_group = s_basis + 2 * a.S;
    __shared__ __align__(8) uint64_t staging_bar;
    if (!stage_bulk(&staging_bar, s_filt, s_exact, s_bc, s_bh, s_basis, s_group, sc, a)) return;

    float4 *s_ctrl = s_group + n_groups(sc.n_cyl) + (threadIdx.x >> 5) * kCtrlSlots;
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int n_warps = (int)((gridDim.x * blockDim.x) >> 5);
    const int items = a.n * a.P;

    for (int it = queue_first(a, warp, lane); it < items; it = queue_next(a, it, n_warps, lane)) {
      const ItemRange ir = item_range(a, it);
      stage_controls(s_ctrl, a, ir.cand, lane);
      double acc = 0.0;
      uint32_t count = 0;
      for (int chunk = ir.c0; chunk < ir.c1; ++chunk) {
        const Checkpoint c = checkpoint_at(m, a, s_basis, s_ctrl, chunk, lane);

        // Sphere centres; per sphere the filter threshold T = margin - (x^2 + y^2) and the
        // scaled coordinates (-2x, -2y), kept in pairs for packed FP32x2 FMAs.
        float X[NSPH], Y[NSPH], Z[NSPH], T[NSPH];
        crane_fk<NSPH>(m, c.q, X, Y, Z);
#pragma unroll
        for (int s = 0; s < NSPH; ++s) {
            T[s] = kFilterMargin - fmaf(X[s], X[s], Y[s] * Y[s]);
            X[s] *= -2.f;   // exact; -0.5 X recovers x
            Y[s] *= -2.f;
        }
        float2 X2[NSPH / 2], Y2[NSPH / 2];
#pragma unroll
        for (int p = 0; p < NSPH / 2; ++p) {
            X2[p] = make_float2(X[2 * p], X[2 * p + 1]);
            Y2[p] = make_float2(Y[2 * p], Y[2 * p + 1]);
        }

        float dmin = CUDART_INF_F;
        // Two obstacles per step: 2 x NSPH power tests rho^2 - (R + r_max)^2 < margin in
        // expanded form (-2x cx - 2y cy + W vs. margin - x^2 - y^2), two packed FMAs per
        // sphere pair; the hit predicates accumulate without branches. Only when a test
        // passes does the lane take the exact capped-cylinder distance.
        constexpr int OB = kObstaclesPerBranch;
        int o = 0;
        for (; o + OB <= sc.n_cyl; o += OB) {
            float4 fo[OB];      // {cx, cy, W, 0} of each obstacle, for the exact path
            uint32_t hit[OB];
            uint32_t any = 0;
#pragma unroll
            for (int b = 0; b < OB; ++b) {
                const float4 f = s_filt[o + b];
                const float2 cx2 = make_float2(f.x, f.x), cy2 = make_float2(f.y, f.y);
                const float2 w2 = make_float2(f.z, f.z);
                fo[b] = f;
                float2 g[NSPH / 2];
#pragma unroll
                for (int p = 0; p < NSPH / 2; ++p) g[p] = __ffma2_rn(X2[p], cx2, __ffma2_rn(Y2[p], cy2, w2));
                hit[b] = any_below<NSPH>(g, T);
                any |= hit[b];
            }
            if (any) {
#pragma unroll
                for (int b = 0; b < OB; ++b)
                    if (hit[b]) dmin = fminf(dmin, exact_cylinders<NSPH>(m, X, Y, Z, T, fo[b], s_exact[o + b]));
            }
        }
        for (; o < sc.n_cyl; ++o) {
            const float4 f0 = s_filt[o];
            bool hit0 = false;
#pragma unroll
            for (int s = 0; s < NSPH; ++s) hit0 |= fmaf(X[s], f0.x, fmaf(Y[s], f0.y, f0.z)) < T[s];
            if (hit0) dmin = fminf(dmin, exact_cylinders<NSPH>(m, X, Y, Z, T, f0, s_exact[o]));
        }
        for (int o = 0; o < sc.n_box; ++o) {
            const float4 c = s_bc[o], h = s_bh[o];
#pragma unroll
            for (int s = 0; s < NSPH; ++s)
                dmin = fminf(dmin, sdf_box(-0.5f * X[s], -0.5f * Y[s], Z[s], c, h) -
                                       m.sph[s].radius);
        }

        unit_accumulate(a, c, dmin, ir.cand, chunk, lane, acc, count);
      }
      item_flush(a, it, acc, count, lane);
    }
}


// d(q) for single configurations: every pair, exact distances (no filter).
template <int NSPH>
__global__ void k_signed_distance(const ModelDev m, const SceneDev sc, const float *q, int n,
                                  float *d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 qi = make_float4(q[4 * i], q[4 * i + 1], q[4 * i + 2], q[4 * i + 3]);
    float x[NSPH], y[NSPH], z[NSPH];
    crane_fk<NSPH>(m, qi, x, y, z);
    float dmin = CUDART_INF_F;
    for (int o = 0; o < sc.n_cyl; ++o) {
        const float4 f = sc.cyl_filt[o], e = sc.cyl_exact[o];
#pragma unroll
        for (int s = 0; s < NSPH; ++s)
            dmin = fminf(dmin, sdf_cylinder(x[s], y[s], z[s], f.x, f.y, e) - m.sph[s].radius);
    }
    for (int o = 0; o < sc.n_box; ++o) {
        const float4 c = sc.box_c[o], h = sc.box_h[o];
#pragma unroll
        for (int s = 0; s < NSPH; ++s)
            dmin = fminf(dmin, sdf_box(x[s], y[s], z[s], c, h) - m.sph[s].radius);
    }
    d[i] = dmin;
}

template <typename F>
int eval_grid(F *kernel, size_t smem, int num_sms, int units, int ctas_per_sm)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kEvalThreads, smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    const int warps_per_block = kEvalThreads / 32;
    const int needed = (units + warps_per_block - 1) / warps_per_block;
    int grid = num_sms * per_sm;
    if (grid > needed) grid = needed;
    return grid < 1 ? 1 : grid;
}

}  // namespace

size_t eval_smem_bytes(int n_cyl, int n_box, int S)
{
    return sizeof(float4) * (2 * (size_t)n_cyl + 2 * (size_t)n_box + 2 * (size_t)S +
                             (size_t)n_groups(n_cyl) + (size_t)(kEvalThreads / 32) * kCtrlSlots);
}

template <typename F>
int raise_smem(F *fn, size_t smem_bytes)
{
    cudaFuncAttributes at{};
    CP_CUDA(cudaFuncGetAttributes(&at, fn));
    if ((size_t)at.maxDynamicSharedSizeBytes < smem_bytes)
        CP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes));
    return CP_OK;
}

int eval_configure(size_t smem_bytes) { return eval_ensure_smem(smem_bytes); }

// Raise (never lower) the dynamic shared-memory limit of the evaluation kernels.
int eval_ensure_smem(size_t smem_bytes)
{
    int rc;
    if ((rc = raise_smem(k_eval<12>, smem_bytes)) != CP_OK) return rc;
    if ((rc = raise_smem(k_eval<16>, smem_bytes)) != CP_OK) return rc;
    if ((rc = raise_smem(k_eval_broad<12>, smem_bytes)) != CP_OK) return rc;
    return raise_smem(k_eval_broad<16>, smem_bytes);
}

int launch_eval(const ModelDev &m, const SceneDev &sc, const EvalArgs &a, int num_sms,
                cudaStream_t st)
{
    const int units = a.n * a.P;   // work items
    if (units == 0) return CP_OK;
    const size_t smem = eval_smem_bytes(sc.n_cyl, sc.n_box, a.S);
    const int cpsm = a.ctas_per_sm;
    if (a.queue != nullptr) CP_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(int), st));
    if (m.n_spheres == 12) {
        if (a.broadphase)
            k_eval_broad<12><<<eval_grid(k_eval_broad<12>, smem, num_sms, units, cpsm), kEvalThreads, smem, st>>>(m, sc, a);
        else
            k_eval<12><<<eval_grid(k_eval<12>, smem, num_sms, units, cpsm), kEvalThreads, smem, st>>>(m, sc, a);
    } else {
        if (a.broadphase)
            k_eval_broad<16><<<eval_grid(k_eval_broad<16>, smem, num_sms, units, cpsm), kEvalThreads, smem, st>>>(m, sc, a);
        else
            k_eval<16><<<eval_grid(k_eval<16>, smem, num_sms, units, cpsm), kEvalThreads, smem, st>>>(m, sc, a);
    }
    CP_LAUNCHED("k_eval");
    return CP_OK;
}

int launch_signed_distance(const ModelDev &m, const SceneDev &sc, const float *q, int n,
                           float *d, cudaStream_t st)
{
    if (n == 0) return CP_OK;
    const int threads = 128;
    const int blocks = (n + threads - 1) / threads;
    if (m.n_spheres == 12)
        k_signed_distance<12><<<blocks, threads, 0, st>>>(m, sc, q, n, d);
    else
        k_signed_distance<16><<<blocks, threads, 0, st>>>(m, sc, q, n, d);
    CP_LAUNCHED("k_signed_distance");
    return CP_OK;
}

}  // namespace cp
