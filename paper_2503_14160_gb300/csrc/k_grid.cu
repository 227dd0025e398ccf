// Polar index of the obstacles for large scenes, and the evaluation kernel that queries it
// (Algorithm 1 step (2), d(q) of Sec. 3.1, arXiv 2503.14160).
//
// Every sphere of a configuration lies on the vertical plane at its slew angle, at signed
// horizontal distance h from the slew axis; so the obstacles a work unit (32 checkpoints of
// one candidate) can reach are those near the few slew angles and the range of |h| that its
// spheres cover. The index cuts the plane into angular bins about the slew axis and rings
// of width dr, and lists each obstacle in every (bin, ring) cell its reach disk (centre and
// broad-phase reach) overlaps, bin-major, so that the rings r0..r1 of one bin are one
// contiguous range. A unit takes the bins of its lanes' slew angles (and of the opposite
// direction when some h is negative) and the rings of its in-band |h|, tests the listed
// obstacles against its box in the slew frame (as the broad-phase form does), and takes
// the survivors through the same per-sphere filter and exact distances. Every obstacle a
// sphere can penetrate lies in a queried cell, passes the box test and the filter, so the
// results equal the exhaustive form's bit for bit.
//
// The index is built by kernels (count, exclusive scan, fill); the order inside a cell does
// not matter because the kernel takes a minimum of exactly computed distances.
#include <cmath>

#include "eval_common.cuh"

namespace cp {
namespace {

constexpr int kPolarThreads = 256;
#ifndef CP_POLAR_MIN_BLOCKS
#define CP_POLAR_MIN_BLOCKS 3   // CTAs of 8 warps resident per SM (at most 80 registers)
#endif
constexpr int kCtrlSlots = CP_MAX_WAYPOINTS + 8;   // control points per warp, float4
constexpr float kPolarPadR = 1e-3f;                // m: rounding of rho and of the ring index
constexpr float kPolarPadA = 1e-4f;                // rad: rounding of the angles and bin index
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kPi = 3.14159265358979323846f;

// Cells of an obstacle record r = {cx, cy, ., reach}: bins a0 .. a0 + na - 1 (mod n_ang) and
// rings r0 .. r1. A point within `reach` of the centre has |rho_p - rho| <= reach and, when
// rho > reach, an angle within asin(reach / rho) of the centre's.
__device__ __forceinline__ void polar_cells(const PolarDev &g, float4 r, int &a0, int &na, int &r0, int &r1)
{
    const float rho = sqrtf(fmaf(r.x, r.x, r.y * r.y));
    const float w = r.w + kPolarPadR;
    r0 = min(max((int)floorf((rho - w) * g.inv_dr), 0), g.n_ring - 1);
    r1 = min(max((int)floorf((rho + w) * g.inv_dr), 0), g.n_ring - 1);
    if (rho <= w + kPolarPadR) {
        a0 = 0;
        na = g.n_ang;
        return;
    }
    const float alpha = asinf(fminf(1.f, w / rho)) * 1.0001f + kPolarPadA;
    const float th = atan2f(r.y, r.x);
    const int b0 = (int)floorf((th - alpha + kPi) * g.inv_da);
    const int b1 = (int)floorf((th + alpha + kPi) * g.inv_da);
    na = b1 - b0 + 1;
    if (na >= g.n_ang) {
        a0 = 0;
        na = g.n_ang;
    } else {
        a0 = ((b0 % g.n_ang) + g.n_ang) % g.n_ang;
    }
}

// Record of obstacle id (cylinders first, then boxes): centre, id, broad-phase reach.
__device__ __forceinline__ float4 polar_record(const SceneDev &sc, int id)
{
    const float4 f = id < sc.n_cyl ? sc.cyl_filt[id] : sc.box_c[id - sc.n_cyl];
    return make_float4(f.x, f.y, __int_as_float(id), f.w);
}

__global__ void k_polar_count(const SceneDev sc, const PolarDev g, int *count)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= sc.n_cyl + sc.n_box) return;
    int a0, na, r0, r1;
    polar_cells(g, polar_record(sc, id), a0, na, r0, r1);
    for (int k = 0; k < na; ++k) {
        const int a = (a0 + k) % g.n_ang;
        for (int r = r0; r <= r1; ++r) atomicAdd(count + a * g.n_ring + r, 1);
    }
}

// Exclusive scan of count[0..n) into start[0..n] (start[n] = total) in one CTA; cursor
// receives a copy of start for the fill.
__global__ void __launch_bounds__(1024) k_polar_scan(const int *count, int n, int *start, int *cursor)
{
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int per = (n + 1023) / 1024;
    const int b = t * per, e = min(n, b + per);
    int acc = 0;
    for (int i = b; i < e; ++i) acc += count[i];
    part[t] = acc;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {   // inclusive Hillis-Steele scan of the parts
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = t > 0 ? part[t - 1] : 0;
    for (int i = b; i < e; ++i) {
        start[i] = run;
        cursor[i] = run;
        run += count[i];
    }
    if (t == 1023) start[n] = part[1023];
}

__global__ void k_polar_fill(const SceneDev sc, const PolarDev g, int *cursor, float4 *items, uint32_t *status)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= sc.n_cyl + sc.n_box) return;
    const float4 rec = polar_record(sc, id);
    int a0, na, r0, r1;
    polar_cells(g, rec, a0, na, r0, r1);
    for (int k = 0; k < na; ++k) {
        const int a = (a0 + k) % g.n_ang;
        for (int r = r0; r <= r1; ++r) {
            const int at = atomicAdd(cursor + a * g.n_ring + r, 1);
            if (at < g.capacity) items[at] = rec;
            else if (status != nullptr) atomicOr(status, DEV_ERR_OVERFLOW);   // the host's bound was short
        }
    }
}

// A surviving cylinder (filter record f = {cx, cy, W, reach}, exact record e = {R, z_lo,
// z_hi, (R + r_max)^2 + margin}) against the lane's spheres: with its centre at p along the
// lane's plane and q across it, sphere s passes when (h_s - p)^2 < e.w - q^2 and its centre
// lies within the cylinder's height range widened by r_max and the gate (so spheres outside
// the scene's band never pass); the passing spheres take the exact distance from their
// Cartesian centres, the same rounded products as every other form.
template <int NSPH>
__device__ __forceinline__ float polar_cylinder(const ModelDev &m, const float *H, const float *Z, float c1,
                                                float s1, float4 f, float4 e)
{
    const float p = fmaf(c1, f.x, s1 * f.y);
    const float q = fmaf(c1, f.y, -(s1 * f.x));
    const float rhs = fmaf(-q, q, e.w);
    const float zlo = e.y - m.r_max - kZGate, zhi = e.z + m.r_max + kZGate;
    float d = CUDART_INF_F;
#pragma unroll
    for (int s = 0; s < NSPH; ++s) {
        const float dh = H[s] - p;
        if (fmaf(dh, dh, -rhs) < 0.f && Z[s] > zlo && Z[s] < zhi)
            d = fminf(d, sdf_cylinder(__fmul_rn(c1, H[s]), __fmul_rn(s1, H[s]), Z[s], f.x, f.y, e) -
                             m.sph[s].radius);
    }
    return d;
}

template <int NSPH>
__global__ void __launch_bounds__(kPolarThreads, CP_POLAR_MIN_BLOCKS)
k_eval_polar(const ModelDev m, const SceneDev sc, const PolarDev g, const EvalArgs a)
{
    // Shared memory: the spline table, then per warp the control points of its candidate.
    extern __shared__ __align__(16) float4 s_basis[];
    float4 *s_ctrl = s_basis + 2 * a.S + (threadIdx.x >> 5) * kCtrlSlots;
    for (int i = threadIdx.x; i < 2 * a.S; i += blockDim.x) s_basis[i] = a.basis[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int n_warps = (int)((gridDim.x * blockDim.x) >> 5);
    const int items = a.n * a.P;
    const float zlo = sc.z_lo_all - m.r_max - kZGate, zhi = sc.z_hi_all + m.r_max + kZGate;
    uint32_t survivors = 0, tests = 0;

    for (int it = warp; it < items; it += n_warps) {
        const ItemRange ir = item_range(a, it);
        stage_controls(s_ctrl, a, ir.cand, lane);
        double acc = 0.0;
        uint32_t count = 0;
        for (int chunk = ir.c0; chunk < ir.c1; ++chunk) {
            const Checkpoint c = checkpoint_at(m, a, s_basis, s_ctrl, chunk, lane);
            float H[NSPH], Z[NSPH], s1, c1;
            crane_fk_polar<NSPH>(m, c.q, H, Z, s1, c1);
            // in-band extent of h at this lane; spheres outside the scene's height band (widened
            // by r_max) can penetrate nothing and take no part
            float hmin, hmax;
            band_extent<NSPH>(H, Z, zlo, zhi, hmin, hmax);
            const bool any_in = hmin <= hmax;
            float dmin = CUDART_INF_F;
            if (__any_sync(0xffffffffu, any_in)) {
                // the unit box (a lane with no in-band sphere adds its first sphere: a larger box
                // is still a bound)
                const float hb[2] = {any_in ? hmin : H[0], any_in ? hmax : H[0]};
                const UnitFrame fr = unit_frame<2>(s1, c1, hb);
                // radial extents on each side of the slew axis, and the spread of slew angles
                const float p_lo = warp_min(any_in && hmax >= 0.f ? fmaxf(hmin, 0.f) : CUDART_INF_F);
                const float p_hi = warp_max(any_in && hmax >= 0.f ? hmax : -CUDART_INF_F);
                const float n_lo = warp_min(any_in && hmin < 0.f ? fmaxf(-hmax, 0.f) : CUDART_INF_F);
                const float n_hi = warp_max(any_in && hmin < 0.f ? -hmin : -CUDART_INF_F);
                const float phi16 = __shfl_sync(0xffffffffu, c.q.x, 16);
                const float dphi = warp_max(any_in ? fabsf(c.q.x - phi16) : 0.f);
                const float phi0 = phi16 - kTwoPi * rintf(phi16 * (1.f / kTwoPi));   // in [-pi, pi]
                const float pad = kPolarPadA + 4e-7f * fabsf(phi16);
#pragma unroll 1
                for (int side = 0; side < 2; ++side) {
                    const float r_lo = side ? n_lo : p_lo, r_hi = side ? n_hi : p_hi;
                    if (!(r_lo <= r_hi)) continue;
                    const float centre = side ? (phi0 >= 0.f ? phi0 - kPi : phi0 + kPi) : phi0;
                    int a0 = (int)floorf((centre - dphi - pad + kPi) * g.inv_da);
                    int na = (int)floorf((centre + dphi + pad + kPi) * g.inv_da) - a0 + 1;
                    if (dphi + pad >= kPi || na >= g.n_ang) {
                        a0 = 0;
                        na = g.n_ang;
                    }
                    a0 = ((a0 % g.n_ang) + g.n_ang) % g.n_ang;
                    const int r0 = min(max((int)floorf((r_lo - kPolarPadR) * g.inv_dr), 0), g.n_ring - 1);
                    const int r1 = min(max((int)floorf((r_hi + kPolarPadR) * g.inv_dr), 0), g.n_ring - 1);
#pragma unroll 1
                    for (int k = 0; k < na; ++k) {
                        const int cell = ((a0 + k) % g.n_ang) * g.n_ring;
                        const int beg = __ldg(g.cell_start + cell + r0);
                        const int end = min(__ldg(g.cell_start + cell + r1 + 1), g.capacity);
                        for (int e0 = beg; e0 < end; e0 += 32) {
                            const int e = e0 + lane;
                            const float4 rec = e < end ? __ldg(g.items + e) : make_float4(0.f, 0.f, 0.f, -1.f);
                            uint32_t mask = __ballot_sync(0xffffffffu, e < end && unit_near(fr, rec));
                            tests += (uint32_t)min(32, end - e0);
                            survivors += __popc(mask);
                            while (mask) {
                                const int id = __shfl_sync(0xffffffffu, __float_as_int(rec.z), __ffs(mask) - 1);
                                mask &= mask - 1;
                                if (id < sc.n_cyl) {
                                    dmin = fminf(dmin, polar_cylinder<NSPH>(m, H, Z, c1, s1,
                                                                            __ldg(sc.cyl_filt + id),
                                                                            __ldg(sc.cyl_exact + id)));
                                } else {
                                    const float4 bc = __ldg(sc.box_c + id - sc.n_cyl);
                                    const float4 bh = __ldg(sc.box_h + id - sc.n_cyl);
#pragma unroll
                                    for (int s = 0; s < NSPH; ++s)
                                        dmin = fminf(dmin, sdf_box(__fmul_rn(c1, H[s]), __fmul_rn(s1, H[s]), Z[s],
                                                                   bc, bh) - m.sph[s].radius);
                                }
                            }
                        }
                    }
                }
            }
            unit_accumulate(a, c, dmin, ir.cand, chunk, lane, acc, count);
        }
        item_flush(a, it, acc, count, lane);
    }
    if (a.work != nullptr && lane == 0) {
        if (survivors != 0) atomicAdd(a.work, (unsigned long long)survivors);
        if (tests != 0) atomicAdd(a.work + 1, (unsigned long long)tests);
    }
}

// Raise (never lower) the dynamic shared-memory limit of a kernel.
template <typename F>
cudaError_t raise_polar_smem(F *fn, size_t smem)
{
    cudaFuncAttributes at{};
    cudaError_t e = cudaFuncGetAttributes(&at, fn);
    if (e == cudaSuccess && (size_t)at.maxDynamicSharedSizeBytes < smem)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

}  // namespace

// Upper bound on the entries of the index for a scene: per obstacle the bins of its angular
// half width asin(reach / rho) (all bins when it covers the axis) times the rings of its
// radial extent, each rounded up by two for the rounding of the device's cell ranges.
int64_t polar_items_bound(const cp_scene *sc, double r_max, int n_ang, int n_ring, double dr)
{
    const double da = 2.0 * M_PI / n_ang;
    auto cells = [&](double cx, double cy, double reach) -> int64_t {
        const double rho = std::sqrt(cx * cx + cy * cy);
        const double w = reach + 2.0 * (double)kPolarPadR + 0.02;
        int64_t rings = (int64_t)std::floor(2.0 * w / dr) + 3;
        if (rings > n_ring) rings = n_ring;
        int64_t bins = n_ang;
        if (rho > w + 0.01) {
            const double alpha = std::asin(std::min(1.0, w / (rho - 0.01))) * 1.001 + 2e-4;
            bins = std::min<int64_t>(n_ang, (int64_t)std::floor(2.0 * alpha / da) + 3);
        }
        return rings * bins;
    };
    int64_t total = 0;
    for (int i = 0; i < sc->n_cyl; ++i) {
        const cp_cylinder &c = sc->cyl[i];
        const double reach = std::sqrt((c.radius + r_max) * (c.radius + r_max) + 0.01) + 0.01;
        total += cells(c.cx, c.cy, reach);
    }
    for (int i = 0; i < sc->n_box; ++i) {
        const cp_box &b = sc->box[i];
        const double hx = 0.5 * (b.hi[0] - b.lo[0]), hy = 0.5 * (b.hi[1] - b.lo[1]);
        const double reach = std::sqrt(hx * hx + hy * hy) + r_max + 0.01;
        total += cells(0.5 * (b.lo[0] + b.hi[0]), 0.5 * (b.lo[1] + b.hi[1]), reach);
    }
    return total;
}

int launch_polar_build(const SceneDev &sc, const PolarDev &g, int *count, int *cursor, int *start,
                       float4 *items, uint32_t *status, cudaStream_t st)
{
    const int n_obs = sc.n_cyl + sc.n_box;
    const int cells = g.n_ang * g.n_ring;
    CP_CUDA(cudaMemsetAsync(count, 0, sizeof(int) * (size_t)cells, st));
    if (n_obs > 0) {
        k_polar_count<<<(n_obs + 255) / 256, 256, 0, st>>>(sc, g, count);
        CP_LAUNCHED("k_polar_count");
    }
    k_polar_scan<<<1, 1024, 0, st>>>(count, cells, start, cursor);
    CP_LAUNCHED("k_polar_scan");
    if (n_obs > 0) {
        k_polar_fill<<<(n_obs + 255) / 256, 256, 0, st>>>(sc, g, cursor, items, status);
        CP_LAUNCHED("k_polar_fill");
    }
    return CP_OK;
}

int launch_eval_polar(const ModelDev &m, const SceneDev &sc, const PolarDev &g, const EvalArgs &a,
                      int num_sms, cudaStream_t st)
{
    const int items = a.n * a.P;
    if (items == 0) return CP_OK;
    const size_t smem = sizeof(float4) * (2 * (size_t)a.S + (size_t)(kPolarThreads / 32) * kCtrlSlots);
    int per_sm = 0;
    if (m.n_spheres == 12) {
        CP_CUDA(raise_polar_smem(k_eval_polar<12>, smem));
        CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eval_polar<12>, kPolarThreads, smem));
    } else {
        CP_CUDA(raise_polar_smem(k_eval_polar<16>, smem));
        CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eval_polar<16>, kPolarThreads, smem));
    }
    if (per_sm < 1) per_sm = 1;
    if (a.ctas_per_sm > 0 && a.ctas_per_sm < per_sm) per_sm = a.ctas_per_sm;
    const int needed = (items + kPolarThreads / 32 - 1) / (kPolarThreads / 32);
    int grid = num_sms * per_sm;
    if (grid > needed) grid = needed;
    if (m.n_spheres == 12)
        k_eval_polar<12><<<grid, kPolarThreads, smem, st>>>(m, sc, g, a);
    else
        k_eval_polar<16><<<grid, kPolarThreads, smem, st>>>(m, sc, g, a);
    CP_LAUNCHED("k_eval_polar");
    return CP_OK;
}

}  // namespace cp
