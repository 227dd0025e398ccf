// Uniform 2-D grid of the obstacles for large scenes, and the evaluation kernel that
// queries it (Algorithm 1 step (2), d(q) of Sec. 3.1, arXiv 2503.14160).
// Cell entries are filter records {cx, cy, W, id}: one load per entry, the same 2-FMA
// reach test as the brute-force kernel, and the exact distance only within reach.
//
// The grid covers a square window centred on the crane base with cells of side h. Every
// obstacle goes into every cell that its footprint, dilated by the largest sphere radius
// (plus a small pad for rounding), overlaps; so a sphere can only touch obstacles listed in
// the cell that holds its centre. Obstacles whose dilated footprint leaves the window are
// also listed separately, and a sphere centre outside the window checks that list. Cell
// lists are built by kernels (count, exclusive scan, fill); the order inside a cell does not
// matter because the kernel takes a minimum of exactly computed distances.
#include <cmath>

#include "eval_common.cuh"

namespace cp {
namespace {

constexpr int kGridThreads = 256;
#ifndef CP_GRID_MIN_BLOCKS
#define CP_GRID_MIN_BLOCKS 4   // CTAs of 8 warps resident per SM (at most 64 registers)
#endif
constexpr float kGridPad = 1e-3f;   // m; covers float rounding of the cell index

// Dilated footprint [x0, x1] x [y0, y1] of obstacle id (cylinders first, then boxes).
__device__ __forceinline__ void footprint(const SceneDev &sc, float r, int id, float &x0,
                                          float &x1, float &y0, float &y1)
{
    if (id < sc.n_cyl) {
        const float4 f = sc.cyl_filt[id], e = sc.cyl_exact[id];
        const float reach = e.x + r + kGridPad;
        x0 = f.x - reach;
        x1 = f.x + reach;
        y0 = f.y - reach;
        y1 = f.y + reach;
    } else {
        const float4 c = sc.box_c[id - sc.n_cyl], h = sc.box_h[id - sc.n_cyl];
        x0 = c.x - h.x - r - kGridPad;
        x1 = c.x + h.x + r + kGridPad;
        y0 = c.y - h.y - r - kGridPad;
        y1 = c.y + h.y + r + kGridPad;
    }
}

// Cell range of a footprint clipped to the window; `outside` when it leaves the window.
__device__ __forceinline__ bool cell_range(const GridDev &g, float x0, float x1, float y0,
                                           float y1, int &ix0, int &ix1, int &iy0, int &iy1)
{
    const float fx0 = (x0 - g.x0) * g.inv_h, fx1 = (x1 - g.x0) * g.inv_h;
    const float fy0 = (y0 - g.y0) * g.inv_h, fy1 = (y1 - g.y0) * g.inv_h;
    const bool outside = fx0 < 0.f || fy0 < 0.f || fx1 >= (float)g.nx || fy1 >= (float)g.ny;
    ix0 = max(0, (int)floorf(fx0));
    iy0 = max(0, (int)floorf(fy0));
    ix1 = min(g.nx - 1, (int)floorf(fx1));
    iy1 = min(g.ny - 1, (int)floorf(fy1));
    return outside;
}

__global__ void k_grid_count(const SceneDev sc, const GridDev g, float r, int *count,
                             int *n_outside)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= sc.n_cyl + sc.n_box) return;
    float x0, x1, y0, y1;
    footprint(sc, r, id, x0, x1, y0, y1);
    int ix0, ix1, iy0, iy1;
    if (cell_range(g, x0, x1, y0, y1, ix0, ix1, iy0, iy1)) atomicAdd(n_outside, 1);
    for (int iy = iy0; iy <= iy1; ++iy)
        for (int ix = ix0; ix <= ix1; ++ix) atomicAdd(count + iy * g.nx + ix, 1);
}

// Exclusive scan of count[0..n) into start[0..n] (start[n] = total) in one CTA; cursor
// receives a copy of start for the fill.
__global__ void __launch_bounds__(1024) k_grid_scan(const int *count, int n, int *start, int *cursor)
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

// Cell entries are records {cx, cy, W, id}: a cylinder's filter record (W as in the
// brute-force kernel) with its id in the last word; boxes carry W = -huge so that the
// filter always passes them on to the exact distance.
__device__ __forceinline__ float4 grid_record(const SceneDev &sc, int id)
{
    if (id < sc.n_cyl) {
        const float4 f = sc.cyl_filt[id];
        return make_float4(f.x, f.y, f.z, __int_as_float(id));
    }
    return make_float4(0.f, 0.f, -3.0e38f, __int_as_float(id));
}

__global__ void k_grid_fill(const SceneDev sc, const GridDev g, float r, int *cursor, float4 *items,
                            float4 *outside, int *outside_cursor)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= sc.n_cyl + sc.n_box) return;
    float x0, x1, y0, y1;
    footprint(sc, r, id, x0, x1, y0, y1);
    const float4 rec = grid_record(sc, id);
    int ix0, ix1, iy0, iy1;
    if (cell_range(g, x0, x1, y0, y1, ix0, ix1, iy0, iy1)) outside[atomicAdd(outside_cursor, 1)] = rec;
    for (int iy = iy0; iy <= iy1; ++iy)
        for (int ix = ix0; ix <= ix1; ++ix) items[atomicAdd(cursor + iy * g.nx + ix, 1)] = rec;
}

// Signed distance of sphere (x, y, z, r) to the obstacle of a cell record.
__device__ __forceinline__ float record_distance(const SceneDev &sc, float4 rec, float x, float y,
                                                 float z, float r)
{
    const int id = __float_as_int(rec.w);
    if (id < sc.n_cyl) {
        const float4 e = __ldg(sc.cyl_exact + id);
        if (z < e.y - r - kZGate || z > e.z + r + kZGate) return CUDART_INF_F;   // cannot penetrate
        return sdf_cylinder(x, y, z, rec.x, rec.y, e) - r;
    }
    const float4 c = __ldg(sc.box_c + id - sc.n_cyl), h = __ldg(sc.box_h + id - sc.n_cyl);
    return sdf_box(x, y, z, c, h) - r;
}

template <int NSPH>
__global__ void __launch_bounds__(kGridThreads, CP_GRID_MIN_BLOCKS)
k_eval_grid(const ModelDev m, const SceneDev sc, const GridDev g, const EvalArgs a)
{
    // Shared memory: the spline table, then per warp, sphere and lane the record
    // {h, z, first entry, end entry} of the sphere's cell (h its signed horizontal distance
    // from the slew axis), read by the rolled sphere loop.
    extern __shared__ __align__(16) float4 s_basis[];
    float4 *s_sph = s_basis + 2 * a.S;
    for (int i = threadIdx.x; i < 2 * a.S; i += blockDim.x) s_basis[i] = a.basis[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int n_warps = (int)((gridDim.x * blockDim.x) >> 5);
    float4 *my_sph = s_sph + (threadIdx.x >> 5) * NSPH * 32 + lane;
    const int units = a.n * a.chunks;
    uint32_t tested = 0;   // cell entries this lane visited
    for (int u = warp; u < units; u += n_warps) {
        const int cand = (int)fdiv((uint32_t)u, a.div_chunks);
        const int chunk = u - cand * a.chunks;
        const Checkpoint c = checkpoint_setup(m, a, s_basis, cand, chunk, lane);
        float H[NSPH], Z[NSPH], s1, c1;
        crane_fk_polar<NSPH>(m, c.q, H, Z, s1, c1);
        // Per sphere the entry range of its cell, looked up for all spheres first so that the
        // loads are in flight together, and kept with h and z in shared memory: the sphere
        // loop below stays rolled (one copy of the entry loop serves all spheres; unrolled,
        // the code outgrows the instruction cache) without per-thread local arrays.
#pragma unroll
        for (int s = 0; s < NSPH; ++s) {
            const float x = __fmul_rn(c1, H[s]), y = __fmul_rn(s1, H[s]);
            const float fx = (x - g.x0) * g.inv_h, fy = (y - g.y0) * g.inv_h;
            int first = -1, end = 0;   // -1: outside the window
            if (fx >= 0.f && fy >= 0.f && fx < (float)g.nx && fy < (float)g.ny) {
                const int cell = (int)fy * g.nx + (int)fx;
                first = __ldg(g.cell_start + cell);
                end = __ldg(g.cell_start + cell + 1);
            }
            my_sph[s * 32] = make_float4(H[s], Z[s], __int_as_float(first), __int_as_float(end));
        }
        __syncwarp();
        float dmin = CUDART_INF_F;
#pragma unroll 1
        for (int s = 0; s < m.n_spheres; ++s) {
            const float4 sp = my_sph[s * 32];
            const float xs = __fmul_rn(c1, sp.x), ys = __fmul_rn(s1, sp.x);
            const float qx = -2.f * xs, qy = -2.f * ys, T = kFilterMargin - fmaf(xs, xs, ys * ys);
            const float r = m.sph[s].radius;
            const float4 *list = g.items;
            int it = __float_as_int(sp.z), end = __float_as_int(sp.w);
            if (it < 0) {
                list = g.outside;
                it = 0;
                end = __ldg(g.n_outside);
            }
            if (sp.y < sc.z_lo_all - r - kZGate || sp.y > sc.z_hi_all + r + kZGate) end = it;   // above or below every obstacle
            tested += (uint32_t)(end - it);
            for (; it < end; ++it) {
                const float4 rec = __ldg(list + it);
                if (fmaf(qx, rec.x, fmaf(qy, rec.y, rec.z)) < T)   // within reach (2-D)
                    dmin = fminf(dmin, record_distance(sc, rec, xs, ys, sp.y, r));
            }
        }
        __syncwarp();
        unit_epilogue(a, c, dmin, cand, chunk, lane);
    }
    if (a.work != nullptr) {
        const uint32_t warp_tested = __reduce_add_sync(0xffffffffu, tested);
        if (lane == 0 && warp_tested != 0) atomicAdd(a.work, (unsigned long long)warp_tested);
    }
}

// Raise (never lower) the dynamic shared-memory limit of a grid kernel.
template <typename F>
cudaError_t raise_grid_smem(F *fn, size_t smem)
{
    cudaFuncAttributes at{};
    cudaError_t e = cudaFuncGetAttributes(&at, fn);
    if (e == cudaSuccess && (size_t)at.maxDynamicSharedSizeBytes < smem)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

}  // namespace

// Upper bound on the cell entries of a scene: per obstacle the cells of its dilated
// footprint, at most floor(side / h) + 2 per axis; one more per axis covers the float
// rounding of the device's cell range.
int64_t grid_items_bound(const cp_scene *sc, double r_max, double h)
{
    const double pad = 2.0 * (r_max + (double)kGridPad);
    int64_t total = 0;
    for (int i = 0; i < sc->n_cyl; ++i) {
        const int64_t c = (int64_t)std::floor((2.0 * sc->cyl[i].radius + pad) / h) + 3;
        total += c * c;
    }
    for (int i = 0; i < sc->n_box; ++i) {
        const cp_box &b = sc->box[i];
        const int64_t cx = (int64_t)std::floor((b.hi[0] - b.lo[0] + pad) / h) + 3;
        const int64_t cy = (int64_t)std::floor((b.hi[1] - b.lo[1] + pad) / h) + 3;
        total += cx * cy;
    }
    return total;
}

int launch_grid_build(const SceneDev &sc, const GridDev &g, float r_max, int *count, int *cursor,
                      int *start, float4 *items, float4 *outside, int *counters /* [2] */,
                      cudaStream_t st)
{
    const int n_obs = sc.n_cyl + sc.n_box;
    const int cells = g.nx * g.ny;
    CP_CUDA(cudaMemsetAsync(count, 0, sizeof(int) * (size_t)cells, st));
    CP_CUDA(cudaMemsetAsync(counters, 0, sizeof(int) * 2, st));
    if (n_obs > 0) {
        k_grid_count<<<(n_obs + 255) / 256, 256, 0, st>>>(sc, g, r_max, count, counters);
        CP_LAUNCHED("k_grid_count");
    }
    k_grid_scan<<<1, 1024, 0, st>>>(count, cells, start, cursor);
    CP_LAUNCHED("k_grid_scan");
    if (n_obs > 0) {
        k_grid_fill<<<(n_obs + 255) / 256, 256, 0, st>>>(sc, g, r_max, cursor, items, outside,
                                                          counters + 1);
        CP_LAUNCHED("k_grid_fill");
    }
    return CP_OK;
}

int launch_eval_grid(const ModelDev &m, const SceneDev &sc, const GridDev &g, const EvalArgs &a,
                     int num_sms, cudaStream_t st)
{
    const int units = a.n * a.chunks;
    if (units == 0) return CP_OK;
    const int nsph = m.n_spheres == 12 ? 12 : 16;
    const size_t smem = sizeof(float4) * (2 * (size_t)a.S + (size_t)(kGridThreads / 32) * nsph * 32);
    int per_sm = 0;
    if (m.n_spheres == 12) {
        CP_CUDA(raise_grid_smem(k_eval_grid<12>, smem));
        CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eval_grid<12>, kGridThreads, smem));
    } else {
        CP_CUDA(raise_grid_smem(k_eval_grid<16>, smem));
        CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eval_grid<16>, kGridThreads, smem));
    }
    if (per_sm < 1) per_sm = 1;
    if (a.ctas_per_sm > 0 && a.ctas_per_sm < per_sm) per_sm = a.ctas_per_sm;
    const int needed = (units + kGridThreads / 32 - 1) / (kGridThreads / 32);
    int grid = num_sms * per_sm;
    if (grid > needed) grid = needed;
    if (m.n_spheres == 12)
        k_eval_grid<12><<<grid, kGridThreads, smem, st>>>(m, sc, g, a);
    else
        k_eval_grid<16><<<grid, kGridThreads, smem, st>>>(m, sc, g, a);
    CP_LAUNCHED("k_eval_grid");
    return CP_OK;
}

}  // namespace cp
