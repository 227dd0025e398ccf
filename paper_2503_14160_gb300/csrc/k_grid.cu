// Polar index of the obstacles for large scenes, and the evaluation kernel that queries it
// (Algorithm 1 step (2), d(q) of Sec. 3.1, arXiv 2503.14160).
//
// Every sphere of a configuration lies on the vertical plane at its slew angle, at signed
// horizontal distance h from the slew axis. So the obstacles a checkpoint can touch are
// those within reach of one half-line from the axis (two when some h is negative), over the
// range of |h| its spheres cover. The index cuts the plane into angular bins about the slew
// axis and lists each obstacle in every bin its reach disk overlaps, ordered by the ring
// (of width dr) that holds its centre. A lane takes the bin of its slew angle and the rings
// within the largest reach of its in-band |h|, and tests each listed obstacle against all
// its spheres at once: the obstacle centre at p along the plane and q across it, sphere s
// passes when (h_s - p)^2 + q^2 is below the obstacle's bound (two packed FP32x2 operations
// per sphere pair); passing spheres take the exact distance. Every obstacle a sphere can
// penetrate is listed in the bin of the sphere's angle, within the rings the lane takes, and
// passes the test, and the exact distances are those of the exhaustive form, so the results
// equal the exhaustive form's bit for bit.
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
constexpr float kPolarPadR = 1e-3f;                // m: rounding of rho, |h| and the ring index
constexpr float kPolarPadA = 1e-4f;                // rad: rounding of the angles and bin index
constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPiHi = 6.28318548202514648f;   // 2 pi = kTwoPiHi + kTwoPiLo (Cody-Waite)
constexpr float kTwoPiLo = -1.7484555e-7f;

// Bins of an obstacle record r = {cx, cy, ., reach}: a0 .. a0 + na - 1 (mod n_ang), and the
// ring of its centre. A point within `reach` of the centre has, when rho > reach, an angle
// within asin(reach / rho) of the centre's; when rho <= reach every angle is possible.
__device__ __forceinline__ void polar_cells(const PolarDev &g, float4 r, int &a0, int &na, int &ring)
{
    const float rho = sqrtf(fmaf(r.x, r.x, r.y * r.y));
    const float w = r.w + kPolarPadR;
    ring = min(max((int)floorf(rho * g.inv_dr), 0), g.n_ring - 1);
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

// Entry of obstacle id (cylinders first, then boxes): centre, squared bound, id; and its
// record for the cells (the centre and the broad-phase reach).
__device__ __forceinline__ void polar_entry(const SceneDev &sc, int id, float4 &entry, float4 &cell_rec)
{
    if (id < sc.n_cyl) {
        const float4 f = sc.cyl_filt[id], e = sc.cyl_exact[id];
        entry = make_float4(f.x, f.y, e.w, __int_as_float(id));
        cell_rec = f;
    } else {
        const float4 c = sc.box_c[id - sc.n_cyl];   // w: half diagonal + r_max + 1 cm
        entry = make_float4(c.x, c.y, c.w * c.w, __int_as_float(id));
        cell_rec = c;
    }
}

__global__ void k_polar_count(const SceneDev sc, const PolarDev g, int *count)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= sc.n_cyl + sc.n_box) return;
    float4 entry, rec;
    polar_entry(sc, id, entry, rec);
    int a0, na, ring;
    polar_cells(g, rec, a0, na, ring);
    for (int k = 0; k < na; ++k) atomicAdd(count + ((a0 + k) % g.n_ang) * g.n_ring + ring, 1);
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
    float4 entry, rec;
    polar_entry(sc, id, entry, rec);
    int a0, na, ring;
    polar_cells(g, rec, a0, na, ring);
    for (int k = 0; k < na; ++k) {
        const int at = atomicAdd(cursor + ((a0 + k) % g.n_ang) * g.n_ring + ring, 1);
        if (at < g.capacity) items[at] = entry;
        else if (status != nullptr) atomicOr(status, DEV_ERR_OVERFLOW);   // the host's bound was short
    }
}

// Slew angle wrapped to [-pi, pi]: Cody-Waite reduction by 2 pi in two parts (accurate to a
// few 1e-7 rad for |phi| below 2^14 rad), in FP64 beyond.
__device__ __forceinline__ float wrap_angle(float phi)
{
    if (fabsf(phi) < 16384.f) {
        const float k = rintf(phi * 0.159154943091895336f);
        return fmaf(-k, kTwoPiLo, fmaf(-k, kTwoPiHi, phi));
    }
    const double d = (double)phi;
    return (float)(d - 6.283185307179586477 * rint(d * 0.15915494309189533577));
}

// The exact distance of every sphere whose filter passes against listed obstacle `id` (the
// spheres' Cartesian centres from the same rounded products as every other form; for a
// cylinder only within its height range widened by r_max and the gate).
template <int NSPH>
__device__ __forceinline__ float polar_exact(const ModelDev &m, const SceneDev &sc, const float *H,
                                             const float *Z, float c1, float s1, float p, float rhs, int id)
{
    float d = CUDART_INF_F;
    if (id < sc.n_cyl) {
        const float4 f = __ldg(sc.cyl_filt + id), e = __ldg(sc.cyl_exact + id);
        const float zlo = e.y - m.r_max - kZGate, zhi = e.z + m.r_max + kZGate;
#pragma unroll
        for (int s = 0; s < NSPH; ++s) {
            const float dh = H[s] - p;
            if (fmaf(dh, dh, -rhs) < 0.f && Z[s] > zlo && Z[s] < zhi)
                d = fminf(d, sdf_cylinder(__fmul_rn(c1, H[s]), __fmul_rn(s1, H[s]), Z[s], f.x, f.y, e) -
                                 m.sph[s].radius);
        }
    } else {
        const float4 bc = __ldg(sc.box_c + id - sc.n_cyl), bh = __ldg(sc.box_h + id - sc.n_cyl);
#pragma unroll
        for (int s = 0; s < NSPH; ++s) {
            const float dh = H[s] - p;
            if (fmaf(dh, dh, -rhs) < 0.f)
                d = fminf(d, sdf_box(__fmul_rn(c1, H[s]), __fmul_rn(s1, H[s]), Z[s], bc, bh) - m.sph[s].radius);
        }
    }
    return d;
}

// One work item (candidate, G consecutive units) of the polar form on one warp: per lane a
// checkpoint, its spheres' in-band extent of h, the one or two angular bins and the ring
// range that can hold an obstacle within reach, the packed filter over the listed entries
// and the exact distance of those that pass. kExtras false leaves out the work counters and
// the per-checkpoint outputs (the plan's own evaluations ask for neither); the sums are the
// same.
template <int NSPH, bool kExtras = true>
static __device__ __forceinline__ void polar_item(const ModelDev &m, const SceneDev &sc, const PolarDev &g,
                                                  const EvalArgs &a, const float4 *s_basis, float4 *s_ctrl,
                                                  int it, int lane, uint32_t &survivors, uint32_t &tests)
{
    const float zlo = sc.z_lo_all - m.r_max - kZGate, zhi = sc.z_hi_all + m.r_max + kZGate;
    const ItemRange ir = item_range(a, it);
    stage_controls(s_ctrl, a, ir.cand, lane);
    double acc = 0.0;
    uint32_t count = 0;
    for (int chunk = ir.c0; chunk < ir.c1; ++chunk) {
        const Checkpoint c = checkpoint_at(m, a, s_basis, s_ctrl, chunk, lane);
        float H[NSPH], Z[NSPH], s1, c1;
        crane_fk_polar<NSPH>(m, c.q, H, Z, s1, c1);
        // in-band extent of h at this lane; spheres outside the scene's height band (widened
        // by r_max) can penetrate nothing: they take no part (1e30 in the packed h)
        float hmin, hmax;
        float2 H2[NSPH / 2];
        band_pack<NSPH>(H, Z, zlo, zhi, hmin, hmax, H2);
        float dmin = CUDART_INF_F;
        if (hmin <= hmax) {
            const float phi0 = wrap_angle(c.q.x);
#pragma unroll 1
            for (int side = 0; side < 2; ++side) {
                // spheres with h >= 0 lie on the half-line at the slew angle, those with h < 0
                // on the opposite one, at distance |h| from the axis
                const float r_lo = side ? fmaxf(-hmax, 0.f) : fmaxf(hmin, 0.f);
                const float r_hi = side ? -hmin : hmax;
                if (!(r_lo <= r_hi)) continue;
                const float ang = side ? (phi0 >= 0.f ? phi0 - kPi : phi0 + kPi) : phi0;
                const int bin = min(max((int)floorf((ang + kPi) * g.inv_da), 0), g.n_ang - 1);
                const float reach = g.w_max + kPolarPadR;
                const int r0 = min(max((int)floorf((r_lo - reach) * g.inv_dr), 0), g.n_ring - 1);
                const int r1 = min(max((int)floorf((r_hi + reach) * g.inv_dr), 0), g.n_ring - 1);
                const int cell = bin * g.n_ring;
                const int beg = __ldg(g.cell_start + cell + r0);
                const int end = min(__ldg(g.cell_start + cell + r1 + 1), g.capacity);
                if (kExtras) tests += (uint32_t)max(end - beg, 0);
                for (int e = beg; e < end; ++e) {
                    const float4 rec = __ldg(g.items + e);   // {cx, cy, bound, id}
                    const float p = fmaf(c1, rec.x, s1 * rec.y);
                    const float q = fmaf(c1, rec.y, -(s1 * rec.x));
                    const float rhs = fmaf(-q, q, rec.z);
                    const float2 mp2 = make_float2(-p, -p), mr2 = make_float2(-rhs, -rhs);
                    float2 t[NSPH / 2];
#pragma unroll
                    for (int k = 0; k < NSPH / 2; ++k) {
                        const float2 dh = __fadd2_rn(H2[k], mp2);
                        t[k] = __ffma2_rn(dh, dh, mr2);
                    }
                    if (any_negative<NSPH>(t)) {
                        if (kExtras) ++survivors;
                        dmin = fminf(dmin, polar_exact<NSPH>(m, sc, H, Z, c1, s1, p, rhs, __float_as_int(rec.w)));
                    }
                }
            }
        }
        __syncwarp();
        unit_accumulate<kExtras>(a, c, dmin, ir.cand, chunk, lane, acc, count);
    }
    item_flush(a, it, acc, count, lane);
}

template <int NSPH, bool kExtras>
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
    uint32_t survivors = 0, tests = 0;   // (lane, obstacle) pairs passing the packed filter; tested
    if (a.queue != nullptr) {
        // each warp takes the next item from the launch's counter when it is done with one, so
        // candidates of uneven cost (those in collision take the exact distances) even out;
        // the counter only grows, so every warp leaves once the items are handed out
        for (;;) {
            int it = 0;
            if (lane == 0) it = atomicAdd(a.queue, 1);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= items) break;
            polar_item<NSPH, kExtras>(m, sc, g, a, s_basis, s_ctrl, it, lane, survivors, tests);
        }
    } else {
        for (int it = warp; it < items; it += n_warps)
            polar_item<NSPH, kExtras>(m, sc, g, a, s_basis, s_ctrl, it, lane, survivors, tests);
    }
    if (kExtras && a.work != nullptr) {
        const uint32_t ws = __reduce_add_sync(0xffffffffu, survivors);
        const uint32_t wt = __reduce_add_sync(0xffffffffu, tests);
        if (lane == 0 && ws != 0) atomicAdd(a.work, (unsigned long long)ws);
        if (lane == 0 && wt != 0) atomicAdd(a.work + 1, (unsigned long long)wt);
    }
}

// The evaluations of every query of a batch in one persistent launch. The work is a list of
// tiles {query, first item, end item} (a tile is one query's consecutive work items); each
// CTA takes the next tile from a device counter (an atomic add: no CTA ever waits on
// another) until the list is exhausted. When the query of its tile differs from the one it
// holds, the CTA restages: it copies the query's view (its evaluation arguments, obstacle
// records and polar index) and the query's spline table into shared memory. The warps then
// take the tile's items in turn; an item's arithmetic is that of the single-query launch.
template <int NSPH, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
k_batch_eval_polar(const ModelDev m, const BatchEvalDev *__restrict__ qd, const int4 *__restrict__ tiles,
                   int n_tiles, int *queue, int max_S)
{
    extern __shared__ __align__(16) float4 s_basis[];
    __shared__ __align__(16) unsigned char s_q_raw[sizeof(BatchEvalDev)];   // the held query's view
    BatchEvalDev &s_q = *reinterpret_cast<BatchEvalDev *>(s_q_raw);
    __shared__ int s_tile;
    constexpr int W = THREADS / 32;
    float4 *s_ctrl = s_basis + 2 * max_S + (threadIdx.x >> 5) * kCtrlSlots;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int held = -1;
    uint32_t survivors = 0, tests = 0;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(queue, 1);
        __syncthreads();
        const int t = s_tile;
        if (t >= n_tiles) break;
        const int4 tile = __ldg(tiles + t);
        if (tile.x != held) {
            held = tile.x;
            const int *src = reinterpret_cast<const int *>(qd + held);
            int *dst = reinterpret_cast<int *>(&s_q);
            for (int i = threadIdx.x; i < (int)(sizeof(BatchEvalDev) / sizeof(int)); i += THREADS) dst[i] = __ldg(src + i);
            __syncthreads();
            for (int i = threadIdx.x; i < 2 * s_q.a.S; i += THREADS) s_basis[i] = __ldg(s_q.a.basis + i);
            __syncthreads();
        }
        for (int it = tile.y + wib; it < tile.z; it += W)   // the batch asks for no counters or outputs
            polar_item<NSPH, false>(m, s_q.sc, s_q.g, s_q.a, s_basis, s_ctrl, it, lane, survivors, tests);
        __syncthreads();   // the tile's items are done before s_tile and s_q change
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

// Broad-phase reach of the device records (k_prepare_scene), in FP64.
double cylinder_reach(const cp_cylinder &c, double r_max)
{
    const double reach = c.radius + r_max;
    return std::sqrt(reach * reach + 0.01) + 0.01;
}

double box_reach(const cp_box &b, double r_max)
{
    const double hx = 0.5 * (b.hi[0] - b.lo[0]), hy = 0.5 * (b.hi[1] - b.lo[1]);
    return std::sqrt(hx * hx + hy * hy) + r_max + 0.01;
}

}  // namespace

// Upper bound on the entries of the index for a scene: per obstacle the bins of its angular
// half width asin(reach / rho) (all bins when it covers the axis), rounded up by three for
// the padding and the rounding of the device's bin range.
int64_t polar_items_bound(const cp_scene *sc, double r_max, int n_ang)
{
    const double da = 2.0 * M_PI / n_ang;
    auto bins = [&](double cx, double cy, double reach) -> int64_t {
        const double rho = std::sqrt(cx * cx + cy * cy);
        const double w = reach + 2.0 * (double)kPolarPadR + 0.02;
        if (rho <= w + 0.01) return n_ang;
        const double alpha = std::asin(std::min(1.0, w / (rho - 0.01))) * 1.001 + 2e-4;
        return std::min<int64_t>(n_ang, (int64_t)std::floor(2.0 * alpha / da) + 3);
    };
    int64_t total = 0;
    for (int i = 0; i < sc->n_cyl; ++i) total += bins(sc->cyl[i].cx, sc->cyl[i].cy, cylinder_reach(sc->cyl[i], r_max));
    for (int i = 0; i < sc->n_box; ++i) {
        const cp_box &b = sc->box[i];
        total += bins(0.5 * (b.lo[0] + b.hi[0]), 0.5 * (b.lo[1] + b.hi[1]), box_reach(b, r_max));
    }
    return total;
}

// The largest broad-phase reach of the scene's records, rounded up past the FP32 rounding
// of the records themselves.
float polar_reach_max(const cp_scene *sc, double r_max)
{
    double w = 0.0;
    for (int i = 0; i < sc->n_cyl; ++i) w = std::max(w, cylinder_reach(sc->cyl[i], r_max));
    for (int i = 0; i < sc->n_box; ++i) w = std::max(w, box_reach(sc->box[i], r_max));
    return (float)(w * (1.0 + 1e-5) + 1e-4);
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
    // the plain form (no work counters, no per-checkpoint outputs) drops their bookkeeping
    const bool extras = a.work != nullptr || a.words_out != nullptr || a.pen_out != nullptr;
    auto kern = m.n_spheres == 12 ? (extras ? k_eval_polar<12, true> : k_eval_polar<12, false>)
                                  : (extras ? k_eval_polar<16, true> : k_eval_polar<16, false>);
    int per_sm = 0;
    CP_CUDA(raise_polar_smem(kern, smem));
    CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPolarThreads, smem));
    if (per_sm < 1) per_sm = 1;
    if (a.ctas_per_sm > 0 && a.ctas_per_sm < per_sm) per_sm = a.ctas_per_sm;
    const int needed = (items + kPolarThreads / 32 - 1) / (kPolarThreads / 32);
    int grid = num_sms * per_sm;
    if (grid > needed) grid = needed;
    if (a.queue != nullptr) CP_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(int), st));
    kern<<<grid, kPolarThreads, smem, st>>>(m, sc, g, a);
    CP_LAUNCHED("k_eval_polar");
    return CP_OK;
}

// Batched form: CTAs of 128, 256 or 512 threads (block shape picked by the autotuner).
template <int NSPH, int THREADS>
static auto batch_eval_kernel()
{
    constexpr int MINB = THREADS == 128 ? 2 * CP_POLAR_MIN_BLOCKS : (THREADS == 256 ? CP_POLAR_MIN_BLOCKS : 1);
    return k_batch_eval_polar<NSPH, THREADS, MINB>;
}

template <int NSPH>
static void *batch_eval_fn(int threads)
{
    if (threads == 128) return (void *)batch_eval_kernel<NSPH, 128>();
    if (threads == 256) return (void *)batch_eval_kernel<NSPH, 256>();
    if (threads == 512) return (void *)batch_eval_kernel<NSPH, 512>();
    return nullptr;
}

static size_t batch_eval_smem(int threads, int max_S)
{
    return sizeof(float4) * (2 * (size_t)max_S + (size_t)(threads / 32) * kCtrlSlots);
}

int batch_eval_max_blocks(const ModelDev &m, int threads, int max_S, int num_sms)
{
    void *fn = m.n_spheres == 12 ? batch_eval_fn<12>(threads) : batch_eval_fn<16>(threads);
    if (fn == nullptr) return set_error("batched evaluation: %d threads per CTA is not 128, 256 or 512", threads), -1;
    const size_t smem = batch_eval_smem(threads, max_S);
    cudaFuncAttributes at{};
    CP_CUDA(cudaFuncGetAttributes(&at, fn));
    if ((size_t)at.maxDynamicSharedSizeBytes < smem)
        CP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    return (per_sm < 1 ? 1 : per_sm) * num_sms;
}

int launch_batch_eval_polar(const ModelDev &m, const BatchEvalDev *qd, const int4 *tiles, int n_tiles, int *queue,
                            int max_S, int threads, int blocks, cudaStream_t st)
{
    if (n_tiles == 0) return CP_OK;
    void *fn = m.n_spheres == 12 ? batch_eval_fn<12>(threads) : batch_eval_fn<16>(threads);
    if (fn == nullptr) return set_error("batched evaluation: %d threads per CTA is not 128, 256 or 512", threads), CP_ERR_ARG;
    const size_t smem = batch_eval_smem(threads, max_S);
    ModelDev mm = m;
    void *args[] = {(void *)&mm, (void *)&qd, (void *)&tiles, (void *)&n_tiles, (void *)&queue, (void *)&max_S};
    CP_CUDA(cudaLaunchKernel(fn, dim3(blocks), dim3(threads), args, smem, st));
    CP_LAUNCHED("k_batch_eval_polar");
    return CP_OK;
}

}  // namespace cp
