// Step (1) of Algorithm 1 drawn from the elites of the last update, with no factor
// (arXiv 2503.14160, Sec. 4.1). With C = sum_j w_j (x_(j) - mu)(x_(j) - mu)^T + eps I (steps
// (5)-(6), mu the new mean)
//     xi_i = mu + sigma (sum_j sqrt(w_j) (x_(j) - mu) g_ij + sqrt(eps) g'_i)
// is normal with mean mu and covariance sigma^2 C exactly, so the FP64 moments and the FP64
// Cholesky factor (whose dependent chains are slow on this part) leave the iteration; the
// draw is the product G Y of N x nu normals and the nu x D scaled elite deviations, a dense
// contraction that runs on the tensor cores.
//   k_elite_weights  sigma sqrt(w_j) in FP32, once per planner
//   k_elite_update   one cooperative launch: mu = sum_j w_j x_(j) in FP64 (block partials,
//                    a grid barrier, a fixed-order sum), mu as an FP32 pair mu_f + mu_lo,
//                    and Y[j][d] = sigma sqrt(w_j) (x_(j)d - mu_d) in FP32 (within 4 ulp),
//                    split into two TF32 parts Y = Y_hi + Y_lo, written in the tensor cores'
//                    operand layout
//   k_sample_elites  partial products over a slice of the elites on the tensor cores
//                    (tcgen05, kind::tf32): a CTA takes 128 candidates and all D coordinates;
//                    eight warps generate the normals of 16 elites per pipeline stage
//                    (Philox blocks in place, split G = G_hi + G_lo) into shared memory
//                    while a ninth warp feeds the tensor cores the previous stage; the
//                    accumulator lives in tensor memory. G Y is formed as
//                    G_hi Y_hi + G_hi Y_lo + G_lo Y_hi ("3xTF32": each product within
//                    3 * 2^-22 of the FP32 product, FP32 accumulation)
//   k_sample_reduce  xi = mu + sum of the slices (fixed order) + sigma sqrt(eps) g'
// Normals: candidate i at iteration t has the stream of Philox blocks (b, i, t, query), four
// standard normals per block (Box-Muller on words 0-1 and 2-3); g_ij is normal j, g'_id
// normal nu + d.
#include <algorithm>

#include "cp_internal.cuh"
#include "philox.cuh"
#include "tcgen05.cuh"

namespace cp {
namespace {

constexpr int kTcM = 128;          // candidates per CTA: the MMA's M, one tensor-memory lane each
constexpr int kChunkE = 16;        // elites per pipeline stage: two MMA K steps of 8
constexpr int kTcThreads = 256;    // generator threads, two per candidate row (+ one MMA warp)
constexpr int kStages = 2;
constexpr long long kWaitCycles = 2000000000ll;   // about one second at 2 GHz
#ifndef CP_ELITE_MAX_SLICES
#define CP_ELITE_MAX_SLICES 32   // elite slices of the tensor-core product (partials to add)
#endif

// D padded to the MMA's N granularity (16 for M = 128).
__host__ __device__ inline int padded_d(int D) { return (D + 15) & ~15; }

// Floats per chunk of the packed operand: Y_hi then Y_lo, each Dp rows x 16 elites.
__host__ __device__ inline int chunk_floats(int Dp) { return 2 * Dp * kChunkE; }

// Float index of element (row, k) of a tile of 16 elements of K in the K-major core-matrix
// layout: core (row / 8, k / 4) of 32 floats, cores along K adjacent (128 bytes), row groups
// 4 cores (512 bytes) apart; within a core, row r at 4 r.
__host__ __device__ inline int core_index(int row, int k)
{
    return ((row >> 3) * (kChunkE / 4) + (k >> 2)) * 32 + (row & 7) * 4 + (k & 3);
}

constexpr uint32_t kCoreLbo = 128;                 // bytes between cores adjacent along K
constexpr uint32_t kCoreSbo = 128 * (kChunkE / 4);  // bytes between 8-row groups

size_t tc_smem_bytes(int Dp) { return (size_t)kStages * 4 * (2 * kTcM * kChunkE + 2 * (size_t)Dp * kChunkE); }

uint32_t tmem_columns(int Dp)
{
    uint32_t c = 32;
    while ((int)c < Dp) c <<= 1;
    return c;
}

__global__ void k_elite_weights(const double *__restrict__ w, int nu, double sigma, float *sw)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nu) sw[k] = (float)(sigma * sqrt(w[k]));
}

constexpr int kEUThreads = 256;
constexpr int kSumBatch = 16;  // partials loaded before they are added

// All blocks of a launch wait here until every block has arrived. bar[0] counts arrivals,
// bar[1] is the generation; both start at zero and the last arrival resets the count, so
// the pair is ready for the next launch. The wait is bounded: false when it ran out. Only
// for cooperative launches, whose blocks are all resident at once.
__device__ bool grid_barrier(unsigned int *bar, unsigned int nblocks, long long limit)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = bar + 1;
        const unsigned int g0 = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > limit) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Steps (5) and the operand of the next draw, in one cooperative launch of nb blocks (one
// SM each at most) over the chunks of 16 elites (block b takes chunks b, b + nb, ...):
//  1. mu = sum_j w_j x_(j) (FP64): thread (g, d), g < G = 256 / D' (D' = D rounded up to
//     32), takes elites g, g + G, ... of the block's chunks; the groups are added in order
//     into part[b][d].
//  2. after a grid barrier every block adds part[0..nb)[d] in the same fixed order (so the
//     result is deterministic and identical in every block); block 0 writes mu, its FP32
//     rounding mu_f and the rest mu_lo = mu - mu_f rounded to FP32.
//  3. Y[j][d] = sigma sqrt(w_j) (x_(j)d - mu_d) in FP32 against mu_f + mu_lo: x - mu_f is
//     exact when both lie within a factor of two of each other (Sterbenz) and otherwise
//     rounded once with mu_lo far below it, so with the second difference, the FP32
//     sigma sqrt(w_j) and the product, Y is within 4 ulp of its FP64 value; then the TF32
//     split Y = Y_hi + Y_lo into the tensor cores' layout. Rows d >= D and elites past nu
//     of the packed operand stay zero (the buffer is cleared once).
// FP64 work is one FMA per element and a short fixed sum per coordinate: FP64 throughput is
// a small fraction of FP32 on this part. A barrier that runs out records DEV_ERR_TIMEOUT.
__global__ void __launch_bounds__(kEUThreads)
k_elite_update(const float *__restrict__ elites, const double *__restrict__ w, const float *__restrict__ sw,
               int nu, int D, double *part, unsigned int *bar, double *mu, float *mu_f, float *mu_lo, float *Yp,
               uint32_t *status)
{
    __shared__ double s_acc[kEUThreads];
    __shared__ float s_hi[4 * CP_MAX_WAYPOINTS], s_lo[4 * CP_MAX_WAYPOINTS];
    const int Dr = (D + 31) & ~31, G = kEUThreads / Dr, Dp = padded_d(D);
    const int tid = threadIdx.x, g = tid / Dr, d = tid - g * Dr;
    const bool on = g < G && d < D;
    const int nb = (int)gridDim.x, chunks = (nu + kChunkE - 1) / kChunkE;

    double a = 0.0;
    if (on)
        for (int c = blockIdx.x; c < chunks; c += nb) {   // at most 8 elites of a chunk per thread
            const int e0 = c * kChunkE, ne = min(kChunkE, nu - e0);
            double wv[8];
            float xv[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {   // loads first, all in flight together
                const int k = g + m * G;
                wv[m] = k < ne ? w[e0 + k] : 0.0;
                xv[m] = k < ne ? elites[(size_t)(e0 + k) * D + d] : 0.f;
            }
#pragma unroll
            for (int m = 0; m < 8; ++m) a = fma(wv[m], (double)xv[m], a);
        }
    s_acc[tid] = a;
    __syncthreads();
    if (tid < D) {
        double v = s_acc[tid];
        for (int q = 1; q < G; ++q) v += s_acc[q * Dr + tid];
        part[(size_t)blockIdx.x * D + tid] = v;
    }
    __threadfence();
    const bool ok = grid_barrier(bar, (unsigned int)nb, kWaitCycles);

    double v = 0.0;
    if (on)
        for (int b0 = g; b0 < nb; b0 += kSumBatch * G) {
            double t[kSumBatch];
#pragma unroll
            for (int q = 0; q < kSumBatch; ++q) {
                const int b = b0 + q * G;
                t[q] = b < nb ? __ldcg(part + (size_t)b * D + d) : 0.0;
            }
#pragma unroll
            for (int q = 0; q < kSumBatch; ++q) v += t[q];
        }
    s_acc[tid] = v;
    __syncthreads();
    if (tid < D) {
        double m = s_acc[tid];
        for (int q = 1; q < G; ++q) m += s_acc[q * Dr + tid];
        const float hi = (float)m, lo = (float)(m - (double)hi);
        s_hi[tid] = hi;
        s_lo[tid] = lo;
        if (blockIdx.x == 0) {
            mu[tid] = m;
            mu_f[tid] = hi;
            mu_lo[tid] = lo;
        }
    }
    __syncthreads();

    for (int c = blockIdx.x; c < chunks; c += nb) {
        float *chunk = Yp + (size_t)c * chunk_floats(Dp);
        const int ne = min(kChunkE, nu - c * kChunkE);
        for (int e = tid; e < ne * D; e += kEUThreads) {
            const int k = e / D, dd = e - k * D;
            const int j = c * kChunkE + k;
            const float dev = __fsub_rn(__fsub_rn(elites[(size_t)j * D + dd], s_hi[dd]), s_lo[dd]);
            const float y = __fmul_rn(sw[j], dev);
            const float hi = tc::to_tf32(y), lo = tc::to_tf32(__fsub_rn(y, hi));
            const int idx = core_index(dd, k);
            chunk[idx] = hi;
            chunk[Dp * kChunkE + idx] = lo;
        }
    }
    if (!ok && tid == 0 && status != nullptr) atomicOr(status, DEV_ERR_TIMEOUT);
}

// Slice blockIdx.y of the elite chunks, for candidates 128 blockIdx.x ...:
// P[slice][i][d] = sum over the slice's elites j of g_ij Y[j][d].
// Warp-specialised pipeline over stages of 16 elites (two stages in shared memory):
//  - warps 0-7 (256 threads, two per candidate row) write the stage's normals (G_hi, G_lo,
//    8 per thread), make them visible to the tensor cores (proxy fence) and arrive on the
//    stage's a_full barrier, one arrival per warp; before refilling a stage they wait for
//    its done barrier (the MMAs that read it have completed), never for each other;
//  - warp 8 (one elected lane) brings each packed Y chunk in with a bulk copy (b_full),
//    waits for a_full and b_full, issues the stage's 6 MMAs of 128 x Dp x 8 and commits
//    them to done.
// Every wait is bounded: when one runs out the CTA records DEV_ERR_TIMEOUT, goes on
// (results are then meaningless) and still releases its tensor memory. `withhold` issues
// no operand copy, so that the wait for it runs out on purpose (the test of this path).
__global__ void __launch_bounds__(kTcThreads + 32)
k_sample_elites(const float *__restrict__ Yp, int N, int D, int n_chunks, int slices, uint32_t tmem_cols,
                const PhiloxKeys key, uint32_t iter, uint32_t query, float *P, uint32_t *status, int withhold)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t a_full[kStages], b_full[kStages], done[kStages];
    __shared__ uint32_t s_tmem;
    const int Dp = padded_d(D);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTcM, slice = blockIdx.y;
    const int c_begin = (int)((long long)slice * n_chunks / slices);
    const int n = (int)((long long)(slice + 1) * n_chunks / slices) - c_begin;   // >= 1
    const int a_floats = kTcM * kChunkE, b_floats = chunk_floats(Dp);
    const int stage_floats = 2 * a_floats + b_floats;
    const uint32_t b_bytes = 4u * (uint32_t)b_floats;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&a_full[s], kTcThreads / 32);
            tc::mbar_init(&b_full[s], 1);
            tc::mbar_init(&done[s], 1);
        }
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&s_tmem, tmem_cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    bool late = false;

    if (warp == kTcThreads / 32) {
        if (lane == 0) {
            // Once a wait has run out (`late`), the results of the launch are void: the
            // remaining waits are skipped and no further copy is issued, so a failed launch
            // ends after one wait budget instead of one per stage. Copies already issued and
            // not yet seen complete (`pending`, with their phase parity) are waited for,
            // bounded, before the CTA leaves.
            uint32_t pending = 0, pending_par = 0;
            const uint32_t idesc = tc::idesc_tf32(kTcM, Dp);
            for (int it = 0; it < kStages && it < n && !withhold; ++it) {
                float *b_hi = smem + it * stage_floats + 2 * a_floats;
                tc::mbar_expect_tx(&b_full[it], b_bytes);
                tc::bulk_g2s(b_hi, Yp + (size_t)(c_begin + it) * b_floats, b_bytes, &b_full[it]);
                pending |= 1u << it;   // phase parity 0
            }
            for (int it = 0; it < n; ++it) {
                const int s = it % kStages;
                const uint32_t par = (uint32_t)(it / kStages) & 1u;
                float *a_hi = smem + s * stage_floats, *a_lo = a_hi + a_floats, *b_hi = a_lo + a_floats;
                if (!late && !tc::mbar_wait(&a_full[s], par, kWaitCycles)) late = true;
                if (!late) {
                    if (tc::mbar_wait(&b_full[s], par, kWaitCycles)) pending &= ~(1u << s);
                    else late = true;
                }
                tc::fence_after_sync();
                const uint32_t sa_hi = tc::smem_addr(a_hi), sa_lo = tc::smem_addr(a_lo);
                const uint32_t sb_hi = tc::smem_addr(b_hi), sb_lo = sb_hi + 4u * (uint32_t)(Dp * kChunkE);
#pragma unroll
                for (int ks = 0; ks < kChunkE / 8; ++ks) {
                    const uint32_t o = 2 * kCoreLbo * (uint32_t)ks;   // 8 elements of K: two core matrices
                    const uint64_t ah = tc::desc_kmajor(sa_hi + o, kCoreLbo, kCoreSbo);
                    const uint64_t al = tc::desc_kmajor(sa_lo + o, kCoreLbo, kCoreSbo);
                    const uint64_t bh = tc::desc_kmajor(sb_hi + o, kCoreLbo, kCoreSbo);
                    const uint64_t bl = tc::desc_kmajor(sb_lo + o, kCoreLbo, kCoreSbo);
                    tc::mma_tf32(tmem, ah, bh, idesc, it > 0 || ks > 0);
                    tc::mma_tf32(tmem, ah, bl, idesc, true);
                    tc::mma_tf32(tmem, al, bh, idesc, true);
                }
                tc::mma_commit(&done[s]);
                // the chunk two stages on goes where the previous stage's MMAs read
                const int nx = it + 1, sx = nx % kStages;
                if (it >= 1 && nx < n && !withhold && !late) {
                    if (!tc::mbar_wait(&done[sx], ((nx - kStages) / kStages) & 1, kWaitCycles)) {
                        late = true;
                    } else {
                        float *bx = smem + sx * stage_floats + 2 * a_floats;
                        tc::mbar_expect_tx(&b_full[sx], b_bytes);
                        tc::bulk_g2s(bx, Yp + (size_t)(c_begin + nx) * b_floats, b_bytes, &b_full[sx]);
                        pending |= 1u << sx;
                        pending_par = (pending_par & ~(1u << sx)) | ((uint32_t)((nx / kStages) & 1) << sx);
                    }
                }
            }
            for (int s = 0; s < kStages; ++s)   // copies in flight land before the CTA leaves
                if (pending & (1u << s)) tc::mbar_wait(&b_full[s], (pending_par >> s) & 1u, kWaitCycles);
        }
        __syncwarp();
    } else {
        const int r = tid & (kTcM - 1), half = tid >> 7;   // candidate row; Philox blocks 2 half, 2 half + 1
        const bool row_ok = m0 + r < N;
        for (int it = 0; it < n; ++it) {
            const int s = it % kStages;
            float *a_hi = smem + s * stage_floats, *a_lo = a_hi + a_floats;
            const int c = c_begin + it;
            float h[kChunkE / 8][4], l[kChunkE / 8][4];
#pragma unroll
            for (int q = 0; q < kChunkE / 8; ++q) {   // the normals before the wait for the stage
                const int blk = (kChunkE / 8) * half + q;   // elites 4 blk .. 4 blk + 3 of the chunk
                float z[4] = {0.f, 0.f, 0.f, 0.f};
                if (row_ok) {
                    const uint4 x = philox4x32_10(
                        make_uint4((uint32_t)(c * (kChunkE / 4) + blk), (uint32_t)(m0 + r), iter, query), key);
                    box_muller(x.x, x.y, z[0], z[1]);
                    box_muller(x.z, x.w, z[2], z[3]);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    h[q][e] = tc::to_tf32(z[e]);
                    l[q][e] = tc::to_tf32(z[e] - h[q][e]);
                }
            }
            if (it >= kStages && !late && !tc::mbar_wait(&done[s], ((it - kStages) / kStages) & 1, kWaitCycles))
                late = true;
#pragma unroll
            for (int q = 0; q < kChunkE / 8; ++q) {
                const int off = core_index(r, 4 * ((kChunkE / 8) * half + q));
                *reinterpret_cast<float4 *>(a_hi + off) = make_float4(h[q][0], h[q][1], h[q][2], h[q][3]);
                *reinterpret_cast<float4 *>(a_lo + off) = make_float4(l[q][0], l[q][1], l[q][2], l[q][3]);
            }
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&a_full[s]);
        }
    }
    // the last commit covers every MMA of the CTA
    if (!tc::mbar_wait(&done[(n - 1) % kStages], ((n - 1) / kStages) & 1, kWaitCycles)) late = true;
    tc::fence_after_sync();
    if (warp < kTcThreads / 32) {
        // warp w reads lanes 32 (w % 4) .. of tensor memory, columns 16 (w / 4) + 32 k
        const int quarter = warp & 3, cgroup = warp >> 2;
        const int i = m0 + 32 * quarter + lane;
        float *out = P + ((size_t)slice * N + (size_t)(i < N ? i : 0)) * D;
        for (int c0 = 16 * cgroup; c0 < Dp; c0 += 32) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0, v);
            if (i < N) {
#pragma unroll
                for (int g = 0; g < 4; ++g)
                    if (c0 + 4 * g < D)
                        *reinterpret_cast<float4 *>(out + c0 + 4 * g) =
                            make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
            }
        }
    }
    if (late && status != nullptr) atomicOr(status, DEV_ERR_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols);
}

// xi[i][d] = mu_d + sum_s P[s][i][d] (slices in order) + sigma sqrt(eps) g'_id, four
// coordinates per thread: their normals nu + d .. nu + d + 3 come from one Philox block, or
// two when nu is not a multiple of four.
__global__ void k_sample_reduce(const float *__restrict__ P, int slices, const float *__restrict__ mu_f, int N,
                                int D, int nu, float eps_scale, const PhiloxKeys key, uint32_t iter,
                                uint32_t query, float *xi)
{
    const int D4 = D >> 2;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)N * D4) return;
    const int i = (int)(e / D4), d = 4 * (int)(e - (int64_t)i * D4);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s = 0; s < slices; ++s) {
        const float4 p = *reinterpret_cast<const float4 *>(P + ((size_t)s * N + i) * D + d);
        v.x += p.x;
        v.y += p.y;
        v.z += p.z;
        v.w += p.w;
    }
    const uint32_t j0 = (uint32_t)(nu + d), b0 = j0 >> 2, sh = j0 & 3u;
    float g[8];
    uint4 x = philox4x32_10(make_uint4(b0, (uint32_t)i, iter, query), key);
    box_muller(x.x, x.y, g[0], g[1]);
    box_muller(x.z, x.w, g[2], g[3]);
    if (sh != 0) {
        x = philox4x32_10(make_uint4(b0 + 1, (uint32_t)i, iter, query), key);
        box_muller(x.x, x.y, g[4], g[5]);
        box_muller(x.z, x.w, g[6], g[7]);
    }
    float z[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {   // g[sh + k] without dynamic indexing
        const uint32_t t = sh + (uint32_t)k;
        z[k] = t == 0 ? g[0] : t == 1 ? g[1] : t == 2 ? g[2] : t == 3 ? g[3] : t == 4 ? g[4] : t == 5 ? g[5] : g[6];
    }
    const float4 m = *reinterpret_cast<const float4 *>(mu_f + d);
    *reinterpret_cast<float4 *>(xi + (size_t)i * D + d) =
        make_float4(m.x + fmaf(eps_scale, z[0], v.x), m.y + fmaf(eps_scale, z[1], v.y),
                    m.z + fmaf(eps_scale, z[2], v.z), m.w + fmaf(eps_scale, z[3], v.w));
}

}  // namespace

size_t elite_operand_floats(int nu, int D)
{
    return (size_t)((nu + kChunkE - 1) / kChunkE) * chunk_floats(padded_d(D));
}

// Slices of the elite chunks for N candidates: as many CTAs as are resident on the GPU at
// once (the normals dominate the work, so one wave of equal CTAs), at most 32 slices and at
// least one chunk each. Residency follows from the shared memory of a CTA (dynamic, static
// and the driver's reserve) against the SM's, its threads, registers and tensor-memory
// columns.
int elite_slices(int N, int D, int nu, int num_sms)
{
    const int Dp = padded_d(D);
    const size_t smem = tc_smem_bytes(Dp);
    int dev = 0, sm_smem = 0, reserved = 0, sm_threads = 0;
    cudaFuncAttributes fa{};
    int per_sm = 1;
    if (cudaFuncSetAttribute(k_sample_elites, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_sample_elites, cudaFuncAttributePreferredSharedMemoryCarveout, 100) == cudaSuccess &&
        cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sm_threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev) == cudaSuccess &&
        cudaFuncGetAttributes(&fa, k_sample_elites) == cudaSuccess) {
        per_sm = (int)((size_t)sm_smem / (smem + fa.sharedSizeBytes + (size_t)reserved));
        per_sm = std::min(per_sm, sm_threads / (kTcThreads + 32));
        const int warps = (kTcThreads + 32) / 32;   // registers: allocated per warp in units of 256
        const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
        if (regs_per_warp > 0) per_sm = std::min(per_sm, 65536 / (regs_per_warp * warps));
        per_sm = std::min(per_sm, (int)(512u / tmem_columns(Dp)));
        if (per_sm < 1) per_sm = 1;
    } else {
        cudaGetLastError();
    }
    const int tiles = (N + kTcM - 1) / kTcM;
    const int chunks = (nu + kChunkE - 1) / kChunkE;
    int s = per_sm * num_sms / tiles;
    if (s > chunks) s = chunks;
    if (s > CP_ELITE_MAX_SLICES) s = CP_ELITE_MAX_SLICES;
    return s < 1 ? 1 : s;
}

int launch_elite_weights(const double *w, int nu, double sigma, float *sw, cudaStream_t st)
{
    k_elite_weights<<<(nu + 255) / 256, 256, 0, st>>>(w, nu, sigma, sw);
    CP_LAUNCHED("k_elite_weights");
    return CP_OK;
}

// Blocks of k_elite_update: one per chunk of 16 elites, at most one per two SMs (fewer
// partials to add after the barrier), so that all are resident at once.
int elite_update_blocks(int nu, int num_sms)
{
    const int chunks = (nu + kChunkE - 1) / kChunkE;
    const int cap = num_sms / 2 > 0 ? num_sms / 2 : 1;
    return chunks < cap ? chunks : cap;
}

int launch_elite_update(const float *elites, const double *w, const float *sw, int nu, int D, int blocks,
                        double *part, unsigned int *bar, double *mu, float *mu_f, float *mu_lo, float *Yp,
                        uint32_t *status, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kEUThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CP_CUDA(cudaLaunchKernelEx(&cfg, k_elite_update, elites, w, sw, nu, D, part, bar, mu, mu_f, mu_lo, Yp, status));
    CP_LAUNCHED("k_elite_update");
    return CP_OK;
}

int launch_sample_elites(const float *Yp, const float *mu_f, int N, int K, int nu, int slices, double sigma,
                         double eps, uint64_t seed, uint32_t iter, uint32_t query, float *P, float *xi,
                         uint32_t *status, bool withhold, cudaStream_t st)
{
    const int D = 4 * K, Dp = padded_d(D);
    const int chunks = (nu + kChunkE - 1) / kChunkE;
    if (slices > chunks) slices = chunks;
    const PhiloxKeys key = philox_keys((uint32_t)seed, (uint32_t)(seed >> 32));
    dim3 grid((N + kTcM - 1) / kTcM, slices);
    k_sample_elites<<<grid, kTcThreads + 32, tc_smem_bytes(Dp), st>>>(Yp, N, D, chunks, slices, tmem_columns(Dp), key,
                                                                  iter, query, P, status, withhold ? 1 : 0);
    CP_LAUNCHED("k_sample_elites");
    const int64_t total = (int64_t)N * (D / 4);
    k_sample_reduce<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, slices, mu_f, N, D, nu,
                                                                     (float)(sigma * sqrt(eps)), key, iter,
                                                                     query, xi);
    CP_LAUNCHED("k_sample_reduce");
    return CP_OK;
}

}  // namespace cp
