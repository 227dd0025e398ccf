// Step (1) of Algorithm 1 drawn from the elites of the last update, with no factor
// (arXiv 2503.14160, Sec. 4.1). With C = sum_j w_j (x_(j) - mu)(x_(j) - mu)^T + eps I (steps
// (5)-(6), mu the new mean)
//     xi_i = mu + sigma (sum_j sqrt(w_j) (x_(j) - mu) g_ij + sqrt(eps) g'_i)
// is normal with mean mu and covariance sigma^2 C exactly, so the FP64 moments and the FP64
// Cholesky factor (whose dependent chains are slow on this part) leave the iteration; the
// draw is the product G Y of N x nu normals and the nu x D scaled elite deviations, a dense
// contraction that runs on the tensor cores.
//   k_elite_weights  sigma sqrt(w_j), once per planner
//   k_elite_mean     mu (FP64, about the best elite, fixed order) and Y[j][d] =
//                    sigma sqrt(w_j) (x_(j)d - mu_d), rounded to FP32 and split into two TF32
//                    parts Y = Y_hi + Y_lo, written in the tensor cores' operand layout
//   k_sample_elites  partial products over a slice of the elites on the tensor cores
//                    (tcgen05, kind::tf32): a CTA takes 128 candidates and all D coordinates,
//                    its 256 threads generate the normals of 16 elites per pipeline stage
//                    (Philox blocks in place, split G = G_hi + G_lo) into shared memory
//                    while the previous stage's MMAs run; the accumulator lives in tensor
//                    memory. G Y is formed as G_hi Y_hi + G_hi Y_lo + G_lo Y_hi ("3xTF32":
//                    each product within 3 * 2^-22 of the FP32 product, FP32 accumulation)
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
constexpr int kTcThreads = 256;    // two threads per candidate row
constexpr int kStages = 2;
constexpr long long kWaitCycles = 2000000000ll;   // about one second at 2 GHz

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

__global__ void k_elite_weights(const double *__restrict__ w, int nu, double sigma, double *sw)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nu) sw[k] = sigma * sqrt(w[k]);
}

// One block per coordinate d: mu_d = x_(1)d + sum_j w_j (x_(j)d - x_(1)d), then the row d of
// the packed operand (Y_hi, Y_lo per chunk of 16 elites). The sum runs over the elites in a
// fixed partition (thread t takes j = t, t + 256, ...) and a fixed reduction tree. Rows
// d >= D and elites past nu of the packed operand stay zero (the buffer is cleared once).
__global__ void __launch_bounds__(256)
k_elite_mean(const float *__restrict__ elites, const double *__restrict__ w, const double *__restrict__ sw,
             int nu, int D, double *mu, float *mu_f, float *Yp)
{
    __shared__ double s_part[8];
    __shared__ double s_mu;
    const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const double x1 = (double)elites[d];
    double a0 = 0.0, a1 = 0.0;
    int j = tid;
    for (; j + 256 < nu; j += 512) {
        a0 = fma(w[j], (double)elites[(size_t)j * D + d] - x1, a0);
        a1 = fma(w[j + 256], (double)elites[(size_t)(j + 256) * D + d] - x1, a1);
    }
    if (j < nu) a0 = fma(w[j], (double)elites[(size_t)j * D + d] - x1, a0);
    double v = a0 + a1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) s_part[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int k = 0; k < 8; ++k) sum += s_part[k];
        s_mu = x1 + sum;
        mu[d] = s_mu;
        mu_f[d] = (float)s_mu;
    }
    __syncthreads();
    const double m = s_mu;
    const int Dp = padded_d(D);
    for (int k = tid; k < nu; k += 256) {
        const float y = (float)(sw[k] * ((double)elites[(size_t)k * D + d] - m));
        const float hi = tc::to_tf32(y), lo = tc::to_tf32(y - hi);
        float *chunk = Yp + (size_t)(k / kChunkE) * chunk_floats(Dp);
        const int idx = core_index(d, k % kChunkE);
        chunk[idx] = hi;
        chunk[Dp * kChunkE + idx] = lo;
    }
}

// Slice blockIdx.y of the elite chunks, for candidates 128 blockIdx.x ...:
// P[slice][i][d] = sum over the slice's elites j of g_ij Y[j][d].
// Per stage (16 elites): thread 0 brings the packed Y chunk in with one bulk copy, every
// thread writes 8 normals of its candidate row (G_hi, G_lo) into the stage, and after a
// barrier thread 0 issues 6 MMAs of 128 x Dp x 8 and commits them to the stage's barrier;
// a stage is refilled once that barrier reports its MMAs done. Every wait is bounded: when
// one runs out the CTA records DEV_ERR_TIMEOUT, goes on (results are then meaningless) and
// still releases its tensor memory.
__global__ void __launch_bounds__(kTcThreads)
k_sample_elites(const float *__restrict__ Yp, int N, int D, int n_chunks, int slices, uint32_t tmem_cols,
                uint32_t k0, uint32_t k1, uint32_t iter, uint32_t query, float *P, uint32_t *status)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t full[kStages], done[kStages];
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
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&done[s], 1);
        }
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&s_tmem, tmem_cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;

    const int r = tid & (kTcM - 1), half = tid >> 7;   // candidate row; Philox blocks 2 half, 2 half + 1
    const bool row_ok = m0 + r < N;
    const uint32_t idesc = tc::idesc_tf32(kTcM, Dp);
    bool late = false;
    for (int it = 0; it < n; ++it) {
        const int s = it % kStages;
        float *a_hi = smem + s * stage_floats, *a_lo = a_hi + a_floats, *b_hi = a_lo + a_floats;
        if (it >= kStages && !tc::mbar_wait(&done[s], ((it - kStages) / kStages) & 1, kWaitCycles)) late = true;
        const int c = c_begin + it;
        if (tid == 0) {
            tc::mbar_expect_tx(&full[s], b_bytes);
            tc::bulk_g2s(b_hi, Yp + (size_t)c * b_floats, b_bytes, &full[s]);
        }
#pragma unroll
        for (int q = 0; q < kChunkE / 8; ++q) {
            const int blk = (kChunkE / 8) * half + q;   // elites 4 blk .. 4 blk + 3 of the chunk
            float z[4] = {0.f, 0.f, 0.f, 0.f};
            if (row_ok) {
                const uint4 x = philox4x32_10(
                    make_uint4((uint32_t)(c * (kChunkE / 4) + blk), (uint32_t)(m0 + r), iter, query), k0, k1);
                box_muller(x.x, x.y, z[0], z[1]);
                box_muller(x.z, x.w, z[2], z[3]);
            }
            float h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                h[e] = tc::to_tf32(z[e]);
                l[e] = tc::to_tf32(z[e] - h[e]);
            }
            const int off = core_index(r, 4 * blk);
            *reinterpret_cast<float4 *>(a_hi + off) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4 *>(a_lo + off) = make_float4(l[0], l[1], l[2], l[3]);
        }
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            if (!tc::mbar_wait(&full[s], (it / kStages) & 1, kWaitCycles)) late = true;
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
        }
    }
    // the last commit covers every MMA of the CTA
    if (!tc::mbar_wait(&done[(n - 1) % kStages], ((n - 1) / kStages) & 1, kWaitCycles)) late = true;
    tc::fence_after_sync();
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
    if (late && status != nullptr) atomicOr(status, DEV_ERR_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols);
}

// xi[i][d] = mu_d + sum_s P[s][i][d] (slices in order) + sigma sqrt(eps) g'_id, four
// coordinates per thread: their normals nu + d .. nu + d + 3 come from one Philox block, or
// two when nu is not a multiple of four.
__global__ void k_sample_reduce(const float *__restrict__ P, int slices, const float *__restrict__ mu_f, int N,
                                int D, int nu, float eps_scale, uint32_t k0, uint32_t k1, uint32_t iter,
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
    uint4 x = philox4x32_10(make_uint4(b0, (uint32_t)i, iter, query), k0, k1);
    box_muller(x.x, x.y, g[0], g[1]);
    box_muller(x.z, x.w, g[2], g[3]);
    if (sh != 0) {
        x = philox4x32_10(make_uint4(b0 + 1, (uint32_t)i, iter, query), k0, k1);
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
// and the driver's reserve) against the SM's, its threads and its tensor-memory columns.
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
        per_sm = std::min(per_sm, sm_threads / kTcThreads);
        per_sm = std::min(per_sm, (int)(512u / tmem_columns(Dp)));
        if (per_sm < 1) per_sm = 1;
    } else {
        cudaGetLastError();
    }
    const int tiles = (N + kTcM - 1) / kTcM;
    const int chunks = (nu + kChunkE - 1) / kChunkE;
    int s = per_sm * num_sms / tiles;
    if (s > chunks) s = chunks;
    if (s > 32) s = 32;
    return s < 1 ? 1 : s;
}

int launch_elite_weights(const double *w, int nu, double sigma, double *sw, cudaStream_t st)
{
    k_elite_weights<<<(nu + 255) / 256, 256, 0, st>>>(w, nu, sigma, sw);
    CP_LAUNCHED("k_elite_weights");
    return CP_OK;
}

int launch_elite_mean(const float *elites, const double *w, const double *sw, int nu, int D, double *mu, float *mu_f,
                      float *Yp, cudaStream_t st)
{
    k_elite_mean<<<D, 256, 0, st>>>(elites, w, sw, nu, D, mu, mu_f, Yp);
    CP_LAUNCHED("k_elite_mean");
    return CP_OK;
}

int launch_sample_elites(const float *Yp, const float *mu_f, int N, int K, int nu, int slices, double sigma,
                         double eps, uint64_t seed, uint32_t iter, uint32_t query, float *P, float *xi,
                         uint32_t *status, cudaStream_t st)
{
    const int D = 4 * K, Dp = padded_d(D);
    const int chunks = (nu + kChunkE - 1) / kChunkE;
    if (slices > chunks) slices = chunks;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    dim3 grid((N + kTcM - 1) / kTcM, slices);
    k_sample_elites<<<grid, kTcThreads, tc_smem_bytes(Dp), st>>>(Yp, N, D, chunks, slices, tmem_columns(Dp), k0,
                                                                  k1, iter, query, P, status);
    CP_LAUNCHED("k_sample_elites");
    const int64_t total = (int64_t)N * (D / 4);
    k_sample_reduce<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, slices, mu_f, N, D, nu,
                                                                     (float)(sigma * sqrt(eps)), k0, k1, iter,
                                                                     query, xi);
    CP_LAUNCHED("k_sample_reduce");
    return CP_OK;
}

}  // namespace cp
