// Algorithm 1 step (1): xi_i ~ N(mu, sigma^2 C) (arXiv 2503.14160, Sec. 4.1).
//   k_factor  L L^T = sigma^2 C, FP64 right-looking Cholesky (L D L^T form) in one CTA, D <= 128
//   k_sample  z_i from Philox4x32-10 (Salmon et al., SC'11) + Box-Muller, xi_i = mu + L z_i
// The counter of candidate i, block j, iteration t, query q is (j, i, t, q); the key is
// the 64-bit seed split into two words. Block j gives the normals z[4j..4j+3].
#include "cp_internal.cuh"
#include "philox.cuh"

namespace cp {
namespace {

__global__ void k_philox(const uint4 *__restrict__ ctr, uint32_t k0, uint32_t k1, int64_t n,
                         uint4 *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], k0, k1);
}

constexpr int kFactorThreads = 1024;
constexpr int kFactorMaxD = 4 * CP_MAX_WAYPOINTS;

// 1/a and 1/sqrt(a) for a > 0: a float seed refined by two Newton-Raphson steps in FP64
// (quadratic convergence: 23 -> 46 -> 92 bits). On a part with a narrow FP64 pipe these
// short chains are much faster than a library division or square root. Arguments whose
// float conversion is not a normal number take the IEEE operations instead.
__device__ __forceinline__ double recip_newton(double a)
{
    const float af = (float)a;
    if (!(af > 1e-30f && af < 1e30f)) return 1.0 / a;
    double y = (double)__frcp_rn(af);
    y = fma(y, fma(-a, y, 1.0), y);
    y = fma(y, fma(-a, y, 1.0), y);
    return y;
}

__device__ __forceinline__ double rsqrt_newton(double a)
{
    const float af = (float)a;
    if (!(af > 1e-30f && af < 1e30f)) return 1.0 / sqrt(a);
    double y = (double)rsqrtf(af);
    const double h = 0.5 * a;
    y = y * fma(-h * y, y, 1.5);
    y = y * fma(-h * y, y, 1.5);
    return y;
}

// One CTA, right-looking Cholesky of A = sigma^2 C in shared memory (row stride D + 1) in
// the unscaled (L D L^T) form: step k takes t_i = a_ik / a_kk for the rows below the pivot,
// then a_ij -= t_i a_jk over the trailing lower triangle, one FMA per entry and every lane
// busy. The next pivot's reciprocal is the critical chain of every column; the FP64 pipe is
// narrow, so that chain runs alone on one scheduler: warps are dealt to the SM's four
// schedulers round robin, warp 0 computes a_{k+1,k+1} and its reciprocal (double
// buffered), and the bulk update runs on the warps of the other three schedulers. At the
// end column k holds a_ik = l_ik sqrt(a_kk), so l_ik = a_ik / sqrt(a_kk) with the D square
// roots taken together. Outputs L (double, row-major, upper part zero) and its FP32
// transpose Lt[c][r] = L[r][c] for the sampler. A pivot that is not positive raises
// DEV_ERR_NOT_PD (and is replaced by 1 so that the kernel finishes).
__device__ __forceinline__ void factor_body(const double *__restrict__ C, double sigma2, int D, double *L,
                                            float *Lt, uint32_t *status, double *A)
{
    __shared__ double s_d[2];
    __shared__ double s_t[kFactorMaxD];
    __shared__ int bad;
    const int ld = D + 1;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const bool worker = (warp & 3) != 0;
    const int wtid = ((warp >> 2) * 3 + (warp & 3) - 1) * 32 + lane;   // 0 .. 3/4 blockDim - 1
    const int wcount = (int)blockDim.x / 4 * 3;
    for (int idx = tid; idx < D * D; idx += blockDim.x) {
        const int r = idx / D, c = idx - r * D;
        if (c <= r) A[r * ld + c] = sigma2 * C[idx];
    }
    __syncthreads();
    if (tid == 0) {
        bad = 0;
        double a = A[0];
        if (!(a > 0.0)) {
            bad = 1;
            a = 1.0;
            A[0] = a;
        }
        s_d[0] = recip_newton(a);
    }
    __syncthreads();
    for (int k = 0; k + 1 < D; ++k) {
        const int T = D - k - 1;
        const double d = s_d[k & 1];
        if (worker)
            for (int i = wtid; i < T; i += wcount) s_t[i] = A[(k + 1 + i) * ld + k] * d;
        __syncthreads();
        if (worker) {
            const int E = T * (T + 1) / 2;
            for (int e = wtid + 1; e < E; e += wcount) {   // entry 0 is the pivot
                int ii, jj;
                tri_index(e, ii, jj);
                const int i = k + 1 + ii, j = k + 1 + jj;
                A[i * ld + j] = fma(-s_t[ii], A[j * ld + k], A[i * ld + j]);
            }
        } else if (tid == 0) {
            const int i = k + 1;
            double v = fma(-(A[i * ld + k] * d), A[i * ld + k], A[i * ld + i]);
            if (!(v > 0.0)) {
                bad = 1;
                v = 1.0;
            }
            A[i * ld + i] = v;
            s_d[(k + 1) & 1] = recip_newton(v);
        }
        __syncthreads();
    }
    for (int k = tid; k < D; k += blockDim.x) s_t[k] = rsqrt_newton(A[k * ld + k]);
    __syncthreads();
    for (int idx = tid; idx < D * D; idx += blockDim.x) {
        const int r = idx / D, c = idx - r * D;
        const double l = c <= r ? A[r * ld + c] * s_t[c] : 0.0;
        L[idx] = l;
        Lt[c * D + r] = (float)l;
    }
    __syncthreads();
    if (tid == 0 && bad) atomicOr(status, DEV_ERR_NOT_PD);
}

__global__ void __launch_bounds__(kFactorThreads)
k_factor(const double *__restrict__ C, double sigma2, const double *__restrict__ sigma_dev, int D, double *L,
         float *Lt, uint32_t *status)
{
    if (sigma_dev != nullptr) sigma2 = sigma_dev[0] * sigma_dev[0];   // the step size kept on the device
    extern __shared__ double A[];
    factor_body(C, sigma2, D, L, Lt, status, A);
}

// The factors of every query of a batch, one CTA per query.
__global__ void __launch_bounds__(kFactorThreads) k_batch_factor(const BatchQueryDev *__restrict__ qd)
{
    extern __shared__ double A[];
    const BatchQueryDev &q = qd[blockIdx.x];
    factor_body(q.C, q.sigma2, q.D, q.L, q.Lt, q.status, A);
}

constexpr int kSampleWarps = 8;
constexpr int kSampleThreads = 32 * kSampleWarps;
constexpr int kSampleCands = 8;   // candidates a warp draws at a time

// Shared memory of the sampler: L^T (FP32, column-major, D x D, plus a pad of 32 floats read
// by the lanes past the last row) and per warp the normals of its kSampleCands candidates
// ([D][kSampleCands], candidate fastest).
size_t sample_smem(int K)
{
    const size_t D = 4 * (size_t)K;
    return sizeof(float) * (D * D + 32 + (size_t)kSampleWarps * kSampleCands * D);
}

// Warp w draws the candidates g .. g + 7 of the groups g = g0 + 8 w, g0 + 8 w + g_stride, ...
// below i_end: their normals (Philox counter (j, i, iter, query) for z[4j..4j+3], spread over
// the lanes) go to the warp's buffer; then, 32 rows at a time, lane l holds row r = r0 + l of
// all eight and forms acc = sum_c L[r][c] z[c] over ascending c with one FMA per term (L read
// once for the eight), and writes xi_r = mu_r + acc (added in FP64, rounded once to FP32).
// Columns past the block's last row hold zeros of L for every row of the block and are
// skipped; adding 0 z leaves a nonzero sum unchanged, so each row equals the full D-term sum.
__device__ __forceinline__ void sample_body(const double *__restrict__ mu, const float *__restrict__ Lt, int K,
                                            uint32_t k0, uint32_t k1, uint32_t iter, uint32_t query,
                                            float *xi, int g0, int g_stride, int i_end, float *sm)
{
    const int D = 4 * K;
    float *sL = sm;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *sZ = sm + D * D + 32 + wib * kSampleCands * D;
    for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) sL[idx] = Lt[idx];
    if (threadIdx.x < 32) sL[D * D + threadIdx.x] = 0.f;
    __syncthreads();
    for (int g = g0 + kSampleCands * wib; g < i_end; g += g_stride) {
        for (int pq = lane; pq < kSampleCands * K; pq += 32) {
            const int cnd = pq % kSampleCands, j = pq / kSampleCands;
            const int i = g + cnd;
            float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
            if (i < i_end) {
                const uint4 x = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)i, iter, query), k0, k1);
                box_muller(x.x, x.y, z0, z1);
                box_muller(x.z, x.w, z2, z3);
            }
            sZ[(4 * j + 0) * kSampleCands + cnd] = z0;
            sZ[(4 * j + 1) * kSampleCands + cnd] = z1;
            sZ[(4 * j + 2) * kSampleCands + cnd] = z2;
            sZ[(4 * j + 3) * kSampleCands + cnd] = z3;
        }
        __syncwarp();
        for (int r0 = 0; r0 < D; r0 += 32) {
            const int r = r0 + lane;
            float acc[kSampleCands];
#pragma unroll
            for (int q = 0; q < kSampleCands; ++q) acc[q] = 0.f;
            const int c_last = min(D, r0 + 32);
            for (int c = 0; c < c_last; ++c) {
                const float l = sL[c * D + r];
                const float4 za = *reinterpret_cast<const float4 *>(sZ + c * kSampleCands);
                const float4 zb = *reinterpret_cast<const float4 *>(sZ + c * kSampleCands + 4);
                acc[0] = fmaf(l, za.x, acc[0]);
                acc[1] = fmaf(l, za.y, acc[1]);
                acc[2] = fmaf(l, za.z, acc[2]);
                acc[3] = fmaf(l, za.w, acc[3]);
                acc[4] = fmaf(l, zb.x, acc[4]);
                acc[5] = fmaf(l, zb.y, acc[5]);
                acc[6] = fmaf(l, zb.z, acc[6]);
                acc[7] = fmaf(l, zb.w, acc[7]);
            }
            if (r < D) {
                const double m = mu[r];
#pragma unroll
                for (int q = 0; q < kSampleCands; ++q)
                    if (g + q < i_end) xi[(size_t)(g + q) * D + r] = (float)(m + (double)acc[q]);
            }
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kSampleThreads)
k_sample(const double *__restrict__ mu, const float *__restrict__ Lt, int N, int K,
         uint32_t k0, uint32_t k1, uint32_t iter, uint32_t query, float *xi)
{
    extern __shared__ __align__(16) float sm[];
    const int per_block = kSampleWarps * kSampleCands;
    sample_body(mu, Lt, K, k0, k1, iter, query, xi, blockIdx.x * per_block, gridDim.x * per_block, N, sm);
}

// Every query's draw in one launch: block b of query q takes the kBatchSampleCands
// candidates from b kBatchSampleCands, each warp several groups of kSampleCands in turn (the
// block stages the query's factor once for all of them). A candidate's normals and
// arithmetic do not depend on which warp draws it, so each query's xi equals its plain draw.
__global__ void __launch_bounds__(kSampleThreads)
k_batch_sample(const BatchQueryDev *__restrict__ qd, const int2 *__restrict__ tab, uint32_t iter)
{
    extern __shared__ __align__(16) float sm[];
    const int2 e = tab[blockIdx.x];
    const BatchQueryDev &q = qd[e.x];
    const int b = e.y * kBatchSampleCands;
    static_assert(kBatchSampleCands % (kSampleWarps * kSampleCands) == 0, "whole groups of candidates per warp");
    sample_body(q.mu, q.Lt, q.K, q.seed_lo, q.seed_hi, iter, q.query, q.xi, b, kSampleWarps * kSampleCands,
                min(q.N, b + kBatchSampleCands), sm);
}

}  // namespace

int launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t *out,
                  cudaStream_t st)
{
    if (n == 0) return CP_OK;
    const int threads = 256;
    const int64_t blocks = (n + threads - 1) / threads;
    k_philox<<<(unsigned)blocks, threads, 0, st>>>((const uint4 *)ctr, k0, k1, n, (uint4 *)out);
    CP_LAUNCHED("k_philox");
    return CP_OK;
}

int factor_configure()
{
    const int Dm = 4 * CP_MAX_WAYPOINTS;
    const int max_smem = (int)(sizeof(double) * Dm * (Dm + 1));
    CP_CUDA(cudaFuncSetAttribute(k_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    return CP_OK;
}

int launch_factor(const double *C, double sigma2, const double *sigma_dev, int D, double *L,
                  float *Lt_f, uint32_t *status, cudaStream_t st)
{
    const size_t smem = sizeof(double) * (size_t)D * (D + 1);
    k_factor<<<1, kFactorThreads, smem, st>>>(C, sigma2, sigma_dev, D, L, Lt_f, status);
    CP_LAUNCHED("k_factor");
    return CP_OK;
}

int sample_configure()
{
    CP_CUDA(cudaFuncSetAttribute(k_sample, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sample_smem(CP_MAX_WAYPOINTS)));
    CP_CUDA(cudaFuncSetAttribute(k_batch_sample, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sample_smem(CP_MAX_WAYPOINTS)));
    const int Dm = 4 * CP_MAX_WAYPOINTS;
    CP_CUDA(cudaFuncSetAttribute(k_batch_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(double) * Dm * (Dm + 1))));
    return CP_OK;
}

int launch_batch_factor(const BatchQueryDev *qd, int nq, int max_D, cudaStream_t st)
{
    const size_t smem = sizeof(double) * (size_t)max_D * (max_D + 1);
    k_batch_factor<<<nq, kFactorThreads, smem, st>>>(qd);
    CP_LAUNCHED("k_batch_factor");
    return CP_OK;
}

int launch_batch_sample(const BatchQueryDev *qd, const int2 *tab, int blocks, int max_K, uint32_t iter,
                        cudaStream_t st)
{
    if (blocks == 0) return CP_OK;
    k_batch_sample<<<blocks, kSampleThreads, sample_smem(max_K), st>>>(qd, tab, iter);
    CP_LAUNCHED("k_batch_sample");
    return CP_OK;
}

int launch_sample(const double *mu, const float *Lt_f, int N, int K, uint64_t seed,
                  uint32_t iter, uint32_t query, float *xi, cudaStream_t st)
{
    int dev = 0, sms = 0, per_sm = 0;
    CP_CUDA(cudaGetDevice(&dev));
    CP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = sample_smem(K);
    CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sample, kSampleThreads, smem));
    if (per_sm < 1) per_sm = 1;
    int blocks = (N + kSampleWarps * kSampleCands - 1) / (kSampleWarps * kSampleCands);
    if (blocks > sms * per_sm) blocks = sms * per_sm;
    k_sample<<<blocks, kSampleThreads, smem, st>>>(mu, Lt_f, N, K, (uint32_t)seed,
                                                   (uint32_t)(seed >> 32), iter, query, xi);
    CP_LAUNCHED("k_sample");
    return CP_OK;
}

}  // namespace cp
