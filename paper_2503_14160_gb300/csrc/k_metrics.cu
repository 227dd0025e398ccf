// Per-iteration metrics of Algorithm 1 (arXiv 2503.14160, Sec. 4.1), taken after steps
// (3)-(6) of an iteration: the best cost of the population, its mean cost, the trace of
// the updated covariance C and the fraction of candidates without a checkpoint in collision.
// kMetricsBlocks blocks each sum a fixed range of the candidates and of the elite entries
// (per-thread strided sums, then a fixed shuffle tree and the warps' sums in warp order);
// one thread then adds the blocks' partials in block order. The row is deterministic.
#include "cp_internal.cuh"

namespace cp {
namespace {

constexpr int kMetricsThreads = 256;

__device__ __forceinline__ double block_sum(double v, double *s_part)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) s_part[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kMetricsThreads / 32; ++w) t += s_part[w];
    return t;
}

// Block b: sums over its range of the candidates (J, collision-free count) and of tr C:
// the diagonal of C (block 0) or, when C is not formed (the factor-free sampler), the elite
// entries of its range about the new mean, w_j (x_(j),r - mu_r)^2. part[3 b .. 3 b + 2].
__global__ void __launch_bounds__(kMetricsThreads)
k_iter_metrics_part(const double *__restrict__ J, const uint8_t *__restrict__ flag, int N,
                    const double *__restrict__ C, const float *__restrict__ elites, const double *__restrict__ w,
                    const double *__restrict__ mu, int nu, int D, double *part)
{
    __shared__ double s_part[kMetricsThreads / 32];
    const int b = blockIdx.x;
    const int n_per = (N + kMetricsBlocks - 1) / kMetricsBlocks;
    const int i0 = b * n_per, i1 = min(N, i0 + n_per);
    double js = 0.0, fr = 0.0, tr = 0.0;
    for (int i = i0 + (int)threadIdx.x; i < i1; i += kMetricsThreads) {
        js += J[i];
        fr += flag[i] == 0 ? 1.0 : 0.0;
    }
    if (C != nullptr) {
        if (b == 0)
            for (int r = threadIdx.x; r < D; r += kMetricsThreads) tr += C[(size_t)r * D + r];
    } else {
        const int total = nu * D, e_per = (total + kMetricsBlocks - 1) / kMetricsBlocks;
        const int e0 = b * e_per, e1 = min(total, e0 + e_per);
        for (int idx = e0 + (int)threadIdx.x; idx < e1; idx += kMetricsThreads) {
            const int j = idx / D, r = idx - j * D;
            const double d = (double)elites[idx] - mu[r];
            tr = fma(w[j] * d, d, tr);
        }
    }
    js = block_sum(js, s_part);
    fr = block_sum(fr, s_part);
    tr = block_sum(tr, s_part);
    if (threadIdx.x == 0) {
        part[3 * b] = js;
        part[3 * b + 1] = fr;
        part[3 * b + 2] = tr;
    }
}

// row = {iteration, best J, mean J, tr C, collision-free fraction} from the blocks' partials
// (with D eps added to the elites' scatter when C is not formed).
__global__ void k_iter_metrics(const double *__restrict__ part, const double *__restrict__ best, int N, int D,
                               double eps, int have_C, int iteration, double *row)
{
    if (threadIdx.x != 0) return;
    double js = 0.0, fr = 0.0, tr = 0.0;
    for (int b = 0; b < kMetricsBlocks; ++b) {
        js += part[3 * b];
        fr += part[3 * b + 1];
        tr += part[3 * b + 2];
    }
    row[0] = (double)iteration;
    row[1] = *best;
    row[2] = js / N;
    row[3] = have_C ? tr : tr + D * eps;
    row[4] = fr / N;
}

}  // namespace

int launch_iter_metrics(const double *J, const uint8_t *flag, int N, const double *best, const double *C,
                        const float *elites, const double *w, const double *mu, int nu, int D, double eps,
                        int iteration, double *part, double *row, cudaStream_t st)
{
    k_iter_metrics_part<<<kMetricsBlocks, kMetricsThreads, 0, st>>>(J, flag, N, C, elites, w, mu, nu, D, part);
    CP_LAUNCHED("k_iter_metrics_part");
    k_iter_metrics<<<1, 32, 0, st>>>(part, best, N, D, eps, C != nullptr ? 1 : 0, iteration, row);
    CP_LAUNCHED("k_iter_metrics");
    return CP_OK;
}

}  // namespace cp
