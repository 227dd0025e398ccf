// Per-iteration metrics of Algorithm 1 (arXiv 2503.14160, Sec. 4.1), taken after steps
// (3)-(6) of an iteration: the best cost of the population, its mean cost, the trace of
// the updated covariance C and the fraction of candidates without a checkpoint in collision.
// One CTA; the sums are taken in a fixed order (per-thread strided sums, then a fixed
// shuffle tree and the warps' sums in warp order), so the row is deterministic.
#include "cp_internal.cuh"

namespace cp {
namespace {

constexpr int kMetricsThreads = 1024;

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

// row = {iteration, best J, mean J, tr C, collision-free fraction}. tr C from C itself, or,
// when C is not formed (the factor-free sampler), from the elites about the new mean:
// sum_j w_j |x_(j) - mu|^2 + D eps.
__global__ void __launch_bounds__(kMetricsThreads)
k_iter_metrics(const double *__restrict__ J, const uint8_t *__restrict__ flag, int N, const double *__restrict__ best,
               const double *__restrict__ C, const float *__restrict__ elites, const double *__restrict__ w,
               const double *__restrict__ mu, int nu, int D, double eps, int iteration, double *row)
{
    __shared__ double s_part[kMetricsThreads / 32];
    double js = 0.0, fr = 0.0, tr = 0.0;
    for (int i = threadIdx.x; i < N; i += kMetricsThreads) {
        js += J[i];
        fr += flag[i] == 0 ? 1.0 : 0.0;
    }
    if (C != nullptr) {
        for (int r = threadIdx.x; r < D; r += kMetricsThreads) tr += C[(size_t)r * D + r];
    } else {
        for (int idx = threadIdx.x; idx < nu * D; idx += kMetricsThreads) {
            const int j = idx / D, r = idx - j * D;
            const double d = (double)elites[idx] - mu[r];
            tr = fma(w[j] * d, d, tr);
        }
    }
    js = block_sum(js, s_part);
    fr = block_sum(fr, s_part);
    tr = block_sum(tr, s_part);
    if (threadIdx.x == 0) {
        row[0] = (double)iteration;
        row[1] = *best;
        row[2] = js / N;
        row[3] = C != nullptr ? tr : tr + D * eps;
        row[4] = fr / N;
    }
}

}  // namespace

int launch_iter_metrics(const double *J, const uint8_t *flag, int N, const double *best, const double *C,
                        const float *elites, const double *w, const double *mu, int nu, int D, double eps,
                        int iteration, double *row, cudaStream_t st)
{
    k_iter_metrics<<<1, kMetricsThreads, 0, st>>>(J, flag, N, best, C, elites, w, mu, nu, D, eps, iteration, row);
    CP_LAUNCHED("k_iter_metrics");
    return CP_OK;
}

}  // namespace cp
