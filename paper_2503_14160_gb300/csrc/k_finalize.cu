// The last part of Algorithm 1 step (2): per candidate, the FP64 sums of its work items
// (J_p, the penetration sum, J_l, the path length, and the count of checkpoints in
// collision) added in item order into J = J_p + w_c lambda_c sum_k pen_k + w_l J_l
// (Eq. path opt; arXiv 2503.14160, Sec. 4.1). One thread per candidate; the order of the
// additions is fixed, so results are deterministic.
#include "cp_internal.cuh"

namespace cp {
namespace {

__device__ __forceinline__ void finalize_body(const double *__restrict__ item_sum,
                                              const uint32_t *__restrict__ item_count, int n, int P, double w_c,
                                              double w_l, double lambda_c, double *J, uint8_t *flag, double *terms,
                                              const uint32_t *status, int i)
{
    if (i >= n) return;
    const double *row = item_sum + (size_t)i * P * 4;
    const uint32_t *crow = item_count + (size_t)i * P;
    double jp = 0.0, jc = 0.0, jl = 0.0, len = 0.0;
    uint32_t n_flagged = 0;
    for (int p = 0; p < P; ++p) {
        jp += row[4 * p];
        jc += row[4 * p + 1];
        jl += row[4 * p + 2];
        len += row[4 * p + 3];
        n_flagged += crow[p];
    }
    jc *= lambda_c;
    double Ji = jp + w_c * jc + w_l * jl;
    uint8_t fl = n_flagged > 0 ? 1 : 0;
    if (status != nullptr && *status != 0u) {
        // the evaluation gave up on a bounded wait: some item sums are stale, so no result
        // of this call is valid (NaN cost, flagged)
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        jp = jc = jl = len = Ji = nan;
        fl = 1;
    }
    J[i] = Ji;
    if (flag != nullptr) flag[i] = fl;
    if (terms != nullptr) {
        double *tm = terms + (size_t)i * 5;
        tm[0] = jp;
        tm[1] = jc;
        tm[2] = jl;
        tm[3] = len;
        tm[4] = (double)n_flagged;
    }
}

__global__ void __launch_bounds__(256)
k_eval_finalize(const double *__restrict__ item_sum, const uint32_t *__restrict__ item_count, int n, int P,
                double w_c, double w_l, double lambda_c, double *J, uint8_t *flag, double *terms,
                const uint32_t *status)
{
    finalize_body(item_sum, item_count, n, P, w_c, w_l, lambda_c, J, flag, terms, status,
                  blockIdx.x * blockDim.x + threadIdx.x);
}

// Every query's costs in one launch: block b of query q takes its candidates 256 b ..; the
// mean form takes the single mean candidate of query blockIdx.x (with the terms).
__global__ void __launch_bounds__(256)
k_batch_finalize(const BatchQueryDev *__restrict__ qd, const int2 *__restrict__ tab, const BatchEvalDev *ev)
{
    if (tab != nullptr) {
        const int2 e = tab[blockIdx.x];
        const BatchQueryDev &q = qd[e.x];
        finalize_body(q.item_sum, q.item_count, q.N, q.P, q.w_c, q.w_l, q.lambda_c, q.J, q.flag, nullptr, nullptr,
                      e.y * 256 + (int)threadIdx.x);
    } else {
        const BatchQueryDev &q = qd[blockIdx.x];
        const EvalArgs &a = ev[blockIdx.x].a;
        finalize_body(a.item_sum, a.item_count, 1, a.P, q.w_c, q.w_l, q.lambda_c, q.mean_J, q.mean_flag,
                      q.mean_terms, nullptr, (int)threadIdx.x);
    }
}

}  // namespace

int launch_eval_finalize(const double *item_sum, const uint32_t *item_count, int n, int P,
                         double w_c, double w_l, double lambda_c, double *J, uint8_t *flag,
                         double *terms, cudaStream_t st, const uint32_t *status)
{
    if (n == 0) return CP_OK;
    const int threads = 256;
    k_eval_finalize<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
        item_sum, item_count, n, P, w_c, w_l, lambda_c, J, flag, terms, status);
    CP_LAUNCHED("k_eval_finalize");
    return CP_OK;
}

}  // namespace cp

namespace cp {

int launch_batch_finalize(const BatchQueryDev *qd, const int2 *tab, int blocks, const BatchEvalDev *mean_ev,
                          cudaStream_t st)
{
    if (blocks == 0) return CP_OK;
    k_batch_finalize<<<blocks, tab != nullptr ? 256 : 32, 0, st>>>(qd, tab, mean_ev);
    CP_LAUNCHED("k_batch_finalize");
    return CP_OK;
}

}  // namespace cp
