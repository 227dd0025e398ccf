// Candidate evaluation without any device allocation: the same kernels as cp_evaluate,
// with every piece of scratch memory (obstacle records, spline basis table, per-unit
// partial sums and collision words) carved out of one fixed file-scope device array.
//
// Who needs this: callers that may not allocate GPU memory once they are running, such as
// a crane controller's real-time loop (cudaMalloc can synchronise the device and take an
// unbounded time) or a plug-in inside a host application that owns all device memory in its
// own pool. They pass their inputs and outputs and this call uses nothing else.
#include <atomic>
#include <mutex>

#include "cp_internal.cuh"

namespace cp {
namespace {

// Fixed scratch, held by every GPU that loads the library until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)CP_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_eval_scratch[kStaticScratchBytes];

// Device address of g_eval_scratch per device (the host-side symbol is only a stand-in).
// Looked up once per device; a device reset by the host application (cudaDeviceReset)
// would leave it stale, so the entry point must not be called after one.
constexpr int kMaxDevices = 64;
std::atomic<unsigned char *> g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

// Test hook: issue no staging copy, so that the evaluation's bounded wait runs out.
std::atomic<int> g_withhold_staging{0};

int scratch_address(unsigned char **out)
{
    int dev = 0;
    CP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error("device %d out of range", dev), CP_ERR_ARG;
    unsigned char *p = g_scratch_addr[dev].load();
    if (p == nullptr) {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        p = g_scratch_addr[dev].load();
        if (p == nullptr) {
            void *addr = nullptr;
            CP_CUDA(cudaGetSymbolAddress(&addr, g_eval_scratch));
            p = static_cast<unsigned char *>(addr);
            g_scratch_addr[dev].store(p);
        }
    }
    *out = p;
    return CP_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace cp

using namespace cp;

extern "C" int cp_evaluate_static(const cp_model *model, const cp_cylinder *d_cyl, int32_t n_cyl,
                                  const cp_box *d_box, int32_t n_box, int32_t n_waypoints,
                                  int32_t substeps, double w_c, double w_l, double lambda_c,
                                  const double h_q0[4], const double h_qd[4], const float *d_xi,
                                  int32_t n, double *d_J, uint8_t *d_flag, double *d_terms,
                                  void *stream)
{
    int rc = validate_model(model);
    if (rc != CP_OK) return rc;
    if (n_waypoints < 1 || n_waypoints > CP_MAX_WAYPOINTS || substeps < 1 || substeps > 4096)
        return set_error("n_waypoints must be 1..%d and substeps 1..4096", CP_MAX_WAYPOINTS), CP_ERR_ARG;
    if (n < 0 || n_cyl < 0 || n_box < 0) return set_error("negative count"), CP_ERR_ARG;
    if ((n_cyl > 0 && !d_cyl) || (n_box > 0 && !d_box) || (n > 0 && (!d_xi || !d_J)) ||
        !h_q0 || !h_qd)
        return set_error("NULL argument"), CP_ERR_ARG;
    if (((uintptr_t)d_xi & 15u) != 0) return set_error("d_xi is not 16-byte aligned"), CP_ERR_ARG;
    if (!(w_c >= 0.0) || !(w_l >= 0.0) || !(lambda_c >= 0.0))
        return set_error("cost weights must be >= 0"), CP_ERR_ARG;
    if (n == 0) return CP_OK;

    const int K = n_waypoints, S = substeps;
    const int n_s = (K + 3) * S;
    const int chunks = (n_s + 31) / 32;
    const int G = eval_units_per_item(n, chunks);
    const int P = (chunks + G - 1) / G;
    // scratch layout: status word, cylinder records, box records, basis table, item sums
    const size_t o_status = 0;
    const size_t o_filt = o_status + 256;
    const size_t o_exact = o_filt + align256(sizeof(float4) * (size_t)n_cyl);
    const size_t o_group = o_exact + align256(sizeof(float4) * (size_t)n_cyl);
    const size_t o_bc = o_group + align256(sizeof(float4) * (size_t)n_groups(n_cyl));
    const size_t o_bh = o_bc + align256(sizeof(float4) * (size_t)n_box);
    const size_t o_basis = o_bh + align256(sizeof(float4) * (size_t)n_box);
    const size_t o_sum = o_basis + align256(sizeof(float4) * 2 * (size_t)S);
    const size_t o_count = o_sum + align256(sizeof(double) * 4 * (size_t)P * n);
    const size_t need = o_count + align256(sizeof(uint32_t) * (size_t)P * n);
    if (need > kStaticScratchBytes)
        return set_error("cp_evaluate_static needs %zu bytes of scratch for n = %d, n_s = %d and "
                         "%d + %d obstacles; its fixed scratch holds %zu bytes", need, n, n_s,
                         n_cyl, n_box, kStaticScratchBytes), CP_ERR_ARG;
    int dev = 0, smem_optin = 0, num_sms = 0;
    CP_CUDA(cudaGetDevice(&dev));
    CP_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CP_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = eval_smem_bytes(n_cyl, n_box, S);
    if (smem > (size_t)smem_optin)
        return set_error("%d cylinders and %d boxes need %zu B of shared memory; the device "
                         "allows %d B", n_cyl, n_box, smem, smem_optin), CP_ERR_ARG;
    if ((rc = eval_ensure_smem(smem)) != CP_OK) return rc;

    unsigned char *base = nullptr;
    if ((rc = scratch_address(&base)) != CP_OK) return rc;
    float4 *filt = (float4 *)(base + o_filt), *exact = (float4 *)(base + o_exact);
    float4 *group = (float4 *)(base + o_group);
    float4 *bc = (float4 *)(base + o_bc), *bh = (float4 *)(base + o_bh);
    float4 *basis = (float4 *)(base + o_basis);
    uint32_t *status = (uint32_t *)(base + o_status);
    const cudaStream_t st = (cudaStream_t)stream;
    CP_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), st));

    const ModelDev m = make_model(model);
    if ((rc = launch_prepare_scene(d_cyl, n_cyl, d_box, n_box, m.r_max, filt, exact, group, bc, bh, st)) !=
        CP_OK)
        return rc;
    if ((rc = launch_basis_table(S, basis, st)) != CP_OK) return rc;
    SceneDev sc{filt, exact, n_cyl, bc, bh, n_box, group};
    EvalArgs a{};
    a.xi = (const float4 *)d_xi;
    a.n = n;
    a.K = K;
    a.S = S;
    a.n_s = n_s;
    a.chunks = chunks;
    a.G = G;
    a.P = P;
    a.div_S = fast_div((uint32_t)S);
    a.div_P = fast_div((uint32_t)P);
    a.q0 = make_float4((float)h_q0[0], (float)h_q0[1], (float)h_q0[2], (float)h_q0[3]);
    a.qd = make_float4((float)h_qd[0], (float)h_qd[1], (float)h_qd[2], (float)h_qd[3]);
    a.broadphase = 1;
    a.withhold_staging = g_withhold_staging.load() != 0;
    a.status = status;   // a staging wait that runs out: the finalize writes NaN J, flag 1
    a.basis = basis;
    a.item_sum = (double *)(base + o_sum);
    a.item_count = (uint32_t *)(base + o_count);
    a.words_out = nullptr;
    a.pen_out = nullptr;
    if ((rc = launch_eval(m, sc, a, num_sms, st)) != CP_OK) return rc;
    return launch_eval_finalize(a.item_sum, a.item_count, n, P, w_c, w_l, lambda_c, d_J, d_flag, d_terms, st,
                                status);
}

extern "C" void cp_debug_static_withhold_staging(int32_t on) { g_withhold_staging.store(on != 0); }
