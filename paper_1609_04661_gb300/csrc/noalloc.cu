// dgamp_ct_output_step_noalloc: the Poisson output step without a plan and
// without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a host
// application that reserves all of the GPU's memory for its own pool at
// start-up and forbids further cudaMalloc calls by the libraries it loads,
// or a latency-critical loop that must not pay for (and synchronise on) an
// allocation.  For them this entry point keeps its scratch -- the per-block
// partial sums of tau_s and the block-arrival counter -- in a file-scope
// __device__ array of fixed size that every GPU loading the library holds
// until the process exits.  The caller still passes every input and output.
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace dgct {

int launch_output_step_scratch(const float* z, const float* y, float* s, long long M, int use_prev,
                               double tau_p, double logI0, double* tau_s_out, DevScalars* S,
                               double* partial, int max_blocks, cudaStream_t st);

namespace {

constexpr int kScratchBlocks = 1024;                       // one partial sum per block
constexpr size_t kScratchBytes = sizeof(DevScalars) + kScratchBlocks * sizeof(double);
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code this name is only a stand-in for the
// device symbol, never a device address: its address is looked up with
// cudaGetSymbolAddress on each device before use.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// The looked-up address is valid only for the context it was looked up in:
// after cudaDeviceReset (or a release and re-creation of the primary
// context) the module is loaded again and the array may move.  So each
// device's entry is keyed by the driver's context id, which is never reused
// within a process, and looked up again whenever the current context's id
// differs.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

struct Entry {
    unsigned long long ctx_id;
    void* addr;
};

std::mutex g_mu;
Entry g_cache[kMaxDevices] = {};

void* driver_entry(const char* name) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return p;
}

// Id of the calling thread's current context (0 if none or not available).
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        get_cur = reinterpret_cast<CtxGetCurrentFn>(driver_entry("cuCtxGetCurrent"));
        get_id = reinterpret_cast<CtxGetIdFn>(driver_entry("cuCtxGetId"));
    });
    if (!get_cur || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_scratch in the current device's context.
int scratch_address(void** out) {
    int dev = -1;
    DGCT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return DGAMP_CT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned long long id = current_ctx_id();
    Entry& e = g_cache[dev];
    if (id == 0 || e.addr == nullptr || e.ctx_id != id) {
        void* p = nullptr;
        DGCT_CUDA(cudaGetSymbolAddress(&p, g_scratch));   // also makes the primary context current
        if (id == 0) id = current_ctx_id();
        e.addr = p;
        e.ctx_id = id;   // 0 (no id available): looked up again on every call
    }
    *out = e.addr;
    return DGAMP_CT_OK;
}

}  // namespace
}  // namespace dgct

extern "C" int dgamp_ct_output_step_noalloc(const float* d_z, const float* d_y, const float* d_s_prev,
                                            int64_t M, double I0, double tau_p, float* d_s,
                                            double* d_tau_s, void* stream) {
    using namespace dgct;
    if (!d_z || !d_y || !d_s || !d_tau_s || M < 1) return DGAMP_CT_ERR_INVALID_ARG;
    if (M > DGAMP_CT_NOALLOC_MAX_M) return DGAMP_CT_ERR_INVALID_ARG;
    if (!(I0 > 0) || !std::isfinite(I0) || !(tau_p > 0) || !std::isfinite(tau_p))
        return DGAMP_CT_ERR_INVALID_ARG;
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != DGAMP_CT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    DevScalars* S = reinterpret_cast<DevScalars*>(base);
    double* partial = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + sizeof(DevScalars));
    // the counters must start at zero; the partial sums are overwritten
    DGCT_CUDA(cudaMemsetAsync(S, 0, sizeof(DevScalars), st));
    int use_prev = 0;
    if (d_s_prev) {
        if (d_s_prev != d_s)
            DGCT_CUDA(cudaMemcpyAsync(d_s, d_s_prev, (size_t)M * sizeof(float), cudaMemcpyDeviceToDevice, st));
        use_prev = 1;
    }
    return launch_output_step_scratch(d_z, d_y, d_s, (long long)M, use_prev, tau_p, std::log(I0), d_tau_s, S,
                                      partial, kScratchBlocks, st);
}
