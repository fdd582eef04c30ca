// hts_reduce_stage2_noalloc: stage 2 for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) when they need the
// reduction: services that must not allocate once they are running, code that runs inside a
// host framework which owns every byte of device memory and only lends out the matrices, or
// code on a path where an allocation could block or fail at the worst moment.  Such callers
// cannot provide the `work` buffer of hts_reduce_stage2.  This entry point runs the same
// stage-2 reduction with its scratch (the reflectors of one sweep group and the progress words
// of the chase) in a fixed array compiled into the library instead.
//
// The array is a file-scope __device__ variable, so every GPU that loads this library holds
// kNoAllocScratchBytes of it until the process exits.  Host code may not use the array's
// name as a device address (it is a host-side stand-in); the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the first call for that
// device.
#include <mutex>

#include "hts_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_stage2_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices];   // device address of g_stage2_scratch on each device

// Device address of the scratch array on `device` (looked up once, with `device` current).
hts_status scratch_address(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) return HTS_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[device]) {
        int prev = -1;
        if (cudaGetDevice(&prev) != cudaSuccess) return HTS_ERR_CUDA;
        if (prev != device && cudaSetDevice(device) != cudaSuccess) return HTS_ERR_CUDA;
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_stage2_scratch);
        if (prev != device) cudaSetDevice(prev);
        if (e != cudaSuccess || p == nullptr) return HTS_ERR_CUDA;
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return HTS_OK;
}

}  // namespace

extern "C" hts_status hts_reduce_stage2_noalloc(hts_ctx *ctx, int n, int r,
                                                double *A, int lda, double *B, int ldb,
                                                hts_comp compq, double *Q, int ldq,
                                                hts_comp compz, double *Z, int ldz,
                                                hts_gemm_mode mode, const hts_params *p,
                                                void *stream)
{
    if (!ctx) return HTS_ERR_ARG;
    size_t need = 0;
    const hts_status s = hts_workspace_size(n, r, p, &need);   // validates n and r
    if (s != HTS_OK) return s;
    need = hts::stage2_workspace_bytes_mode(n, r, mode);        // stage 2 alone runs here
    if (need > kNoAllocScratchBytes) return HTS_ERR_WORKSPACE;
    void *scratch = nullptr;
    const hts_status a = scratch_address(ctx->device, &scratch);
    if (a != HTS_OK) return a;
    return hts_reduce_stage2(ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode, p, scratch,
                             kNoAllocScratchBytes, stream);
}
