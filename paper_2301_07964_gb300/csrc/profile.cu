// Measurement utilities (include/hts_profile.h): per-launch CUDA-event profiling and an FP64
// throughput probe.  Neither is part of the reduction itself.
#include <cstdlib>

#include "hts_internal.cuh"

namespace hts {

ProfScope::ProfScope(hts_ctx *c, cudaStream_t s) : ctx(c), st(s), idx(-1)
{
    hts_prof_state &p = ctx->prof;
    if (!p.enabled) return;
    if (p.used >= p.cap) {
        ++p.dropped;
        return;
    }
    idx = p.used++;
    cudaEventRecord(p.ev[2 * idx], st);
}

void ProfScope::done(int kind, double flops, double bytes, double mma_flops)
{
    if (idx < 0) return;
    hts_prof_state &p = ctx->prof;
    cudaEventRecord(p.ev[2 * idx + 1], st);
    p.kind[idx] = kind;
    p.flops[idx] = flops;
    p.bytes[idx] = bytes;
    p.mma[idx] = mma_flops;
}

namespace {

void prof_free(hts_prof_state &p)
{
    if (p.ev) {
        for (int i = 0; i < 2 * p.cap; ++i)
            if (p.ev[i]) cudaEventDestroy(p.ev[i]);
    }
    std::free(p.ev);
    std::free(p.kind);
    std::free(p.flops);
    std::free(p.bytes);
    std::free(p.mma);
    p = hts_prof_state{};
}

// Each thread runs 8 independent FMA chains; 2 flops per FMA.
__global__ void k_fp64_probe(double *out, int iters, double a, double b)
{
    double x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace hts

using namespace hts;

extern "C" {

hts_status hts_profile_begin(hts_ctx *ctx, int max_launches)
{
    if (!ctx || max_launches <= 0) return HTS_ERR_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    prof_free(ctx->prof);
    hts_prof_state &p = ctx->prof;
    p.cap = max_launches;
    p.ev = static_cast<cudaEvent_t *>(std::calloc(2 * (size_t)max_launches, sizeof(cudaEvent_t)));
    p.kind = static_cast<int *>(std::calloc(max_launches, sizeof(int)));
    p.flops = static_cast<double *>(std::calloc(max_launches, sizeof(double)));
    p.bytes = static_cast<double *>(std::calloc(max_launches, sizeof(double)));
    p.mma = static_cast<double *>(std::calloc(max_launches, sizeof(double)));
    hts_status st = HTS_OK;
    if (!p.ev || !p.kind || !p.flops || !p.bytes || !p.mma) st = HTS_ERR_CUDA;
    for (int i = 0; st == HTS_OK && i < 2 * max_launches; ++i)
        if (cudaEventCreate(&p.ev[i]) != cudaSuccess) st = HTS_ERR_CUDA;
    if (st != HTS_OK) prof_free(p);
    else p.enabled = 1;
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return st;
}

hts_status hts_profile_end(hts_ctx *ctx, hts_kernel_profile out[HTS_K_NKINDS], int *dropped)
{
    if (!ctx || !out) return HTS_ERR_ARG;
    hts_prof_state &p = ctx->prof;
    for (int k = 0; k < HTS_K_NKINDS; ++k) out[k] = hts_kernel_profile{};
    if (dropped) *dropped = p.dropped;
    hts_status st = HTS_OK;
    for (int i = 0; st == HTS_OK && i < p.used; ++i)   // launches may sit on two streams
        if (cudaEventSynchronize(p.ev[2 * i + 1]) != cudaSuccess) st = HTS_ERR_CUDA;
    for (int i = 0; st == HTS_OK && i < p.used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]) != cudaSuccess) {
            st = HTS_ERR_CUDA;
            break;
        }
        hts_kernel_profile &o = out[p.kind[i] < HTS_K_NKINDS ? p.kind[i] : HTS_K_UTIL];
        o.launches += 1;
        o.ms += ms;
        o.flops += p.flops[i];
        o.bytes += p.bytes[i];
        o.mma_flops += p.mma[i];
    }
    prof_free(p);
    return st;
}

hts_status hts_probe_fp64_peak(void *stream, double *tflops)
{
    if (!tflops) return HTS_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HTS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HTS_ERR_CUDA;
    const int blocks = sms * 8, threads = 256, iters = 4000;
    double *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * (size_t)blocks * threads) != cudaSuccess) return HTS_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    hts_status s = HTS_OK;
    for (int rep = 0; rep < 3 && s == HTS_OK; ++rep) {
        cudaEventRecord(e0, st);
        k_fp64_probe<<<blocks, threads, 0, st>>>(buf, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = HTS_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (s != HTS_OK) return s;
    *tflops = 2.0 * 8 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
    return HTS_OK;
}

}  // extern "C"
