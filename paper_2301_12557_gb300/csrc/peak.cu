// Arithmetic peaks of the GPU this library runs on, measured: the roofline
// denominators of the pair kernels (FP32 for the fast path, FP64 for the
// plain FP64 path and the near-edge rescue).  The paper has no counterpart;
// it benchmarks CPUs.
//
// Each thread runs NCH independent multiply-add chains for `iters` steps, so
// the loop is bound by the issue rate of the fused multiply-add alone (no
// memory traffic, NCH >= 4 times the latency in flight per warp), on a grid
// that fills every SM to its thread limit.  Three loops:
//   FFMA   binary32 a = a * m + c         2 flops per lane per instruction
//   FFMA2  packed binary32 (two lanes)    4 flops per lane per instruction
//   DFMA   binary64 a = a * m + c         2 flops per lane per instruction
// The chains converge to c / (1 - m) and stay finite.  Nothing is written
// unless the final sum equals a value the chains cannot reach, which keeps
// the compiler from removing the loop without adding memory traffic.
#include <stdint.h>

#include "pc_host.hpp"

namespace pc {

constexpr int PEAK_NT = 256;   // threads per CTA
constexpr int PEAK_NCH = 8;    // independent chains per thread

__global__ void __launch_bounds__(PEAK_NT) k_peak_ffma(long long iters, float *sink) {
    float a[PEAK_NCH];
#pragma unroll
    for (int k = 0; k < PEAK_NCH; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    const float m = 0.99999988f, c = 1.0e-7f;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PEAK_NCH; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PEAK_NCH; ++k) s += a[k];
    if (s == -1.0f) sink[blockIdx.x * PEAK_NT + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PEAK_NT) k_peak_ffma2(long long iters, float *sink) {
    float2 a[PEAK_NCH];
#pragma unroll
    for (int k = 0; k < PEAK_NCH; ++k)
        a[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)(threadIdx.x + 2 * k) * 1e-3f);
    const float2 m = make_float2(0.99999988f, 0.99999988f), c = make_float2(1.0e-7f, 1.0e-7f);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PEAK_NCH; ++k) a[k] = __ffma2_rn(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PEAK_NCH; ++k) s += a[k].x + a[k].y;
    if (s == -1.0f) sink[blockIdx.x * PEAK_NT + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PEAK_NT) k_peak_dfma(long long iters, float *sink) {
    double a[PEAK_NCH];
#pragma unroll
    for (int k = 0; k < PEAK_NCH; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
    const double m = 0.9999999999, c = 1.0e-10;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PEAK_NCH; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PEAK_NCH; ++k) s += a[k];
    if (s == -1.0) sink[blockIdx.x * PEAK_NT + threadIdx.x] = (float)s;
}

}  // namespace pc

using namespace pc;

extern "C" pc_status pc_fp_peak(int kind, long long iters, void *stream, double *tflops, float *ms) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (kind < 0 || kind > 2 || iters < 0 || !tflops)
        return fail(PC_EINVAL, "pc_fp_peak: kind must be 0 (FFMA), 1 (FFMA2) or 2 (DFMA), iters >= 0");
    if (iters == 0) iters = (kind == 2) ? (1ll << 14) : (1ll << 18);
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 1, thr = 2048;
    PC_CUDA(cudaGetDevice(&dev));
    PC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PC_CUDA(cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
    void (*k)(long long, float *) = kind == 0 ? k_peak_ffma : (kind == 1 ? k_peak_ffma2 : k_peak_dfma);
    int per_sm = 0;
    PC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, PEAK_NT, 0));
    per_sm = std::max(1, std::min(per_sm, thr / PEAK_NT));
    const int grid = sms * per_sm;
    cudaEvent_t e0, e1;
    PC_CUDA(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    // one short launch first: clocks up, module loaded
    k<<<grid, PEAK_NT, 0, st>>>(iters / 16 + 1, nullptr);
    note_launch();
    cudaEventRecord(e0, st);
    k<<<grid, PEAK_NT, 0, st>>>(iters, nullptr);
    note_launch();
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "pc_fp_peak launch");
    const double flops_per_step = (kind == 1 ? 4.0 : 2.0) * PEAK_NCH;
    const double flops = flops_per_step * (double)iters * (double)grid * PEAK_NT;
    *tflops = flops / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return PC_OK;
}
