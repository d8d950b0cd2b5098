// Binary64 pipe probe: the peak against which the worker kernel's roofline is
// quoted.  Not a step of the cipher (the paper has no counterpart).
//
// The worker keystream (Sec. II-B, Algorithm 2) is bound by the SM
// sub-partitions' binary64 pipes, which GB300 provides at a small fraction of
// its FP32 rate.  The probe measures that rate: one CTA per SM (a dynamic shared-memory
// request larger than half an SM keeps it to one), 4 k warps per CTA so that
// every one of the SM's four sub-partitions carries k warps, and every lane
// runs eight independent fused multiply-add chains.  Its result is the number
// of binary64 lane-operations it executed; the caller times the launch with
// CUDA events and divides.
#include "common.cuh"

namespace fhd {
namespace {

constexpr int kProbeChains = 8;
constexpr int kProbeSmem = 120 * 1024;   // > half of an SM's shared memory: one CTA per SM

__global__ void __launch_bounds__(1024) fp64_probe_kernel(uint32_t iters, double a, double b, double *sink) {
    double x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = 1.0 + 1e-3 * (double)(threadIdx.x + 37 * k);
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = __fma_rn(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s = __dadd_rn(s, x[k]);
    // A store the compiler cannot remove and that practically never happens: the chains stay live.
    if (s == a) sink[blockIdx.x] = s;
}

}  // namespace

cudaError_t launch_fp64_probe(uint32_t warps_per_subpartition, uint32_t iters, double *sink, uint64_t *lane_ops,
                              cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fp64_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem);
    if (e != cudaSuccess) return e;
    const uint32_t threads = 128u * warps_per_subpartition;
    // a slightly below 1 and b small keep every chain finite and away from subnormals for any iters
    fp64_probe_kernel<<<sms, threads, kProbeSmem, s>>>(iters, 1.0 - 0x1p-20, 0x1p-30, sink);
    note_launch();
    *lane_ops = (uint64_t)sms * threads * iters * kProbeChains;
    return cudaGetLastError();
}

}  // namespace fhd
