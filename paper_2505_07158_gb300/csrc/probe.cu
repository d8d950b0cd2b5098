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
#include "binary64_int.cuh"
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

// Operand pairs for the integer binary64 check: class h3 % 7 of pair i (splitmix64 of the seed and i):
// any bit patterns; the chaotic range (|x| ~ 2^-3 .. 2^5); near cancellation (b ~ -a); exponent
// differences of 48..61 (the alignment boundary of the sum); few significand bits (exact products and ties);
// zeros and subnormals; any normal exponents.
__device__ __forceinline__ uint64_t splitmix(uint64_t &x) {
    uint64_t z = (x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ void check_pair(uint64_t seed, uint64_t i, uint64_t &A, uint64_t &B) {
    uint64_t st = seed ^ (i * 0xd1b54a32d192ed03ull);
    const uint64_t h1 = splitmix(st), h2 = splitmix(st), h3 = splitmix(st);
    const uint64_t E = 0x7ffull << 52;
    switch (h3 % 7) {
        case 0: A = h1; B = h2; break;
        case 1: A = (h1 & ~E) | ((1020 + h1 % 9) << 52); B = (h2 & ~E) | ((1020 + h2 % 9) << 52); break;
        case 2: A = (h1 & ~E) | ((1000 + h1 % 40) << 52); B = (A ^ kSign) ^ (h2 & ((1ull << (h2 % 53)) - 1)); break;
        case 3:
            A = (h1 & ~E) | (1023ull << 52);
            B = ((h2 & ~E) | ((1023 - 48 - h2 % 14) << 52)) ^ ((h3 & 8) ? kSign : 0);
            break;
        case 4: {
            const int k = (int)(h3 % 30);
            A = ((h1 & ((1ull << k) - 1)) << (52 - k)) | ((1010 + h1 % 30) << 52) | (h1 & kSign);
            B = (((h2 & ~E) | ((1010 + h2 % 30) << 52)) >> (52 - k)) << (52 - k);
            break;
        }
        case 5: A = h1; B = (h3 & 16) ? (h2 & kSign) : (h2 & kMant); break;
        default: A = (h1 & ~E) | ((1 + h1 % 2046) << 52); B = (h2 & ~E) | ((1 + h2 % 2046) << 52); break;
    }
}

// Every lane of a warp takes part in every round (the wrappers vote across the warp); pairs past the end
// are computed and not counted.
__global__ void __launch_bounds__(256) binary64_check_kernel(uint64_t pairs, uint64_t seed,
                                                             unsigned long long *counts) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long bad_m = 0, bad_a = 0, fast_m = 0, fast_a = 0;
    for (uint64_t base = 0; base < pairs; base += stride) {
        const uint64_t i = base + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        uint64_t A, B;
        check_pair(seed, i, A, B);
        const double a = __longlong_as_double((long long)A), b = __longlong_as_double((long long)B);
        const double pm = i64_mul(a, b), pa = i64_add(a, b);
        const double nm = __dmul_rn(a, b), na = __dadd_rn(a, b);
        bool spm, spa;
        b64_mul(A, B, spm);
        b64_add(A, B, spa);
        if (i < pairs) {
            // NaN results: any NaN of the binary64 instruction is the one the fallback produced
            bad_m += __double_as_longlong(pm) != __double_as_longlong(nm);
            bad_a += __double_as_longlong(pa) != __double_as_longlong(na);
            fast_m += !spm;
            fast_a += !spa;
        }
    }
    atomicAdd(counts + 0, bad_m);
    atomicAdd(counts + 1, bad_a);
    atomicAdd(counts + 2, fast_m);
    atomicAdd(counts + 3, fast_a);
}

}  // namespace

cudaError_t launch_binary64_check(uint64_t pairs, uint64_t seed, unsigned long long *counts, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    binary64_check_kernel<<<sms * 8, 256, 0, s>>>(pairs, seed, counts);
    note_launch();
    return cudaGetLastError();
}

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
