// Frame statistics of the paper's evaluation, batched over frames and
// channels: histogram variance and chi^2 (Sec. III-A, Eqs. (4)-(5)),
// adjacent-pixel correlation (Sec. III-B, Eqs. (6)-(9)), information entropy
// and local Shannon entropy (Sec. III-C, Eqs. (10)-(11)), NPCR and UACI
// (Sec. IV-B, Eqs. (14)-(15)).
//
// Frames are one contiguous batch [count][h][w][C] of uint8.  Counting work
// (histograms, changed pixels, |a - b|, the correlation sums) is exact
// integer arithmetic; only the final formula of each statistic rounds.
// GPU mapping: the histogram and NPCR/UACI passes stream the frames once with
// 16-byte loads (memory bound) in groups of 16 * C bytes, so that every byte's
// channel is a compile-time constant (C is a template parameter); per-warp
// shared-memory histograms, or per-thread channel sums built four bytes at a
// time with the SIMD byte instructions, are merged with one global atomic per
// counter and CTA, and a per-(frame, channel) warp finishes the statistic.  The correlation and local-entropy
// statistics read only the sampled pairs and blocks (a few kB per frame).
#include "bounds.cuh"
#include "common.cuh"

namespace fhd {
namespace {

constexpr int kStatThreads = 256;
constexpr int kStatWarps = kStatThreads / 32;

__global__ void zero_kernel(unsigned long long *p, uint64_t n) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) p[k] = 0;
}

// Channel of byte k of the batch: frames hold whole pixels, so it is k mod C.
// Histogram pass: CTA b covers bytes [b * chunk, (b + 1) * chunk) of the
// batch (chunk a multiple of 16 * C that divides the frame, so a CTA stays in
// one frame and starts on channel 0).  A thread takes groups of 16 * C bytes
// (C 16-byte loads), in which byte q belongs to channel q mod C: the channel
// of every byte is a compile-time constant.  The CTA's counters are
// [channel][bin][lane]: each lane counts in its own bank, so the shared
// atomics of a warp never conflict on a bank; at the end the 32 lane copies
// are summed and added to the frame's global histogram.
template <int C>
__global__ void __launch_bounds__(kStatThreads) hist_kernel(const uint8_t *frames, uint64_t total, uint64_t frame_bytes,
                                                            uint64_t chunk, unsigned long long *hist) {
    extern __shared__ uint32_t sh[];   // C * 256 * 32
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t k = threadIdx.x; k < C * 256 * 32; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    const uint64_t b0 = (uint64_t)blockIdx.x * chunk;
    const uint64_t b1 = min(b0 + chunk, total);
    uint32_t *mine = sh + lane;
    constexpr uint32_t G = 16 * C;
    const bool vec = (reinterpret_cast<uintptr_t>(frames + b0) & 15) == 0 && (b1 - b0) % G == 0;
    if (vec) {
        for (uint64_t k = b0 + G * (uint64_t)threadIdx.x; k < b1; k += G * (uint64_t)blockDim.x) {
            if (!FHD_IN(k + G - 1, total, kSiteStats)) break;
            uint4 v[C];
#pragma unroll
            for (int m = 0; m < C; ++m) v[m] = __ldcs(reinterpret_cast<const uint4 *>(frames + k) + m);
#pragma unroll
            for (int m = 0; m < C; ++m) {
                const uint32_t wd[4] = {v[m].x, v[m].y, v[m].z, v[m].w};
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    atomicAdd(&mine[(((16 * m + q) % C) * 256 + ((wd[q >> 2] >> (8 * (q & 3))) & 255)) * 32], 1u);
            }
        }
    } else {
        for (uint64_t t = b0 + threadIdx.x; t < b1; t += blockDim.x)
            atomicAdd(&mine[((uint32_t)(t % C) * 256 + frames[t]) * 32], 1u);
    }
    __syncthreads();
    const uint64_t f = b0 / frame_bytes;
    for (uint32_t q = threadIdx.x; q < C * 256; q += blockDim.x) {
        const uint32_t *row = sh + q * 32;
        uint32_t s = 0;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) s += row[(l + q) & 31];   // rotated start: the threads of a warp read 32 banks
        if (s) atomicAdd(&hist[f * C * 256 + q], (unsigned long long)s);
    }
}

// One warp per (frame, channel): var(Z) (Eq. 4) = S2/256 - (S1/256)^2,
// chi^2 (Eq. 5) = (256 S2 - N^2) / N, H (Eq. 10) = log2 N - (sum z log2 z) / N.
__global__ void hist_finish_kernel(const unsigned long long *hist, uint32_t items, uint32_t *hist32, double *out) {
    const uint32_t item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (item >= items) return;
    const unsigned long long *z = hist + (uint64_t)item * 256;
    unsigned long long s1 = 0, s2 = 0;
    double zl = 0.0;
    for (int i = lane; i < 256; i += 32) {
        const unsigned long long v = z[i];
        s1 += v;
        s2 += v * v;
        if (v) zl += (double)v * log2((double)v);
        if (hist32) hist32[(uint64_t)item * 256 + i] = (uint32_t)v;
    }
    for (int o = 16; o; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        zl += __shfl_xor_sync(0xffffffffu, zl, o);
    }
    if (lane == 0) {
        const double N = (double)s1;
        const double m1 = N / 256.0;
        out[3 * item + 0] = (double)s2 / 256.0 - m1 * m1;
        out[3 * item + 1] = (double)(long long)(256ull * s2 - s1 * s1) / N;
        out[3 * item + 2] = log2(N) - zl / N;
    }
}

// Bytes of 32-bit word m of a 16 * C-byte group that belong to channel c.
template <int C>
__host__ __device__ constexpr uint32_t chan_mask(int m, int c) {
    uint32_t r = 0;
    for (int t = 0; t < 4; ++t)
        if ((4 * m + t) % C == c) r |= 0xFFu << (8 * t);
    return r;
}

// NPCR / UACI pass: per CTA chunk and 16 * C-byte groups as in hist_kernel.
// Four bytes at a time: __vabsdiffu4 gives |a - b| per byte, __vcmpne4 marks
// the differing bytes, and a channel's bytes of the word are summed with
// __dp4a through a compile-time mask.
template <int C>
__global__ void __launch_bounds__(kStatThreads) npcr_kernel(const uint8_t *a, const uint8_t *b, uint64_t total,
                                                            uint64_t frame_bytes, uint64_t chunk,
                                                            unsigned long long *acc) {
    __shared__ unsigned long long sacc[4][2];
    if (threadIdx.x < 8) sacc[threadIdx.x >> 1][threadIdx.x & 1] = 0;
    __syncthreads();
    uint32_t changed[C], diff[C];
#pragma unroll
    for (int c = 0; c < C; ++c) changed[c] = diff[c] = 0;
    const uint64_t b0 = (uint64_t)blockIdx.x * chunk;
    const uint64_t b1 = min(b0 + chunk, total);
    constexpr uint32_t G = 16 * C;
    const bool vec = ((reinterpret_cast<uintptr_t>(a + b0) | reinterpret_cast<uintptr_t>(b + b0)) & 15) == 0 &&
                     (b1 - b0) % G == 0;
    if (vec) {
        for (uint64_t k = b0 + G * (uint64_t)threadIdx.x; k < b1; k += G * (uint64_t)blockDim.x) {
            if (!FHD_IN(k + G - 1, total, kSiteStats)) break;
            uint4 va[C], vb[C];
#pragma unroll
            for (int m = 0; m < C; ++m) {
                va[m] = __ldcs(reinterpret_cast<const uint4 *>(a + k) + m);
                vb[m] = __ldcs(reinterpret_cast<const uint4 *>(b + k) + m);
            }
#pragma unroll
            for (int m = 0; m < 4 * C; ++m) {
                const uint32_t x = (&va[m >> 2].x)[m & 3], y = (&vb[m >> 2].x)[m & 3];
                const uint32_t d = __vabsdiffu4(x, y);
                const uint32_t ne = __vcmpne4(x, y) & 0x01010101u;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    constexpr uint32_t ones = 0x01010101u;
                    const uint32_t mk = chan_mask<C>(m, c);
                    diff[c] = __dp4a(d & mk, ones, diff[c]);
                    changed[c] = __dp4a(ne & mk, ones, changed[c]);
                }
            }
        }
    } else {
        for (uint64_t t = b0 + threadIdx.x; t < b1; t += blockDim.x) {
            const uint32_t c = (uint32_t)(t % C);
            const int x = a[t], y = b[t];
#pragma unroll
            for (int cc = 0; cc < C; ++cc)
                if ((uint32_t)cc == c) {
                    changed[cc] += x != y;
                    diff[cc] += (uint32_t)abs(x - y);
                }
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        unsigned long long x = changed[c], y = diff[c];
        for (int o = 16; o; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&sacc[c][0], x);
            atomicAdd(&sacc[c][1], y);
        }
    }
    __syncthreads();
    const uint64_t f = b0 / frame_bytes;
    if (threadIdx.x < 2 * C) atomicAdd(&acc[(f * C + (threadIdx.x >> 1)) * 2 + (threadIdx.x & 1)], sacc[threadIdx.x >> 1][threadIdx.x & 1]);
}

__global__ void npcr_finish_kernel(const unsigned long long *acc, uint32_t items, uint64_t wh, double *out) {
    const uint32_t item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= items) return;
    out[2 * item + 0] = 100.0 * (double)acc[2 * item] / (double)wh;
    out[2 * item + 1] = 100.0 * (double)acc[2 * item + 1] / ((double)wh * 255.0);
}

// Correlation: one CTA per (frame, direction); pairs[(f * 3 + d) * npairs + k] = (i, j) of x; y is the
// neighbour (0, 1), (1, 0) or (1, 1).  Exact sums sx, sy, sxx, syy, sxy per channel, then
// r = (N sxy - sx sy) / sqrt((N sxx - sx^2)(N syy - sy^2)).
__global__ void __launch_bounds__(kStatThreads) corr_kernel(const uint8_t *frames, uint32_t h, uint32_t w, uint32_t C,
                                                            const uint32_t *pairs, uint32_t npairs, long long *sums,
                                                            double *out, unsigned *status) {
    __shared__ long long red[kStatWarps][4][5];
    const uint32_t f = blockIdx.x / 3, d = blockIdx.x % 3;
    const uint32_t di = d == 0 ? 0 : 1, dj = d == 1 ? 0 : 1;
    const uint8_t *F = frames + (uint64_t)f * h * w * C;
    const uint32_t *pp = pairs + 2 * ((uint64_t)blockIdx.x * npairs);
    long long acc[4][5] = {};
    for (uint32_t k = threadIdx.x; k < npairs; k += blockDim.x) {
        const uint32_t i = pp[2 * k], j = pp[2 * k + 1];
        if (i + di >= h || j + dj >= w) {   // out of the frame: counted nowhere, reported
            atomicOr(status, 1u);
            continue;
        }
        if (!FHD_IN(((uint64_t)(i + di) * w + j + dj) * C + C - 1, (uint64_t)h * w * C, kSiteStats)) continue;
        const uint8_t *px = F + ((uint64_t)i * w + j) * C;
        const uint8_t *py = F + ((uint64_t)(i + di) * w + j + dj) * C;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if ((uint32_t)c < C) {
                const long long x = px[c], y = py[c];
                acc[c][0] += x;
                acc[c][1] += y;
                acc[c][2] += x * x;
                acc[c][3] += y * y;
                acc[c][4] += x * y;
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            long long v = acc[c][m];
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][c][m] = v;
        }
    __syncthreads();
    if (threadIdx.x < C) {
        const uint32_t c = threadIdx.x;
        long long s[5] = {0, 0, 0, 0, 0};
        for (int w8 = 0; w8 < kStatWarps; ++w8)
            for (int m = 0; m < 5; ++m) s[m] += red[w8][c][m];
        const long long N = (long long)npairs;
        long long *so = sums + ((uint64_t)(f * C + c) * 3 + d) * 5;
        for (int m = 0; m < 5; ++m) so[m] = s[m];
        const double num = (double)(N * s[4] - s[0] * s[1]);
        const double vx = (double)(N * s[2] - s[0] * s[0]), vy = (double)(N * s[3] - s[1] * s[1]);
        out[(uint64_t)(f * C + c) * 3 + d] = num / sqrt(vx * vy);
    }
}

// Local Shannon entropy: one CTA per (frame, block) builds the block's
// histograms in shared memory and writes each channel's entropy; a second
// kernel takes the mean over the k blocks in block order (a fixed summation
// order, so the result does not depend on scheduling).
__global__ void __launch_bounds__(kStatThreads) block_entropy_kernel(const uint8_t *frames, uint32_t h, uint32_t w,
                                                                     uint32_t C, const uint32_t *blocks, uint32_t k,
                                                                     uint32_t bs, double *ent, unsigned *status) {
    __shared__ uint32_t hist[4][256];
    const uint32_t f = blockIdx.x / k, q = blockIdx.x % k;
    const uint8_t *F = frames + (uint64_t)f * h * w * C;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t r0 = blocks[2 * ((uint64_t)f * k + q)], c0 = blocks[2 * ((uint64_t)f * k + q) + 1];
    const bool inside = r0 + bs <= h && c0 + bs <= w;
    for (uint32_t t = threadIdx.x; t < 4 * 256; t += blockDim.x) (&hist[0][0])[t] = 0;
    __syncthreads();
    if (inside) {
        for (uint32_t i = 0; i < bs; ++i) {
            const uint8_t *row = F + ((uint64_t)(r0 + i) * w + c0) * C;
            for (uint32_t t = threadIdx.x; t < bs * C; t += blockDim.x)
                if (FHD_IN(((uint64_t)(r0 + i) * w + c0) * C + t, (uint64_t)h * w * C, kSiteStats))
                    atomicAdd(&hist[t % C][row[t]], 1u);
        }
    } else if (threadIdx.x == 0) {
        atomicOr(status, 1u);
    }
    __syncthreads();
    if ((uint32_t)warp < C) {
        double e = 0.0;
        for (int i = lane; i < 256; i += 32) {
            const uint32_t z = hist[warp][i];
            if (z) e += (double)z * log2((double)z);
        }
        for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        const double T = (double)bs * (double)bs;
        if (lane == 0) ent[((uint64_t)f * k + q) * C + warp] = log2(T) - e / T;
    }
}

__global__ void block_entropy_mean_kernel(const double *ent, uint32_t count, uint32_t C, uint32_t k, double *out) {
    const uint32_t item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= count * C) return;
    const uint32_t f = item / C, c = item % C;
    double acc = 0.0;
    for (uint32_t q = 0; q < k; ++q) acc += ent[((uint64_t)f * k + q) * C + c];
    out[item] = acc / (double)k;
}

// Bytes per CTA of the streaming passes: a multiple of 16 * C near `target`
// that divides the frame, so that a CTA never spans two frames and starts on
// channel 0; frames without such a divisor down to target/16 get one CTA each.
uint64_t stat_chunk(uint64_t frame_bytes, uint32_t C, uint64_t target = 65536) {
    const uint64_t unit = 16ull * C;
    if (frame_bytes % unit != 0 || frame_bytes <= target) return frame_bytes;
    for (uint64_t chunk = unit * (target / unit); chunk >= target / 16; chunk -= unit)
        if (frame_bytes % chunk == 0) return chunk;
    return frame_bytes;
}

unsigned zero_grid(uint64_t n) {
    const uint64_t g = (n + 255) / 256;
    return (unsigned)(g < 1024 ? (g ? g : 1) : 1024);
}

}  // namespace

cudaError_t launch_stats_histogram(const uint8_t *frames, uint32_t count, uint64_t frame_bytes, uint32_t C,
                                   unsigned long long *hist64, uint32_t *hist32, double *out, cudaStream_t s) {
    const uint64_t total = (uint64_t)count * frame_bytes;
    const uint64_t items = (uint64_t)count * C;
    zero_kernel<<<zero_grid(items * 256), 256, 0, s>>>(hist64, items * 256);
    note_launch();
    const uint64_t chunk = stat_chunk(frame_bytes, C, 1u << 19);   // ~512 kB: amortises the 32-copy merge
    const uint64_t ctas = (total + chunk - 1) / chunk;
    const size_t smem = (size_t)C * 256 * 32 * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(hist_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 131072);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(hist_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 131072);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(hist_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 131072);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(hist_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 131072);
    if (e != cudaSuccess) return e;
    switch (C) {
        case 1: hist_kernel<1><<<(unsigned)ctas, kStatThreads, smem, s>>>(frames, total, frame_bytes, chunk, hist64); break;
        case 2: hist_kernel<2><<<(unsigned)ctas, kStatThreads, smem, s>>>(frames, total, frame_bytes, chunk, hist64); break;
        case 3: hist_kernel<3><<<(unsigned)ctas, kStatThreads, smem, s>>>(frames, total, frame_bytes, chunk, hist64); break;
        default: hist_kernel<4><<<(unsigned)ctas, kStatThreads, smem, s>>>(frames, total, frame_bytes, chunk, hist64); break;
    }
    note_launch();
    hist_finish_kernel<<<(unsigned)((items + 7) / 8), 256, 0, s>>>(hist64, (uint32_t)items, hist32, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_stats_npcr(const uint8_t *a, const uint8_t *b, uint32_t count, uint64_t frame_bytes, uint32_t C,
                              uint64_t wh, unsigned long long *acc, double *out, cudaStream_t s) {
    const uint64_t total = (uint64_t)count * frame_bytes;
    const uint64_t items = (uint64_t)count * C;
    zero_kernel<<<zero_grid(items * 2), 256, 0, s>>>(acc, items * 2);
    note_launch();
    const uint64_t chunk = stat_chunk(frame_bytes, C);
    const unsigned grid = (unsigned)((total + chunk - 1) / chunk);
    switch (C) {
        case 1: npcr_kernel<1><<<grid, kStatThreads, 0, s>>>(a, b, total, frame_bytes, chunk, acc); break;
        case 2: npcr_kernel<2><<<grid, kStatThreads, 0, s>>>(a, b, total, frame_bytes, chunk, acc); break;
        case 3: npcr_kernel<3><<<grid, kStatThreads, 0, s>>>(a, b, total, frame_bytes, chunk, acc); break;
        default: npcr_kernel<4><<<grid, kStatThreads, 0, s>>>(a, b, total, frame_bytes, chunk, acc); break;
    }
    note_launch();
    npcr_finish_kernel<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(acc, (uint32_t)items, wh, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_stats_correlation(const uint8_t *frames, uint32_t count, uint32_t h, uint32_t w, uint32_t C,
                                     const uint32_t *pairs, uint32_t npairs, long long *sums, double *out,
                                     unsigned *status, cudaStream_t s) {
    corr_kernel<<<count * 3, kStatThreads, 0, s>>>(frames, h, w, C, pairs, npairs, sums, out, status);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_stats_local_entropy(const uint8_t *frames, uint32_t count, uint32_t h, uint32_t w, uint32_t C,
                                       const uint32_t *blocks, uint32_t k, uint32_t bs, double *ent, double *out,
                                       unsigned *status, cudaStream_t s) {
    block_entropy_kernel<<<count * k, kStatThreads, 0, s>>>(frames, h, w, C, blocks, k, bs, ent, status);
    note_launch();
    block_entropy_mean_kernel<<<(count * C + 127) / 128, 128, 0, s>>>(ent, count, C, k, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fhd

FHD_BOUNDS_TAKER(take_bounds_stats)
