// K1: SHA-256 of every sub-frame of every frame in a batch, and the XOR fold.
//
// Sec. II-A of the paper (Algorithm 1, partition / hash / fold): a frame's N
// bytes are split into n sub-frames f_i, h_i = SHA-256(f_i), and the frame
// digest is H = h_1 xor ... xor h_n.  Sub-frame i is the byte range
// [floor(i*N/n), floor((i+1)*N/n)).  SHA-256 follows FIPS 180-4.
//
// GPU mapping: one thread per sub-frame message (a message is inherently
// sequential).  The 64-byte blocks are read with 16-byte vector loads when the
// message start is 16-byte aligned (true for every video size whose N/n is a
// multiple of 16) and byte loads otherwise; the next block is loaded while
// the current one is compressed.  Rotations are funnel shifts, the three-input
// boolean functions map onto LOP3.
#include <mutex>

#include "common.cuh"

namespace fhd {
namespace {

__constant__ uint32_t kK[64] = {
    0x428a2f98u, 0x71374491u, 0xb5c0fbcfu, 0xe9b5dba5u, 0x3956c25bu, 0x59f111f1u, 0x923f82a4u, 0xab1c5ed5u,
    0xd807aa98u, 0x12835b01u, 0x243185beu, 0x550c7dc3u, 0x72be5d74u, 0x80deb1feu, 0x9bdc06a7u, 0xc19bf174u,
    0xe49b69c1u, 0xefbe4786u, 0x0fc19dc6u, 0x240ca1ccu, 0x2de92c6fu, 0x4a7484aau, 0x5cb0a9dcu, 0x76f988dau,
    0x983e5152u, 0xa831c66du, 0xb00327c8u, 0xbf597fc7u, 0xc6e00bf3u, 0xd5a79147u, 0x06ca6351u, 0x14292967u,
    0x27b70a85u, 0x2e1b2138u, 0x4d2c6dfcu, 0x53380d13u, 0x650a7354u, 0x766a0abbu, 0x81c2c92eu, 0x92722c85u,
    0xa2bfe8a1u, 0xa81a664bu, 0xc24b8b70u, 0xc76c51a3u, 0xd192e819u, 0xd6990624u, 0xf40e3585u, 0x106aa070u,
    0x19a4c116u, 0x1e376c08u, 0x2748774cu, 0x34b0bcb5u, 0x391c0cb3u, 0x4ed8aa4au, 0x5b9cca4fu, 0x682e6ff3u,
    0x748f82eeu, 0x78a5636fu, 0x84c87814u, 0x8cc70208u, 0x90befffau, 0xa4506cebu, 0xbef9a3f7u, 0xc67178f2u};

__device__ __forceinline__ uint32_t rotr(uint32_t x, int n) { return __funnelshift_r(x, x, n); }
__device__ __forceinline__ uint32_t bswap(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

struct ShaState {
    uint32_t h[8];
    __device__ __forceinline__ void init() {
        h[0] = 0x6a09e667u; h[1] = 0xbb67ae85u; h[2] = 0x3c6ef372u; h[3] = 0xa54ff53au;
        h[4] = 0x510e527fu; h[5] = 0x9b05688cu; h[6] = 0x1f83d9abu; h[7] = 0x5be0cd19u;
    }
    // One FIPS 180-4 compression; w[] holds the block as big-endian words.
    __device__ __forceinline__ void compress(uint32_t w[16]) {
        uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
#pragma unroll
        for (int t = 0; t < 64; ++t) {
            uint32_t wt;
            if (t < 16) {
                wt = w[t];
            } else {
                uint32_t w15 = w[(t - 15) & 15], w2 = w[(t - 2) & 15];
                uint32_t s0 = rotr(w15, 7) ^ rotr(w15, 18) ^ (w15 >> 3);
                uint32_t s1 = rotr(w2, 17) ^ rotr(w2, 19) ^ (w2 >> 10);
                wt = w[t & 15] + s0 + w[(t - 7) & 15] + s1;
                w[t & 15] = wt;
            }
            uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
            uint32_t ch = (e & f) ^ (~e & g);
            uint32_t t1 = hh + S1 + ch + kK[t] + wt;
            uint32_t S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
            uint32_t mj = (a & b) ^ (a & c) ^ (b & c);
            uint32_t t2 = S0 + mj;
            hh = g; g = f; f = e; e = d + t1;
            d = c; c = b; b = a; a = t1 + t2;
        }
        h[0] += a; h[1] += b; h[2] += c; h[3] += d;
        h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
    }
};

__device__ __forceinline__ void load_block16(const uint8_t *p, uint4 q[4]) {
    const uint4 *v = reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = __ldg(v + k);
}

__device__ __forceinline__ void block_words(const uint4 q[4], uint32_t w[16]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        w[4 * k + 0] = bswap(q[k].x);
        w[4 * k + 1] = bswap(q[k].y);
        w[4 * k + 2] = bswap(q[k].z);
        w[4 * k + 3] = bswap(q[k].w);
    }
}

// SHA-256 of len bytes at p (device memory); digest as 8 big-endian-valued words.
__device__ void sha256_message(const uint8_t *p, uint64_t len, uint32_t out[8]) {
    ShaState st;
    st.init();
    uint64_t full = len >> 6;
    uint32_t w[16];
    if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
        if (full) {
            uint4 cur[4], nxt[4];
            load_block16(p, cur);
            for (uint64_t b = 0; b < full; ++b) {
                if (b + 1 < full) load_block16(p + 64 * (b + 1), nxt);
                block_words(cur, w);
                st.compress(w);
#pragma unroll
                for (int k = 0; k < 4; ++k) cur[k] = nxt[k];
            }
        }
    } else {
        for (uint64_t b = 0; b < full; ++b) {
            const uint8_t *q = p + 64 * b;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                w[k] = ((uint32_t)q[4 * k] << 24) | ((uint32_t)q[4 * k + 1] << 16) |
                       ((uint32_t)q[4 * k + 2] << 8) | (uint32_t)q[4 * k + 3];
            st.compress(w);
        }
    }
    // Padding (FIPS 180-4 Sec. 5.1.1): 0x80, zeros, 64-bit big-endian bit length.
    uint32_t rem = (uint32_t)(len & 63);
    const uint8_t *tail = p + 64 * full;
    uint64_t bits = len * 8;
    uint32_t nblk = (rem + 9 <= 64) ? 1 : 2;
    for (uint32_t blk = 0; blk < nblk; ++blk) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            uint32_t word = 0;
#pragma unroll
            for (int byte = 0; byte < 4; ++byte) {
                uint32_t pos = blk * 64 + 4 * k + byte;
                uint32_t v = 0;
                if (pos < rem) v = tail[pos];
                else if (pos == rem) v = 0x80u;
                word = (word << 8) | v;
            }
            w[k] = word;
        }
        if (blk == nblk - 1) {
            w[14] = (uint32_t)(bits >> 32);
            w[15] = (uint32_t)bits;
        }
        st.compress(w);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) out[k] = st.h[k];
}

__device__ __forceinline__ void store_digest(uint8_t *dst, const uint32_t h[8]) {
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);   // 32-byte slots, 4-byte aligned
#pragma unroll
    for (int k = 0; k < 8; ++k) d[k] = bswap(h[k]);
}

// One thread per (frame, sub-frame) of a batch.
__global__ void __launch_bounds__(64) sha_subframes_kernel(const __grid_constant__ Batch b) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t n = b.n;
    if (t >= b.count * n) return;
    const FrameDesc &fd = b.f[t / n];
    uint32_t i = t % n;
    uint64_t lo = (uint64_t)(((unsigned __int128)fd.N * i) / n);
    uint64_t hi = (uint64_t)(((unsigned __int128)fd.N * (i + 1)) / n);
    uint32_t h[8];
    sha256_message(fd.src + lo, hi - lo, h);
    store_digest(fd.part + 32 * i, h);
}

__global__ void __launch_bounds__(64) sha_plain_kernel(const uint8_t *data, uint64_t nbytes, uint32_t n,
                                                       uint32_t count, uint8_t *part) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * n) return;
    uint32_t k = t / n, i = t % n;
    uint64_t lo = (uint64_t)(((unsigned __int128)nbytes * i) / n);
    uint64_t hi = (uint64_t)(((unsigned __int128)nbytes * (i + 1)) / n);
    uint32_t h[8];
    sha256_message(data + k * nbytes + lo, hi - lo, h);
    store_digest(part + 32ull * t, h);
}

// digest[k] = XOR over i of part[k*n + i]; one warp per buffer, lane = byte-word.
__global__ void fold_kernel(const uint8_t *part, uint32_t n, uint32_t count, uint8_t *digest) {
    uint32_t k = blockIdx.x;
    uint32_t lane = threadIdx.x;
    if (k >= count || lane >= 8) return;
    const uint32_t *p = reinterpret_cast<const uint32_t *>(part + 32ull * n * k);
    uint32_t acc = 0;
    for (uint32_t i = 0; i < n; ++i) acc ^= p[8 * i + lane];
    reinterpret_cast<uint32_t *>(digest + 32ull * k)[lane] = acc;
}

// Scratch of fhd_frame_digest_noalloc: the per-sub-frame digests of one call,
// in a fixed device array so that the call allocates nothing.  Every GPU that
// loads the library holds it (2 MiB) until the process exits.
constexpr uint32_t kNoAllocMaxDigests = 1u << 16;
static __device__ __align__(256) uint8_t g_noalloc_part[32u * kNoAllocMaxDigests];

}  // namespace

uint32_t noalloc_max_digests() { return kNoAllocMaxDigests; }

// Device address of g_noalloc_part for the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress -- once per device, on the first call made while that
// device is current -- and cached.
cudaError_t noalloc_scratch(uint8_t **out) {
    static std::mutex mu;
    static void *addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_part);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    *out = static_cast<uint8_t *>(addr[dev]);
    return cudaSuccess;
}

cudaError_t launch_sha_subframes(const Batch &b, cudaStream_t s) {
    uint32_t threads = b.count * b.n;
    if (!threads) return cudaSuccess;
    // Small blocks spread the (few, long) message threads over many SMs.
    uint32_t bs = threads >= 152u * 64u ? 64 : 32;
    sha_subframes_kernel<<<(threads + bs - 1) / bs, bs, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_sha_plain(const uint8_t *data, uint64_t nbytes, uint32_t n, uint32_t count, uint8_t *part,
                             cudaStream_t s) {
    uint32_t threads = count * n;
    if (!threads) return cudaSuccess;
    uint32_t bs = 32;
    sha_plain_kernel<<<(threads + bs - 1) / bs, bs, 0, s>>>(data, nbytes, n, count, part);
    return cudaGetLastError();
}

cudaError_t launch_fold(const uint8_t *part, uint32_t n, uint32_t count, uint8_t *digest, cudaStream_t s) {
    if (!count) return cudaSuccess;
    fold_kernel<<<count, 32, 0, s>>>(part, n, count, digest);
    return cudaGetLastError();
}

}  // namespace fhd
