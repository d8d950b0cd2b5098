// K1: SHA-256 of every sub-frame of every frame in a batch, and the XOR fold.
//
// Sec. II-A of the paper (Algorithm 1, partition / hash / fold): a frame's N
// bytes are split into n sub-frames f_i, h_i = SHA-256(f_i), and the frame
// digest is H = h_1 xor ... xor h_n.  Sub-frame i is the byte range
// [floor(i*N/n), floor((i+1)*N/n)).  SHA-256 follows FIPS 180-4.
//
// GPU mapping: a message is inherently sequential, and with n = 32 a frame has
// only 32 of them, so the time of one message is the time of the frame.  Each
// message therefore gets two threads in two warps of one CTA: a producer lane
// brings the 64-byte blocks in (cp.async into a four-block shared-memory ring
// when the message start is 16-byte aligned, byte loads otherwise; an L2
// prefetch runs eight blocks ahead), expands the message schedule and stores
// W[t] + K[t] into a double-buffered shared-memory ring; the consumer lane
// runs only the 64 compression rounds of the previous block.  The two warps
// meet at one named barrier per block.  Rotations are funnel shifts, the
// three-input boolean functions map onto LOP3.
#include <mutex>

#include "common.cuh"
#include "sha256_dev.cuh"

namespace fhd {
namespace {

// Sub-frame messages of a batch: message m is sub-frame m % n of frame m / n.
__global__ void __launch_bounds__(64) sha_subframes_kernel(const __grid_constant__ Batch b) {
    __shared__ ShaSmem sm;
    const uint32_t n = b.n;
    sha_pipeline(
        [&](uint32_t m, const uint8_t *&p, uint64_t &len, uint8_t *&out) {
            if (!FHD_IN(m / n, b.count, kSiteShaDigest)) return false;
            const FrameDesc &fd = b.f[m / n];
            const uint32_t i = m % n;
            const uint64_t lo = (uint64_t)(((unsigned __int128)fd.N * i) / n);
            const uint64_t hi = (uint64_t)(((unsigned __int128)fd.N * (i + 1)) / n);
            if (!FHD_IN(hi, fd.N + 1, kSiteShaMessage)) return false;
            p = fd.src + lo;
            len = hi - lo;
            out = fd.part + 32ull * i;
            return true;
        },
        b.count * n, blockIdx.x, threadIdx.x, 1, sm);
}

// `count` buffers of nbytes laid end to end, n sub-frames each.
__global__ void __launch_bounds__(64) sha_plain_kernel(const uint8_t *data, uint64_t nbytes, uint32_t n,
                                                       uint32_t count, uint8_t *part) {
    __shared__ ShaSmem sm;
    sha_pipeline(
        [&](uint32_t m, const uint8_t *&p, uint64_t &len, uint8_t *&out) {
            const uint32_t k = m / n, i = m % n;
            const uint64_t lo = (uint64_t)(((unsigned __int128)nbytes * i) / n);
            const uint64_t hi = (uint64_t)(((unsigned __int128)nbytes * (i + 1)) / n);
            if (!FHD_IN(k, count, kSiteShaDigest) || !FHD_IN(hi, nbytes + 1, kSiteShaMessage)) return false;
            p = data + k * nbytes + lo;
            len = hi - lo;
            out = part + 32ull * m;
            return true;
        },
        count * n, blockIdx.x, threadIdx.x, 1, sm);
}

// Sub-frame messages of the decrypted frames (dst) of a batch, for the
// receiver-side check; digests go to part (n per frame).
__global__ void __launch_bounds__(64) sha_dst_kernel(const __grid_constant__ Batch b) {
    __shared__ ShaSmem sm;
    const uint32_t n = b.n;
    sha_pipeline(
        [&](uint32_t m, const uint8_t *&p, uint64_t &len, uint8_t *&out) {
            if (!FHD_IN(m / n, b.count, kSiteShaDigest)) return false;
            const FrameDesc &fd = b.f[m / n];
            const uint32_t i = m % n;
            const uint64_t lo = (uint64_t)(((unsigned __int128)fd.N * i) / n);
            const uint64_t hi = (uint64_t)(((unsigned __int128)fd.N * (i + 1)) / n);
            if (!FHD_IN(hi, fd.N + 1, kSiteShaMessage)) return false;
            p = fd.dst + lo;
            len = hi - lo;
            out = fd.part + 32ull * i;
            return true;
        },
        b.count * n, blockIdx.x, threadIdx.x, 1, sm);
}

// ok[k] = (frame k's digest recomputed from its sub-frame digests, by the batch's digest mode) == frame k's
// transmitted digest.
__global__ void verify_kernel(const __grid_constant__ Batch b, uint8_t *ok) {
    const uint32_t k = blockIdx.x, lane = threadIdx.x;
    if (k >= b.count) return;
    const FrameDesc &fd = b.f[k];
    uint32_t diff = 0;
    if (b.digest_mode == FHD_DIGEST_TREE) {
        if (lane == 0) {
            uint32_t h[8];
            tree_digest(fd.part, b.n, h);
            const uint32_t *t = reinterpret_cast<const uint32_t *>(fd.digest);
            for (int q = 0; q < 8; ++q) diff |= bswap(h[q]) ^ t[q];
        }
    } else if (lane < 8) {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(fd.part);
        uint32_t acc = 0;
        for (uint32_t i = 0; i < b.n; ++i) acc ^= p[8 * i + lane];
        diff = acc ^ reinterpret_cast<const uint32_t *>(fd.digest)[lane];
    }
    diff = __reduce_or_sync(0xffffffffu, diff);
    if (lane == 0) ok[fd.slot] = diff == 0 ? 1 : 0;
}

// Tree digests of a batch: one thread per frame, written to the frame's digest.
__global__ void tree_batch_kernel(const __grid_constant__ Batch b) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= b.count) return;
    const FrameDesc &fd = b.f[k];
    uint32_t h[8];
    tree_digest(fd.part, b.n, h);
    store_digest(fd.digest, h);
}

// Tree digests of `count` buffers' sub-frame digests (part[k*n .. k*n + n)); one thread per buffer.
__global__ void tree_kernel(const uint8_t *part, uint32_t n, uint32_t count, uint8_t *digest) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    uint32_t h[8];
    tree_digest(part + 32ull * n * k, n, h);
    store_digest(digest + 32ull * k, h);
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

// The digest of every frame of a batch: H = h_1 xor ... xor h_n over the
// frame's n sub-frame digests (Algorithm 1), written to the frame's digest.
__global__ void fold_batch_kernel(const __grid_constant__ Batch b) {
    const uint32_t k = blockIdx.x, lane = threadIdx.x;
    if (k >= b.count || lane >= 8) return;
    const FrameDesc &fd = b.f[k];
    const uint32_t *p = reinterpret_cast<const uint32_t *>(fd.part);
    uint32_t acc = 0;
    for (uint32_t i = 0; i < b.n; ++i) acc ^= p[8 * i + lane];
    reinterpret_cast<uint32_t *>(fd.digest)[lane] = acc;
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
    const uint32_t msgs = b.count * b.n;
    if (!msgs) return cudaSuccess;
    sha_subframes_kernel<<<(msgs + kMsgPerCta - 1) / kMsgPerCta, 64, 0, s>>>(b);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_verify(const Batch &b, uint8_t *ok, cudaStream_t s) {
    const uint32_t msgs = b.count * b.n;
    if (!msgs) return cudaSuccess;
    sha_dst_kernel<<<(msgs + kMsgPerCta - 1) / kMsgPerCta, 64, 0, s>>>(b);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    verify_kernel<<<b.count, 32, 0, s>>>(b, ok);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sha_plain(const uint8_t *data, uint64_t nbytes, uint32_t n, uint32_t count, uint8_t *part,
                             cudaStream_t s) {
    const uint32_t msgs = count * n;
    if (!msgs) return cudaSuccess;
    sha_plain_kernel<<<(msgs + kMsgPerCta - 1) / kMsgPerCta, 64, 0, s>>>(data, nbytes, n, count, part);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_fold_batch(const Batch &b, cudaStream_t s) {
    if (!b.count) return cudaSuccess;
    fold_batch_kernel<<<b.count, 32, 0, s>>>(b);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tree_batch(const Batch &b, cudaStream_t s) {
    if (!b.count) return cudaSuccess;
    tree_batch_kernel<<<(b.count + 31) / 32, 32, 0, s>>>(b);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tree(const uint8_t *part, uint32_t n, uint32_t count, uint8_t *digest, cudaStream_t s) {
    if (!count) return cudaSuccess;
    tree_kernel<<<(count + 31) / 32, 32, 0, s>>>(part, n, count, digest);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_fold(const uint8_t *part, uint32_t n, uint32_t count, uint8_t *digest, cudaStream_t s) {
    if (!count) return cudaSuccess;
    fold_kernel<<<count, 32, 0, s>>>(part, n, count, digest);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fhd

FHD_BOUNDS_TAKER(take_bounds_sha)
