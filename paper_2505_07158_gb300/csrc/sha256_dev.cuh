// Device code of the sub-frame SHA-256 (FIPS 180-4) shared by the digest kernels and the persistent batch
// kernel: the producer/consumer message pipeline and the tree digest.  See sha256.cu for the design.
#pragma once
#include "bounds.cuh"
#include "common.cuh"
#include "sha256_core.cuh"

namespace fhd {
namespace {

__device__ __forceinline__ uint32_t rotr(uint32_t x, int n) { return __funnelshift_r(x, x, n); }
__device__ __forceinline__ uint32_t bswap(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

struct ShaState {
    uint32_t h[8];
    __device__ __forceinline__ void init() { sha256_init(h); }
};

__device__ __forceinline__ void block_words(const uint4 q[4], uint32_t w[16]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        w[4 * k + 0] = bswap(q[k].x);
        w[4 * k + 1] = bswap(q[k].y);
        w[4 * k + 2] = bswap(q[k].z);
        w[4 * k + 3] = bswap(q[k].w);
    }
}

__device__ __forceinline__ void store_digest(uint8_t *dst, const uint32_t h[8]) {
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);   // 32-byte slots, 4-byte aligned
#pragma unroll
    for (int k = 0; k < 8; ++k) d[k] = bswap(h[k]);
}

constexpr int kMsgPerCta = 32;
constexpr uint64_t kPrefetchBlocks = 8;
constexpr uint64_t kRing = 4;

// Blocks of a padded message of len bytes (FIPS 180-4 Sec. 5.1.1).
__device__ __forceinline__ uint64_t padded_blocks(uint64_t len) { return (len >> 6) + ((len & 63) + 9 <= 64 ? 1 : 2); }

// Block b of the padded message (p, len) as 16 big-endian words.  cur holds
// block b's raw bytes when it is a full block on the aligned path.
__device__ __forceinline__ void message_block(const uint8_t *p, uint64_t len, uint64_t b, bool aligned16,
                                              const uint4 cur[4], uint32_t w[16]) {
    const uint64_t full = len >> 6;
    if (b < full) {
        if (!FHD_IN(64 * b + 63, len, kSiteShaBlock)) {
#pragma unroll
            for (int k = 0; k < 16; ++k) w[k] = 0;
            return;
        }
        if (aligned16) {
            block_words(cur, w);
        } else {
            const uint8_t *q = p + 64 * b;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                w[k] = ((uint32_t)q[4 * k] << 24) | ((uint32_t)q[4 * k + 1] << 16) | ((uint32_t)q[4 * k + 2] << 8) |
                       (uint32_t)q[4 * k + 3];
        }
        return;
    }
    const uint32_t rem = (uint32_t)(len & 63);
    const uint32_t blk = (uint32_t)(b - full);           // 0 or 1 within the tail
    const uint8_t *tail = p + 64 * full;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        uint32_t word = 0;
#pragma unroll
        for (int byte = 0; byte < 4; ++byte) {
            const uint32_t pos = blk * 64 + 4 * k + byte;
            uint32_t v = 0;
            if (pos < rem) v = tail[pos];
            else if (pos == rem) v = 0x80u;
            word = (word << 8) | v;
        }
        w[k] = word;
    }
    if (b == padded_blocks(len) - 1) {
        const uint64_t bits = len * 8;
        w[14] = (uint32_t)(bits >> 32);
        w[15] = (uint32_t)bits;
    }
}

// 16-byte asynchronous global -> shared copy (Ampere-class cp.async, L2 only), its commit and wait.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The producer and consumer warps of one pipeline meet at hardware barrier `id` (64 threads).
__device__ __forceinline__ void named_barrier_64(uint32_t id) {
    __syncwarp();
    asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

// Shared memory of one pipeline: the W + K ring the consumer reads and the block ring the producer fills.
struct ShaSmem {
    uint32_t wk[2][64][32];
    uint4 ring[4][4][32];
};

// 32 messages per pipeline: of its 64 threads (rtid 0..63), warp 0 compresses and warp 1 produces W + K.
// Pipeline `unit` takes messages 32 unit .. 32 unit + 31 of the nmsg messages; message m is located by
// locate(m, p, len, out) and its digest goes to out (32 bytes); locate returns false for a message that
// failed a range check (checked builds), which is then skipped.  `bar` is the hardware barrier id the
// pipeline's two warps use.
template <class Locate>
__device__ void sha_pipeline(Locate locate, uint32_t nmsg, uint32_t unit, uint32_t rtid, uint32_t bar, ShaSmem &sm) {
    uint32_t(*wk)[64][kMsgPerCta] = sm.wk;
    const int lane = rtid & 31;
    const bool producer = rtid >= 32;
    const uint32_t m = unit * kMsgPerCta + lane;
    bool active = m < nmsg;
    const uint8_t *p = nullptr;
    uint64_t len = 0;
    uint8_t *out = nullptr;
    if (active) active = locate(m, p, len, out);
    const uint64_t nb = active ? padded_blocks(len) : 0;
    const uint64_t NB = __reduce_max_sync(0xffffffffu, (unsigned)nb);   // < 2^32 blocks per message
    if (producer) {
        // Message bytes reach shared memory by cp.async, kRing - 1 blocks ahead of the block being
        // expanded (one commit group per block, empty when the lane has nothing to copy), so no
        // register waits on a load in flight; an L2 prefetch runs kPrefetchBlocks ahead of that.
        uint4(*ring)[4][kMsgPerCta] = sm.ring;
        const bool al = (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
        const uint64_t full = len >> 6;
        auto issue = [&](uint64_t blk) {
            if (active && al && blk < full && FHD_IN(64 * blk + 63, len, kSiteShaBlock)) {
#pragma unroll
                for (int q = 0; q < 4; ++q) cp_async16(&ring[blk % kRing][q][lane], p + 64 * blk + 16 * q);
            }
            cp_async_commit();
        };
        for (uint64_t k = 0; k + 1 < kRing; ++k) issue(k);
        for (uint64_t b = 0; b < NB; ++b) {
            // Refills the slot of block b - 1, whose bytes were consumed in the previous iteration.
            issue(b + kRing - 1);
            if (b < nb) {
                if (b + kPrefetchBlocks < full) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + 64 * (b + kPrefetchBlocks)));
                cp_async_wait<kRing - 1>();     // block b has landed
                uint4 cur[4];
                if (al && b < full) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) cur[q] = ring[b % kRing][q][lane];
                }
                uint32_t w[16];
                message_block(p, len, b, al, cur, w);
                uint32_t(*dst)[kMsgPerCta] = wk[b & 1];
#pragma unroll
                for (int t = 0; t < 64; ++t) {
                    uint32_t wt;
                    if (t < 16) {
                        wt = w[t];
                    } else {
                        const uint32_t w15 = w[(t - 15) & 15], w2 = w[(t - 2) & 15];
                        const uint32_t s0 = rotr(w15, 7) ^ rotr(w15, 18) ^ (w15 >> 3);
                        const uint32_t s1 = rotr(w2, 17) ^ rotr(w2, 19) ^ (w2 >> 10);
                        wt = w[t & 15] + s0 + w[(t - 7) & 15] + s1;
                        w[t & 15] = wt;
                    }
                    dst[t][lane] = wt + kSha256K[t];
                }
            }
            named_barrier_64(bar);                 // block b is ready; block b-1 has been consumed
        }
        named_barrier_64(bar);                     // pairs with the consumer's last wait
        cp_async_wait<0>();
    } else {
        ShaState st;
        st.init();
        named_barrier_64(bar);                     // block 0 ready
        for (uint64_t b = 0; b < NB; ++b) {
            if (b < nb) {
                const uint32_t(*src)[kMsgPerCta] = wk[b & 1];
                // all 64 W+K words into registers first: the rounds never wait on shared memory
                uint32_t wkr[64];
#pragma unroll
                for (int t = 0; t < 64; ++t) wkr[t] = src[t][lane];
                uint32_t a = st.h[0], bb = st.h[1], c = st.h[2], d = st.h[3];
                uint32_t e = st.h[4], f = st.h[5], g = st.h[6], hh = st.h[7];
                // The round written so that only Sigma1(e) and Ch(e, f, g) sit on the e -> e' chain:
                // h + K + W and d + h + K + W use values known three rounds ahead (h = e, d = a
                // of round t - 3), so e' = (d + h + K + W) + Sigma1 + Ch is shift, LOP3, IADD3.
#pragma unroll
                for (int t = 0; t < 64; ++t) {
                    const uint32_t hk = hh + wkr[t];
                    const uint32_t dhk = d + hk;
                    const uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
                    const uint32_t ch = (e & f) ^ (~e & g);
                    const uint32_t S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
                    const uint32_t mj = (a & bb) ^ (a & c) ^ (bb & c);
                    const uint32_t t1 = hk + S1 + ch;
                    hh = g; g = f; f = e; e = dhk + S1 + ch;
                    d = c; c = bb; bb = a; a = t1 + S0 + mj;
                }
                st.h[0] += a; st.h[1] += bb; st.h[2] += c; st.h[3] += d;
                st.h[4] += e; st.h[5] += f; st.h[6] += g; st.h[7] += hh;
            }
            named_barrier_64(bar);                 // done with block b; block b+1 ready
        }
        if (active) store_digest(out, st.h);
    }
}

// Tree digest (an option of this library, not of the paper): SHA-256 of the n sub-frame digests at `part`
// concatenated in order, 32 n bytes; one thread.  The stored digests are big-endian bytes, so each message
// word is the byte swap of a stored 32-bit word.  32 n bytes end on a half or a whole 64-byte block: the
// padding (0x80, zeros, the 64-bit bit length 256 n) always fits in the last block.
__device__ void tree_digest(const uint8_t *part, uint32_t n, uint32_t h[8]) {
    ShaState st;
    st.init();
    const uint32_t *p = reinterpret_cast<const uint32_t *>(part);
    const uint32_t words = 8 * n;
    uint32_t w[16];
    uint32_t i = 0;
    for (; i + 16 <= words; i += 16) {
#pragma unroll
        for (int k = 0; k < 16; ++k) w[k] = bswap(__ldcg(p + i + k));
        sha256_compress(st.h, w);
    }
    const uint32_t rem = words - i;   // 0 or 8
#pragma unroll
    for (int k = 0; k < 16; ++k) w[k] = (uint32_t)k < rem ? bswap(__ldcg(p + i + k)) : 0u;
    w[rem] = 0x80000000u;
    const uint64_t bits = 256ull * n;
    w[14] = (uint32_t)(bits >> 32);
    w[15] = (uint32_t)bits;
    sha256_compress(st.h, w);
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = st.h[k];
}

}  // namespace
}  // namespace fhd
