// K3 / K4: the bit-level confusion + XOR of Sec. II-C (Algos 3-7) and its
// exact inverse, as two coalesced passes per frame.
//
// The paper expands every pixel into 8 bits of an [8w x h] matrix (Algo 3),
// rotates each row's bitstring by d_h (Algo 4), rotates each pixel column by
// d_v rows (Algo 5), XORs with B (Algo 6) and packs the bits (Algo 7).  With
// the least-significant-bit-first expansion of Algo 3, a channel row's
// bitstring is its little-endian byte string, so a row rotation by
// s = 8a + r bits is a byte rotation by a plus a funnel shift by r: for four
// consecutive output bytes of one channel row, with A[0..4] the source bytes
// at pixels j - a - 1 .. j - a + 3 (mod w) packed little-endian into a 40-bit
// value V, the four rotated bytes are the low 32 bits of V >> (8 - r).  No bit
// matrix is materialised.  With s_h(i, c) = D[c*h + i] mod 8w and
// s_v(j, c) = D[C*h + c*w + j] mod h:
//   G[i, j, c] = rowrot(F[i, :, c], s_h(i, c))[j]            (row pass, Algo 4)
//   E[i, j, c] = B[i, j, c] ^ G[(i - s_v(j, c)) mod h, j, c]  (column pass, Algos 5-6)
//
// Row pass: a CTA stages a band of whole rows in shared memory with 16-byte
// loads, every thread builds four output bytes of one channel with one
// funnel shift, and the band leaves with 16-byte stores.  Column pass: a CTA
// owns a full-height strip of P pixel columns; 16-byte loads of the strip's
// row segments, each byte scattered into its vertically rotated row of the
// shared strip, then the strip leaves row by row XORed with B in 16-byte
// stores.  Both passes read and write whole rows or row segments, so every
// global access is a coalesced vector; the intermediate frame G lives in the
// keystream scratch.  Decryption runs the column pass first (E ^ B scattered
// to un-rotated rows) and then the row pass rotating right.
#include "common.cuh"

namespace fhd {
namespace {

constexpr int kStripThreads = 512;
constexpr int kRowThreads = 256;
constexpr int kRowsV = 4;                 // row segments per batch of independent vector loads
constexpr int kRowsW = 8;                 // strip rows per batch of independent word loads (column pass)
constexpr size_t kSmemLimit = 232448;     // opt-in dynamic shared memory per CTA on sm_100/sm_103
constexpr size_t kRowSmemTarget = 32768;  // row pass: bands of 2 rows at 1080p

// n mod d for n < 2^16, 1 <= d <= 2^18, by one 64-bit multiply: with
// M = floor(2^40/d) + 1 and e = M d - 2^40 in (0, d], n M / 2^40 exceeds n/d
// by n e / (d 2^40) < 1/d, so its floor is floor(n/d).
struct FastMod {
    uint32_t d;
    unsigned long long M;
    __device__ __forceinline__ explicit FastMod(uint32_t dd) : d(dd), M((1ull << 40) / dd + 1) {}
    __device__ __forceinline__ uint32_t mod(uint32_t n) const {
        uint32_t q = (uint32_t)(((unsigned long long)n * M) >> 40);
        return n - q * d;
    }
};

// Last frame whose first CTA (strip or row numbering) is <= cta.
template <bool kRow>
__device__ __forceinline__ uint32_t find_frame(const Batch &b, uint32_t cta) {
    uint32_t lo = 0, hi = b.count;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if ((kRow ? b.f[mid].rcta0 : b.f[mid].cta0) <= cta) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool aligned(const void *p, uintptr_t a) {
    return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0;
}

// Vector width (1, 4 or 16 bytes) usable for contiguous strip rows.
__device__ __forceinline__ uint32_t strip_vec(uint64_t rowB, uint32_t P, uint32_t C, uint32_t Pe, const void *p0,
                                              const void *p1, const void *p2) {
    if (rowB % 16 == 0 && (P * C) % 16 == 0 && (Pe * C) % 16 == 0 && aligned(p0, 16) && aligned(p1, 16) &&
        aligned(p2, 16))
        return 16;
    if (rowB % 4 == 0 && (P * C) % 4 == 0 && (Pe * C) % 4 == 0 && aligned(p0, 4) && aligned(p1, 4) && aligned(p2, 4))
        return 4;
    return 1;
}

// Column pass.  Encrypt: S[(i + s_v) mod h][q] = G[i][q]; E = S ^ B.
// Decrypt: S[(i - s_v) mod h][q] = (E ^ B)[i][q]; G = S.
template <bool kEnc>
__global__ void __launch_bounds__(kStripThreads, 2) strip_kernel(const __grid_constant__ Batch b, uint32_t cta_base) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t cta = cta_base + blockIdx.x;
    const FrameDesc &fd = b.f[find_frame<false>(b, cta)];
    const uint32_t h = fd.h, w = fd.w, C = fd.C, P = fd.P;
    const uint32_t j0 = (cta - fd.cta0) * P;
    const uint32_t Pe = min(P, w - j0);
    const uint32_t RP = P * C;
    const uint32_t QC = Pe * C;
    const uint64_t rowB = (uint64_t)w * C;
    const uint64_t base = (uint64_t)j0 * C;
    const uint8_t *src = kEnc ? fd.G : fd.src;
    uint8_t *out = kEnc ? fd.dst : fd.G;
    const uint16_t *Dv = fd.D + (uint64_t)C * h;
    const FastMod modH(h);
    uint8_t *S = smem;

    // ---- phase 1: loads of the strip rows, bytes scattered to their rotated rows.  With 4-byte-aligned
    // rows a lane owns one 32-bit word of the strip row (the lanes of a warp hold consecutive words), so
    // in each byte store the lanes hit consecutive banks up to the row term 16 d (mod 32): at most two
    // lanes share a bank.
    const uint32_t vec = strip_vec(rowB, P, C, Pe, src, out, fd.B);
    if (vec >= 4) {
        const uint32_t nw = QC / 4;                    // words per strip row
        const uint32_t RT = blockDim.x / nw;           // rows in parallel
        if (threadIdx.x < nw * RT) {
            const uint32_t j = threadIdx.x % nw, tr = threadIdx.x / nw;
            uint32_t ht[4];   // row offset of each byte: s_v (encrypt) or h - s_v (decrypt)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t q = 4 * j + k, jj = q / C, c = q - jj * C;
                const uint32_t t = modH.mod(Dv[(uint64_t)c * w + j0 + jj]);
                ht[k] = kEnc ? t : h - t;
            }
            const uint8_t *sp = src + base + 4 * j;
            const uint8_t *bp = fd.B + base + 4 * j;
            for (uint32_t ib = tr; ib < h; ib += kRowsW * RT) {
                uint32_t e[kRowsW];
#pragma unroll
                for (int k = 0; k < kRowsW; ++k) {
                    const uint32_t i = ib + k * RT;
                    if (i < h) {
                        e[k] = __ldcs(reinterpret_cast<const unsigned int *>(sp + (uint64_t)i * rowB));
                        if (!kEnc) e[k] ^= __ldcs(reinterpret_cast<const unsigned int *>(bp + (uint64_t)i * rowB));
                    }
                }
#pragma unroll
                for (int k = 0; k < kRowsW; ++k) {
                    const uint32_t i = ib + k * RT;
                    if (i < h) {
#pragma unroll
                        for (int bb = 0; bb < 4; ++bb) {
                            uint32_t d = i + ht[bb];
                            d = d >= h ? d - h : d;
                            S[(size_t)d * RP + 4 * j + bb] = (uint8_t)(e[k] >> (8 * bb));
                        }
                    }
                }
            }
        }
    } else {
        const uint32_t RT = blockDim.x / QC;
        if (threadIdx.x < QC * RT) {
            const uint32_t q = threadIdx.x % QC, tr = threadIdx.x / QC;
            const uint32_t jj = q / C, c = q - jj * C;
            const uint32_t t = modH.mod(Dv[(uint64_t)c * w + j0 + jj]);
            const uint32_t ht = kEnc ? t : h - t;
            for (uint32_t i = tr; i < h; i += RT) {
                const uint64_t o = (uint64_t)i * rowB + base + q;
                uint8_t e = src[o];
                if (!kEnc) e ^= fd.B[o];
                uint32_t d = i + ht;
                d = d >= h ? d - h : d;
                S[(size_t)d * RP + q] = e;
            }
        }
    }
    __syncthreads();

    // ---- phase 2: the strip leaves row by row (XORed with B when encrypting)
    const uint32_t nv = QC / vec;
    const uint32_t RT = blockDim.x / nv;
    if (threadIdx.x >= nv * RT) return;
    const uint32_t tv = threadIdx.x % nv, tr = threadIdx.x / nv;
    if (vec == 16) {
        for (uint32_t ib = tr; ib < h; ib += kRowsV * RT) {
            uint4 g[kRowsV], k4[kRowsV];
#pragma unroll
            for (int k = 0; k < kRowsV; ++k) {
                const uint32_t i = ib + k * RT;
                if (i < h) {
                    g[k] = *reinterpret_cast<const uint4 *>(S + (size_t)i * RP + 16 * tv);
                    if (kEnc) k4[k] = __ldcs(reinterpret_cast<const uint4 *>(fd.B + (uint64_t)i * rowB + base + 16 * tv));
                }
            }
#pragma unroll
            for (int k = 0; k < kRowsV; ++k) {
                const uint32_t i = ib + k * RT;
                if (i < h) {
                    uint4 v = g[k];
                    if (kEnc) { v.x ^= k4[k].x; v.y ^= k4[k].y; v.z ^= k4[k].z; v.w ^= k4[k].w; }
                    uint4 *dstp = reinterpret_cast<uint4 *>(out + (uint64_t)i * rowB + base + 16 * tv);
                    if (kEnc) __stcs(dstp, v); else *dstp = v;
                }
            }
        }
    } else if (vec == 4) {
        for (uint32_t i = tr; i < h; i += RT) {
            const uint64_t o = (uint64_t)i * rowB + base + 4 * tv;
            uint32_t g = *reinterpret_cast<const uint32_t *>(S + (size_t)i * RP + 4 * tv);
            if (kEnc) g ^= *reinterpret_cast<const uint32_t *>(fd.B + o);
            *reinterpret_cast<uint32_t *>(out + o) = g;
        }
    } else {
        for (uint32_t i = tr; i < h; i += RT) {
            const uint64_t o = (uint64_t)i * rowB + base + tv;
            uint8_t g = S[(size_t)i * RP + tv];
            if (kEnc) g ^= fd.B[o];
            out[o] = g;
        }
    }
}

// Row pass over a band of RB whole rows.  Encrypt: G = left rotation of each
// channel row of F by s_h bits.  Decrypt: output = right rotation of each
// channel row of G by s_h bits.
//
// Interleaved RGB rows with w % 4 == 0 take a planar route: a thread
// produces one 4-pixel group (12 bytes): for each channel the two words of
// the channel plane that hold its source bytes are deinterleaved from the
// staged row with __byte_perm (the five source bytes sit in two adjacent
// plane words), one 64-to-32-bit funnel shift by 8*(byte offset) + bit shift
// gives the four rotated bytes, and the three channels' words are
// interleaved back.  Other shapes take the byte-wise route.
template <bool kEnc>
__global__ void __launch_bounds__(kRowThreads) row_kernel(const __grid_constant__ Batch b, uint32_t cta_base) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t cta = cta_base + blockIdx.x;
    const FrameDesc &fd = b.f[find_frame<true>(b, cta)];
    const uint32_t h = fd.h, w = fd.w, C = fd.C, RB = fd.RB;
    const uint32_t i0 = (cta - fd.rcta0) * RB;
    const uint32_t nr = min(RB, h - i0);
    const uint32_t rowB = w * C;
    const uint32_t pitch = (rowB + 15) & ~15u;
    const uint8_t *src = (kEnc ? fd.src : fd.G) + (uint64_t)i0 * rowB;
    uint8_t *dst = (kEnc ? fd.G : fd.dst) + (uint64_t)i0 * rowB;
    uint8_t *In = smem;                                          // RB rows
    uint8_t *Out = smem + (size_t)RB * pitch;                    // RB rows
    uint32_t *sh = reinterpret_cast<uint32_t *>(smem + 2 * (size_t)RB * pitch);   // row shifts [r * C + c]
    const FastMod modW8(8 * w);

    // ---- load the band (rows are contiguous in global memory)
    const bool v16 = rowB % 16 == 0 && aligned(src, 16) && aligned(dst, 16);
    if (v16) {
        const uint32_t nvr = rowB / 16;
        for (uint32_t k = threadIdx.x; k < nr * nvr; k += blockDim.x) {
            const uint32_t r = k / nvr, v = k - r * nvr;
            *reinterpret_cast<uint4 *>(In + (size_t)r * pitch + 16 * v) =
                __ldcs(reinterpret_cast<const uint4 *>(src + (uint64_t)r * rowB + 16 * v));
        }
    } else {
        for (uint32_t k = threadIdx.x; k < nr * rowB; k += blockDim.x) {
            const uint32_t r = k / rowB, q = k - r * rowB;
            In[(size_t)r * pitch + q] = src[(uint64_t)r * rowB + q];
        }
    }
    for (uint32_t k = threadIdx.x; k < nr * C; k += blockDim.x) {
        const uint32_t r = k / C, c = k - r * C;
        sh[k] = modW8.mod(fd.D[(uint64_t)c * h + i0 + r]);
    }
    __syncthreads();

    if (C == 3 && (w & 3) == 0 && v16) {
        // ---- planar route, one pass: a thread builds the 12 output bytes of one 4-pixel group.  For each
        // channel the two source words of its plane are deinterleaved on the fly from the staged row (a
        // plane word u is the channel's bytes of the interleaved words 3u .. 3u+2), rotated with one
        // funnel shift, and the three rotated plane words are interleaved back into Out.  With w % 4 == 0
        // the source offset within a plane word is the same for every group of a channel row, so a row
        // needs only a word offset and a shift amount per channel.
        const uint32_t W4 = w >> 2;
        uint8_t *Outp = Out;
        for (uint32_t r = 0; r < nr; ++r) {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(In + (size_t)r * pitch);
            uint32_t *orow = reinterpret_cast<uint32_t *>(Outp + (size_t)r * pitch);
            uint32_t du[3], fs[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const uint32_t sc = sh[r * 3 + c];
                const uint32_t a = sc >> 3, rr = sc & 7;
                // first source byte of the plane for output pixel 0: -a-1 (encrypt) or a (decrypt), mod w
                int s0 = kEnc ? -(int)a - 1 : (int)a;
                if (s0 < 0) s0 += (int)w;
                du[c] = (uint32_t)s0 >> 2;
                const uint32_t o = (uint32_t)s0 & 3;
                fs[c] = kEnc ? 8 * o + 8 - rr : 8 * o + rr;
            }
            for (uint32_t g = threadIdx.x; g < W4; g += blockDim.x) {
                uint32_t q[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    uint32_t u = g + du[c];
                    u = u >= W4 ? u - W4 : u;
                    const uint32_t u1 = u + 1 == W4 ? 0 : u + 1;
                    const uint32_t a0 = row[3 * u], a1 = row[3 * u + 1], a2 = row[3 * u + 2];
                    const uint32_t b0 = row[3 * u1], b1 = row[3 * u1 + 1], b2 = row[3 * u1 + 2];
                    uint32_t lo, hi;
                    if (c == 0) {
                        lo = __byte_perm(__byte_perm(a0, a1, 0x0630), a2, 0x5210);
                        hi = __byte_perm(__byte_perm(b0, b1, 0x0630), b2, 0x5210);
                    } else if (c == 1) {
                        lo = __byte_perm(__byte_perm(a0, a1, 0x0741), a2, 0x6210);
                        hi = __byte_perm(__byte_perm(b0, b1, 0x0741), b2, 0x6210);
                    } else {
                        lo = __byte_perm(__byte_perm(a0, a1, 0x0052), a2, 0x7410);
                        hi = __byte_perm(__byte_perm(b0, b1, 0x0052), b2, 0x7410);
                    }
                    q[c] = __funnelshift_rc(lo, hi, fs[c]);
                }
                uint32_t *wp = orow + 3 * g;
                wp[0] = __byte_perm(__byte_perm(q[0], q[1], 0x1040), q[2], 0x3410);
                wp[1] = __byte_perm(__byte_perm(q[1], q[0], 0x2601), q[2], 0x3250);
                wp[2] = __byte_perm(__byte_perm(q[2], q[0], 0x3072), q[1], 0x3710);
            }
        }
        __syncthreads();
        const uint32_t nvr = rowB / 16;
        for (uint32_t r = 0; r < nr; ++r)
            for (uint32_t v = threadIdx.x; v < nvr; v += blockDim.x)
                *reinterpret_cast<uint4 *>(dst + (uint64_t)r * rowB + 16 * v) =
                    *reinterpret_cast<const uint4 *>(Outp + (size_t)r * pitch + 16 * v);
        return;
    }

    // ---- byte-wise route: four output bytes of one channel per thread, one funnel shift each
    const uint32_t nq = (w + 3) >> 2;
    for (uint32_t rc = 0; rc < nr * C; ++rc) {
        const uint32_t r = rc / C, c = rc - r * C;
        const uint32_t s = sh[rc];
        const uint32_t a = s >> 3, rr = s & 7;
        const uint8_t *row = In + (size_t)r * pitch + c;
        uint8_t *orow0 = Out + (size_t)r * pitch + c;
        for (uint32_t k = threadIdx.x; k < nq; k += blockDim.x) {
            const uint32_t j = 4 * k;
            const uint32_t nm = min(4u, w - j);
            // first source pixel: j - a - 1 (encrypt) or j + a (decrypt), mod w
            int p0 = kEnc ? (int)j - (int)a - 1 : (int)(j + a);
            if (p0 < 0) p0 += (int)w;
            if (p0 >= (int)w) p0 -= (int)w;
            uint32_t A0, A1, A2, A3, A4;
            if ((uint32_t)p0 + 4 < w) {
                const uint8_t *p = row + (uint32_t)p0 * C;
                A0 = p[0]; A1 = p[C]; A2 = p[2 * C]; A3 = p[3 * C]; A4 = p[4 * C];
            } else {
                uint32_t q = (uint32_t)p0;
                A0 = row[q * C]; q = q + 1 == w ? 0 : q + 1;
                A1 = row[q * C]; q = q + 1 == w ? 0 : q + 1;
                A2 = row[q * C]; q = q + 1 == w ? 0 : q + 1;
                A3 = row[q * C]; q = q + 1 == w ? 0 : q + 1;
                A4 = row[q * C];
            }
            const uint32_t X = A0 | (A1 << 8) | (A2 << 16) | (A3 << 24);
            const uint32_t o = __funnelshift_r(X, A4, kEnc ? 8 - rr : rr);
            uint8_t *orow = orow0 + j * C;
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if ((uint32_t)m < nm) orow[(uint32_t)m * C] = (uint8_t)(o >> (8 * m));
        }
    }
    __syncthreads();

    // ---- store the band
    if (v16) {
        const uint32_t nvr = rowB / 16;
        for (uint32_t k = threadIdx.x; k < nr * nvr; k += blockDim.x) {
            const uint32_t r = k / nvr, v = k - r * nvr;
            *reinterpret_cast<uint4 *>(dst + (uint64_t)r * rowB + 16 * v) =
                *reinterpret_cast<const uint4 *>(Out + (size_t)r * pitch + 16 * v);
        }
    } else {
        for (uint32_t k = threadIdx.x; k < nr * rowB; k += blockDim.x) {
            const uint32_t r = k / rowB, q = k - r * rowB;
            dst[(uint64_t)r * rowB + q] = Out[(size_t)r * pitch + q];
        }
    }
}

// Single-pass encryption (row rotation, column rotation and XOR in one kernel) for interleaved RGB frames
// with w % 16 == 0, strip widths P in {16, 32, 64} and 16-byte aligned buffers.  A CTA owns a full-height
// strip of P pixel columns of the output.
//
// Phase 1 builds the strip of G (the row-rotated frame) directly from F.  For source row i' and channel c,
// the P output plane bytes of the strip are the rotation of a window of P/4 + 1 plane words of F's
// channel-c plane at the row's offset (mod w); in the interleaved row those are 12 (P/4 + 1) consecutive
// bytes (mod the row length).  Each warp takes a few source rows at a time: its lanes copy the rows'
// 3 windows into a per-warp staging buffer as 16-byte chunks (coalesced loads of whole sectors, the
// window rounded out to 16-byte boundaries), issued one iteration ahead into registers; then each unit --
// two plane words, eight pixels of channel c -- reads its three plane words' interleaved words from the
// buffer, deinterleaves them with byte permutes, makes its eight rotated bytes with two funnel shifts, and
// stores each byte into its vertically rotated row of the shared strip, S[(i' + s_v(j, c)) mod h][j, c]
// (Algo 5).  Phase 2 streams the strip out row by row XORed with B (Algo 6) in 16-byte loads and
// stores.  DRAM traffic is one read of F and B and one write of E: G never exists in memory.
constexpr int kGatherWarps = 12;
constexpr int kGatherThreads = 32 * kGatherWarps;

template <int P>
struct GatherShape {
    static constexpr uint32_t G4 = P / 4;                             // plane words per strip row and channel
    static constexpr uint32_t G2 = P / 8;                             // units per window
    static constexpr uint32_t RW = 32 / (3 * G2);                     // source rows per warp and iteration
    static constexpr uint32_t NW = 3 * RW;                            // windows per warp and iteration
    static constexpr uint32_t NC = (12 * (G4 + 1) + 12 + 15) / 16;    // 16-byte chunks per window (bound)
    static constexpr uint32_t NCH = NW * NC;                          // chunks per warp and iteration
    static constexpr uint32_t CPL = (NCH + 31) / 32;                  // chunks per lane
};

// Shared memory of the gather route for a strip of height h and width P: the strip, the per-warp staging
// buffers and the row-rotation table.
__host__ __device__ constexpr size_t gather_stage_bytes(uint32_t P) {
    return (size_t)kGatherWarps * 16 *
           (P == 16 ? GatherShape<16>::NCH : P == 32 ? GatherShape<32>::NCH : GatherShape<64>::NCH);
}

__device__ __forceinline__ uint32_t plane_word(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t s1, uint32_t s2) {
    return __byte_perm(__byte_perm(w0, w1, s1), w2, s2);
}

// Row rotation of a channel row with distance d for the gather: the source window of output plane word g
// starts at plane word (g + du) mod W4 and the four rotated bytes are the funnel shift by fs (1..32) of
// that plane word and the next.
struct RowRot {
    uint32_t du, fs;
};
__device__ __forceinline__ RowRot row_rot(uint32_t d, uint32_t w, const FastMod &modW8) {
    const uint32_t sh = modW8.mod(d);
    const uint32_t s0 = w - 1 - (sh >> 3);   // first source pixel of output pixel 0: (-a - 1) mod w
    return {s0 >> 2, 8 * (s0 & 3) + 8 - (sh & 7)};
}

template <int P>
__device__ __forceinline__ void gather_phase1(const FrameDesc &fd, uint32_t j0, uint32_t Pe, uint8_t *S,
                                              uint8_t *stage_all, const uint16_t *tab) {
    using GS = GatherShape<P>;
    const uint32_t h = fd.h, w = fd.w, rowB = 3 * w, W4 = w >> 2, RP = 3 * P, hRP = h * RP;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint4 *stage = reinterpret_cast<uint4 *>(stage_all) + warp * GS::NCH;
    const FastMod modH(h), modW8(8 * w);
    const uint32_t Ge2 = Pe >> 3;
    // window lane (lane < NW): window `lane` of an iteration is source row base + lane / 3, channel lane % 3
    const uint32_t wr = lane / 3, wc = lane - 3 * wr;
    // unit lane (lane < NW * G2): window lane / G2, unit g of it
    const uint32_t uwi = lane / GS::G2, g = lane - uwi * GS::G2;
    const uint32_t ur = uwi / 3, c = uwi - 3 * ur;
    const bool unit = lane < GS::NW * GS::G2 && g < Ge2;
    const uint32_t s1 = c == 0 ? 0x0630u : c == 1 ? 0x0741u : 0x0052u;
    const uint32_t s2 = c == 0 ? 0x5210u : c == 1 ? 0x6210u : 0x7410u;
    uint32_t ab[8];   // strip offset of byte m of source row 0: its rotated row s_v, times RP, plus its column
#pragma unroll
    for (int m = 0; m < 8; ++m)
        ab[m] = (unit ? modH.mod(fd.D[3ull * h + (uint64_t)c * w + j0 + 8 * g + m]) : 0) * RP + (8 * g + m) * 3 + c;
    const uint32_t rows_per_it = GS::RW * kGatherWarps;
    const uint32_t iters = (h + rows_per_it - 1) / rows_per_it;
    const uint8_t *src = fd.src;

    // Window parameters of iteration it (window lanes): aligned start A of the window in its row, the
    // offset of the window's first plane word past A, the funnel shift.
    auto params = [&](uint32_t it, uint32_t &A, uint32_t &off, uint32_t &fs) {
        const uint32_t i = (it * kGatherWarps + warp) * GS::RW + wr;
        A = off = 0;
        fs = 32;
        if (lane < GS::NW && i < h) {
            RowRot r;
            if (tab) {
                const uint32_t v = tab[wc * h + i];
                r.du = v >> 5;
                r.fs = (v & 31) + 1;
            } else {
                r = row_rot(fd.D[(uint64_t)wc * h + i], w, modW8);
            }
            uint32_t us = (j0 >> 2) + r.du;
            us = us >= W4 ? us - W4 : us;
            const uint32_t b0 = 12 * us;
            A = b0 & ~15u;
            off = b0 - A;
            fs = r.fs;
        }
    };
    // Chunk k of this lane in an iteration: window cw[k] (its row cr[k] within the iteration's rows), byte
    // 16 ck[k] of the window; fixed per lane.
    uint32_t cw[GS::CPL], cr[GS::CPL], ck16[GS::CPL];
#pragma unroll
    for (uint32_t k = 0; k < GS::CPL; ++k) {
        const uint32_t q = lane + 32 * k;
        const uint32_t wi = q < GS::NCH ? q / GS::NC : 0;
        cw[k] = wi;
        cr[k] = q < GS::NCH ? wi / 3 : h;   // row h: never loaded
        ck16[k] = 16 * (q - wi * GS::NC);
    }
    const bool short_row = 16 * GS::NC > rowB;   // the window may wrap around the row end more than once
    auto fetch = [&](uint32_t it, uint32_t A, uint4 (&reg)[GS::CPL]) {
        const uint32_t base = (it * kGatherWarps + warp) * GS::RW;
#pragma unroll
        for (uint32_t k = 0; k < GS::CPL; ++k) {
            const uint32_t Aw = __shfl_sync(0xffffffffu, A, cw[k]);
            const uint32_t i = base + cr[k];
            reg[k] = make_uint4(0, 0, 0, 0);
            if (i < h) {
                uint32_t o = Aw + ck16[k];
                o = o >= rowB ? o - rowB : o;
                if (short_row)
                    while (o >= rowB) o -= rowB;
                // F rows serve several strips: keep them in L2
                reg[k] = __ldcg(reinterpret_cast<const uint4 *>(src + i * rowB + o));
            }
        }
    };
    uint32_t A, off, fs;
    uint4 reg[GS::CPL];
    params(0, A, off, fs);
    fetch(0, A, reg);
    for (uint32_t it = 0; it < iters; ++it) {
        // the staging buffer takes iteration it's chunks once the previous iteration has read it
        __syncwarp();
#pragma unroll
        for (uint32_t k = 0; k < GS::CPL; ++k)
            if (lane + 32 * k < GS::NCH) stage[lane + 32 * k] = reg[k];
        const uint32_t cur_off = off, cur_fs = fs;
        if (it + 1 < iters) {   // next iteration's window parameters and chunk loads, in flight meanwhile
            params(it + 1, A, off, fs);
            fetch(it + 1, A, reg);
        }
        __syncwarp();
        const uint32_t uoff = __shfl_sync(0xffffffffu, cur_off, uwi < GS::NW ? uwi : 0);
        const uint32_t ufs = __shfl_sync(0xffffffffu, cur_fs, uwi < GS::NW ? uwi : 0);
        const uint32_t i = (it * kGatherWarps + warp) * GS::RW + ur;
        if (unit && i < h) {
            const uint32_t *wd = reinterpret_cast<const uint32_t *>(
                reinterpret_cast<const uint8_t *>(stage + uwi * GS::NC) + uoff + 24 * g);
            const uint32_t x0 = plane_word(wd[0], wd[1], wd[2], s1, s2);
            const uint32_t x1 = plane_word(wd[3], wd[4], wd[5], s1, s2);
            const uint32_t x2 = plane_word(wd[6], wd[7], wd[8], s1, s2);
            const uint32_t q0 = __funnelshift_rc(x0, x1, ufs);
            const uint32_t q1 = __funnelshift_rc(x1, x2, ufs);
            const uint32_t iRP = i * RP;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                uint32_t a = iRP + ab[m];
                a = a >= hRP ? a - hRP : a;
                S[a] = (uint8_t)((m < 4 ? q0 : q1) >> (8 * (m & 3)));
            }
        }
    }
}

__global__ void __launch_bounds__(kGatherThreads, 2) gather_encrypt_kernel(const __grid_constant__ Batch b,
                                                                           uint32_t cta_base, int use_tab) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t cta = cta_base + blockIdx.x;
    const FrameDesc &fd = b.f[find_frame<false>(b, cta)];
    const uint32_t h = fd.h, w = fd.w, P = fd.P;
    const uint32_t j0 = (cta - fd.cta0) * P;
    const uint32_t Pe = min(P, w - j0);
    const uint32_t RP = 3 * P, QC = 3 * Pe, rowB = 3 * w;
    const uint32_t t = threadIdx.x;
    uint8_t *S = smem;
    uint8_t *stage = smem + (((size_t)h * RP + 15) & ~(size_t)15);
    uint16_t *tab = use_tab ? reinterpret_cast<uint16_t *>(stage + gather_stage_bytes(P)) : nullptr;
    if (tab) {   // [c * h + i] = du << 5 | (fs - 1); du < W4 <= 1024
        const FastMod modW8(8 * w);
        for (uint32_t k = t; k < 3 * h; k += kGatherThreads) {
            const RowRot r = row_rot(fd.D[k], w, modW8);
            tab[k] = (uint16_t)((r.du << 5) | (r.fs - 1));
        }
        __syncthreads();
    }
    if (P == 16) gather_phase1<16>(fd, j0, Pe, S, stage, tab);
    else if (P == 32) gather_phase1<32>(fd, j0, Pe, S, stage, tab);
    else gather_phase1<64>(fd, j0, Pe, S, stage, tab);
    __syncthreads();

    // ---- phase 2: E = S ^ B, row by row, 16-byte vectors
    const uint32_t nv = QC / 16;
    const uint32_t RT = kGatherThreads / nv;
    if (t >= nv * RT) return;
    const uint32_t tv = t % nv, tr = t / nv;
    const uint64_t base = (uint64_t)j0 * 3 + 16 * tv;
    for (uint32_t ib = tr; ib < h; ib += kRowsV * RT) {
        uint4 v[kRowsV], k4[kRowsV];
#pragma unroll
        for (int k = 0; k < kRowsV; ++k) {
            const uint32_t i = ib + k * RT;
            if (i < h) {
                v[k] = *reinterpret_cast<const uint4 *>(S + (size_t)i * RP + 16 * tv);
                k4[k] = __ldcs(reinterpret_cast<const uint4 *>(fd.B + (uint64_t)i * rowB + base));
            }
        }
#pragma unroll
        for (int k = 0; k < kRowsV; ++k) {
            const uint32_t i = ib + k * RT;
            if (i < h) {
                uint4 o = v[k];
                o.x ^= k4[k].x; o.y ^= k4[k].y; o.z ^= k4[k].z; o.w ^= k4[k].w;
                __stcs(reinterpret_cast<uint4 *>(fd.dst + (uint64_t)i * rowB + base), o);
            }
        }
    }
}

}  // namespace

size_t strip_smem_bytes(uint32_t h, uint32_t P, uint32_t C) { return ((size_t)h * P * C + 15) & ~(size_t)15; }

uint32_t row_band(uint32_t w, uint32_t C) {
    const size_t pitch = ((size_t)w * C + 15) & ~(size_t)15;
    size_t rb = kRowSmemTarget / (2 * pitch + 16);
    if (rb < 1) rb = 1;
    if (rb > 16) rb = 16;
    return (uint32_t)rb;
}

// Two row-sized buffers per row (input and output) and the row shifts.
size_t row_smem_bytes(uint32_t w, uint32_t C, uint32_t RB) {
    const size_t pitch = ((size_t)w * C + 15) & ~(size_t)15;
    return 2 * (size_t)RB * pitch + 4 * (size_t)RB * C;
}

uint32_t permute_strips(uint32_t w, uint32_t P) { return (w + P - 1) / P; }

static uint32_t g_override_key[64][3];
static uint32_t g_override_P[64];
static int g_overrides = 0;

int set_strip_override(uint32_t h, uint32_t w, uint32_t C, uint32_t P) {
    for (int k = 0; k < g_overrides; ++k)
        if (g_override_key[k][0] == h && g_override_key[k][1] == w && g_override_key[k][2] == C) {
            g_override_P[k] = P;
            return 0;
        }
    if (g_overrides >= 64) return -1;
    g_override_key[g_overrides][0] = h;
    g_override_key[g_overrides][1] = w;
    g_override_key[g_overrides][2] = C;
    g_override_P[g_overrides++] = P;
    return 0;
}

// Widest power-of-two strip (<= 128 pixels, no wider than the frame needs)
// whose column-pass working set fits the opt-in shared memory; an autotuner
// override (if any and if it fits) wins.
uint32_t strip_width(uint32_t h, uint32_t w, uint32_t C) {
    for (int k = 0; k < g_overrides; ++k)
        if (g_override_key[k][0] == h && g_override_key[k][1] == w && g_override_key[k][2] == C && g_override_P[k] &&
            g_override_P[k] <= 128 && strip_smem_bytes(h, g_override_P[k], C) <= kSmemLimit)
            return g_override_P[k];
    uint32_t P = 128;
    while (P > 1 && (P / 2 >= w || strip_smem_bytes(h, P, C) > kSmemLimit)) P /= 2;
    return strip_smem_bytes(h, P, C) <= kSmemLimit ? P : 0;
}

cudaError_t permute_prepare() {
    const void *fns[5] = {(const void *)strip_kernel<true>, (const void *)strip_kernel<false>,
                          (const void *)row_kernel<true>, (const void *)row_kernel<false>,
                          (const void *)gather_encrypt_kernel};
    for (const void *f : fns) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static int g_route = FHD_ROUTE_TWO_PASS;

int set_encrypt_route(int route) {
    if (route != FHD_ROUTE_TWO_PASS && route != FHD_ROUTE_SINGLE_PASS) return -1;
    g_route = route;
    return 0;
}

// The single pass takes a batch whose every frame is interleaved RGB with w % 16 == 0, a strip width that
// is a multiple of 16 and 16-byte aligned source, destination and keystream.
static bool single_pass_ok(const Batch &b) {
    auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    for (uint32_t k = 0; k < b.count; ++k) {
        const FrameDesc &f = b.f[k];
        if (f.C != 3 || f.w % 16 || (f.P != 16 && f.P != 32 && f.P != 64) || !al(f.src) || !al(f.dst) || !al(f.B))
            return false;
    }
    return true;
}

// Encrypt: row pass then column pass, or one gather pass (FHD_ROUTE_SINGLE_PASS) where the batch allows
// it; decrypt: column
// pass then row pass.  (Running the two passes per group of frames, so that a group's intermediate
// frames stay in L2 between its two passes, measured slower: the smaller launches lose more to wave
// tails than L2 residency saves.)
cudaError_t launch_permute(const Batch &b, bool encrypt, cudaStream_t s) {
    if (!b.count || !b.perm_ctas) return cudaSuccess;
    size_t ssm = 0, rsm = 0;
    for (uint32_t k = 0; k < b.count; ++k) {
        const FrameDesc &f = b.f[k];
        const size_t a = strip_smem_bytes(f.h, f.P, f.C), r = row_smem_bytes(f.w, f.C, f.RB);
        ssm = ssm > a ? ssm : a;
        rsm = rsm > r ? rsm : r;
    }
    cudaError_t e;
    if (encrypt && g_route == FHD_ROUTE_SINGLE_PASS && single_pass_ok(b)) {
        // Strip + staging buffers, and the rotation table (3h 16-bit entries) where every frame's plane-word
        // offsets fit in it and it costs no CTA per SM.
        size_t gsm = 0, tsm = 0;
        bool tab = true;
        for (uint32_t k = 0; k < b.count; ++k) {
            const FrameDesc &f = b.f[k];
            const size_t g = strip_smem_bytes(f.h, f.P, f.C) + gather_stage_bytes(f.P);
            gsm = gsm > g ? gsm : g;
            tsm = tsm > g + 6ull * f.h ? tsm : g + 6ull * f.h;
            tab = tab && f.w / 4 <= 1024;
        }
        constexpr size_t kSmPerSm = 233472, kReserved = 1024;
        tab = tab && tsm <= kSmemLimit && kSmPerSm / (tsm + kReserved) >= kSmPerSm / (gsm + kReserved);
        if (gsm <= kSmemLimit) {
            gather_encrypt_kernel<<<b.perm_ctas, kGatherThreads, tab ? tsm : gsm, s>>>(b, 0, tab ? 1 : 0);
            note_launch();
            return cudaGetLastError();
        }
    }
    if (encrypt) {
        row_kernel<true><<<b.row_ctas, kRowThreads, rsm, s>>>(b, 0);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        strip_kernel<true><<<b.perm_ctas, kStripThreads, ssm, s>>>(b, 0);
        note_launch();
    } else {
        strip_kernel<false><<<b.perm_ctas, kStripThreads, ssm, s>>>(b, 0);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        row_kernel<false><<<b.row_ctas, kRowThreads, rsm, s>>>(b, 0);
        note_launch();
    }
    return cudaGetLastError();
}

}  // namespace fhd
