// Device code of the confusion + XOR passes (Sec. II-C, Algos 3-7) and their inverse, shared by the
// permutation kernels and the persistent batch kernel: the column pass over a full-height strip and the row
// pass over a band of rows, each run by a group of threads that meets at a caller-given barrier.  See
// permute.cu for the design.
#pragma once
#include "bounds.cuh"
#include "common.cuh"

namespace fhd {
namespace {

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
// Loads of the passes.  kL2 (the persistent kernel, whose inputs other CTAs of the same launch produce):
// through L2 only, never a possibly stale L1 line; otherwise streaming loads (read once, evict first).
template <bool kL2, class T>
__device__ __forceinline__ T pass_ld(const T *p) {
    if (kL2) return __ldcg(p);
    return __ldcs(p);
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

// 4 x 4 byte transpose: byte m of word r becomes byte r of word m.
__device__ __forceinline__ void transpose4x4(uint32_t &a, uint32_t &b, uint32_t &c, uint32_t &d) {
    const uint32_t t0 = __byte_perm(a, b, 0x5140), t1 = __byte_perm(a, b, 0x7362);
    const uint32_t t2 = __byte_perm(c, d, 0x5140), t3 = __byte_perm(c, d, 0x7362);
    a = __byte_perm(t0, t2, 0x5410);
    b = __byte_perm(t0, t2, 0x7632);
    c = __byte_perm(t1, t3, 0x5410);
    d = __byte_perm(t1, t3, 0x7632);
}

// Column-word layout of a strip (the column pass's shared memory when h % 4 == 0).  A word holds four
// consecutive rows of one byte column (row 4k + r in byte r).  The strip's QC byte columns form NL = QC / 4
// column quads; the word of row quad p and column q = 4 lam + m sits at p * 4NL + m NL + lam.  A thread owns
// one column quad lam and row quads p = p0, p0 + nq, ...: LT threads per row quad (NL, rounded up), so that the
// threads of a warp take one or two row quads and the NL (or NL + 16) words they touch at a time lie in
// distinct banks: with LT = 16 the pitch 4NL must be 16 mod 32.
struct ColWords {
    uint32_t NL, LT;
};
__device__ __forceinline__ ColWords col_words(uint32_t QC) {
    const uint32_t NL = QC >> 2;
    return {NL, NL <= 16 && (NL & 7) == 4 ? 16u : (NL + 31) & ~31u};
}

// Column pass over a strip in the column-word layout: for each column q of the strip, out[d][q] =
// X[(d - s'_q) mod h][q] with s'_q = s_v (encrypt) or h - s_v (decrypt); X = G (encrypt) or E ^ B (decrypt),
// and the output is XORed with B when encrypting.  With s'_q = 4 a + b:
// * phase 1: the thread loads four rows of its four columns (one 32-bit word per row), transposes them into
//   four column words and stores column q's word of row quad k at row quad (k + a) mod h/4: the rotation by
//   whole row quads;
// * phase 2: output row quad t of column q is bytes 4 - b .. 7 - b of the column's words at row quads t - 1
//   and t (one byte permute: the rest of the rotation), transposed back into four row words.
// Every shared access is one 32-bit word per thread in distinct banks; every global access is a 32-bit word
// per thread, consecutive across the threads of a row quad.
template <bool kEnc, bool kL2, class Sync>
__device__ void strip_pass_cw(const FrameDesc &fd, uint32_t j0, uint32_t QC, ColWords cw, uint8_t *smem, uint32_t tid,
                              uint32_t nthr, Sync sync) {
    // row quads per thread and batch: 16 (8 in the persistent kernel, whose task bodies share 128 registers)
    // independent 32-bit loads in flight
    constexpr int kU = kL2 ? 2 : 4;
    const uint32_t h = fd.h, w = fd.w, C = fd.C, H4 = h >> 2, NL = cw.NL, QP = QC;
    const uint64_t rowB = (uint64_t)w * C, base = (uint64_t)j0 * C;
    const uint64_t rw = rowB >> 2;   // 32-bit words per frame row
    const uint8_t *src = kEnc ? fd.G : fd.src;
    uint8_t *out = kEnc ? fd.dst : fd.G;
    uint32_t *S = reinterpret_cast<uint32_t *>(smem);
    [[maybe_unused]] const size_t words = (size_t)H4 * QP;
    const uint32_t lam = tid % cw.LT, p0 = tid / cw.LT, nq = nthr / cw.LT;
    const bool live = lam < NL;
    // per column m of the thread's quad: whole row quads of the rotation (16 bits each) and the rest (2 bits)
    uint32_t a01 = 0, a23 = 0, bs = 0;
    const uint32_t *sp = reinterpret_cast<const uint32_t *>(src + base) + lam;
    const uint32_t *bp = reinterpret_cast<const uint32_t *>(fd.B + base) + lam;
    if (live) {
        const FastMod modH(h);
        const uint16_t *Dv = fd.D + (uint64_t)C * h;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t q = 4 * lam + m, jj = q / C, c = q - jj * C;
            const uint64_t dv = (uint64_t)c * w + j0 + jj;
            const uint32_t t = FHD_IN(dv, (uint64_t)C * w, kSiteStripShift) ? modH.mod(pass_ld<kL2>(Dv + dv)) : 0;
            const uint32_t sp2 = kEnc ? t : (t ? h - t : 0);
            if (m < 2) a01 |= (sp2 >> 2) << (16 * m);
            else a23 |= (sp2 >> 2) << (16 * (m - 2));
            bs |= (sp2 & 3) << (2 * m);
        }
        for (uint32_t k0 = p0; k0 < H4; k0 += kU * nq) {
            uint32_t v[kU][4];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t k = k0 + u * nq;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const uint64_t o = (uint64_t)(4 * k + r) * rw;
                    v[u][r] = 0;
                    if (k < H4 && FHD_IN(base + 4 * (o + lam) + 3, fd.N, kSiteStripLoad)) {
                        v[u][r] = pass_ld<kL2>(sp + o);
                        if (!kEnc) v[u][r] ^= pass_ld<kL2>(bp + o);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t k = k0 + u * nq;
                if (k >= H4) break;
                transpose4x4(v[u][0], v[u][1], v[u][2], v[u][3]);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    uint32_t p = k + (((m < 2 ? a01 : a23) >> (16 * (m & 1))) & 0xffffu);
                    p = p >= H4 ? p - H4 : p;
                    const size_t i = (size_t)p * QP + m * NL + lam;
                    if (FHD_IN(i, words, kSiteStripSmem)) S[i] = v[u][m];
                }
            }
        }
    }
    sync();
    if (!live) return;
    uint32_t *op = reinterpret_cast<uint32_t *>(out + base) + lam;
    for (uint32_t t0 = p0; t0 < H4; t0 += kU * nq) {
        uint32_t kb[kU][4];   // B words of the batch's output rows (encrypt), loaded before any store
        if (kEnc) {
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t t = t0 + u * nq;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const uint64_t o = (uint64_t)(4 * t + r) * rw;
                    kb[u][r] = t < H4 && FHD_IN(base + 4 * (o + lam) + 3, fd.N, kSiteStripLoad) ? pass_ld<kL2>(bp + o) : 0;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint32_t t = t0 + u * nq;
            if (t >= H4) break;
            const uint32_t tm = t ? t - 1 : H4 - 1;
            uint32_t v[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const size_t i0 = (size_t)tm * QP + m * NL + lam, i1 = (size_t)t * QP + m * NL + lam;
                const uint32_t sel = 0x7654u - ((bs >> (2 * m)) & 3) * 0x1111u;
                v[m] = FHD_IN(i0, words, kSiteStripSmem) && FHD_IN(i1, words, kSiteStripSmem)
                           ? __byte_perm(S[i0], S[i1], sel)
                           : 0;
            }
            transpose4x4(v[0], v[1], v[2], v[3]);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint64_t o = (uint64_t)(4 * t + r) * rw;
                if (!FHD_IN(base + 4 * (o + lam) + 3, fd.N, kSiteStripStore)) continue;
                if (kEnc) __stcs(op + o, v[r] ^ kb[u][r]);
                else op[o] = v[r];
            }
        }
    }
}

// Column pass.  Encrypt: S[(i + s_v) mod h][q] = G[i][q]; E = S ^ B.
// Decrypt: S[(i - s_v) mod h][q] = (E ^ B)[i][q]; G = S.
// Column pass over strip `strip` of frame fd by the nthr threads (tid = 0..nthr-1) of a group that meets at
// sync(); smem holds the strip (strip_smem_bytes).
template <bool kEnc, bool kL2 = false, class Sync>
__device__ void strip_pass(const FrameDesc &fd, uint32_t strip, uint8_t *smem, uint32_t tid, uint32_t nthr, Sync sync) {
    const uint32_t h = fd.h, w = fd.w, C = fd.C, P = fd.P;
    const uint32_t j0 = strip * P;
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
    if (!FHD_IN(j0, w, kSiteStripSmem)) return;   // a strip past the frame (the same for the whole group)
    {
        // the column-word route: rows of whole row quads, 32-bit aligned rows and pointers, and a strip whose
        // column-word pitch is its row length (no padding: it fits the strip's shared memory)
        const ColWords cw = col_words(QC);
        if ((h & 3) == 0 && (QC & 3) == 0 && rowB % 4 == 0 && base % 4 == 0 && nthr % cw.LT == 0 &&
            (cw.LT != 16 || (QC & 31) == 16) && aligned(src, 4) && aligned(out, 4) && aligned(fd.B, 4)) {
            strip_pass_cw<kEnc, kL2>(fd, j0, QC, cw, smem, tid, nthr, sync);
            return;
        }
    }

    // ---- phase 1: loads of the strip rows, bytes scattered to their rotated rows.  With 4-byte-aligned
    // rows a lane owns one 32-bit word of the strip row (the lanes of a warp hold consecutive words), so
    // in each byte store the lanes hit consecutive banks up to the row term 16 d (mod 32): at most two
    // lanes share a bank.
    const uint32_t vec = strip_vec(rowB, P, C, Pe, src, out, fd.B);
    if (vec >= 4) {
        const uint32_t nw = QC / 4;                    // words per strip row
        const uint32_t RT = nthr / nw;           // rows in parallel
        if (tid < nw * RT) {
            const uint32_t j = tid % nw, tr = tid / nw;
            uint32_t ht[4];   // row offset of each byte: s_v (encrypt) or h - s_v (decrypt)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t q = 4 * j + k, jj = q / C, c = q - jj * C;
                const uint64_t dv = (uint64_t)c * w + j0 + jj;
                const uint32_t t = FHD_IN(dv, (uint64_t)C * w, kSiteStripShift) ? modH.mod(pass_ld<kL2>(Dv + dv)) : 0;
                ht[k] = kEnc ? t : h - t;
            }
            const uint8_t *sp = src + base + 4 * j;
            const uint8_t *bp = fd.B + base + 4 * j;
            for (uint32_t ib = tr; ib < h; ib += kRowsW * RT) {
                uint32_t e[kRowsW];
#pragma unroll
                for (int k = 0; k < kRowsW; ++k) {
                    const uint32_t i = ib + k * RT;
                    if (i < h && FHD_IN(base + 4 * j + (uint64_t)i * rowB + 3, fd.N, kSiteStripLoad)) {
                        e[k] = pass_ld<kL2>(reinterpret_cast<const unsigned int *>(sp + (uint64_t)i * rowB));
                        if (!kEnc) e[k] ^= pass_ld<kL2>(reinterpret_cast<const unsigned int *>(bp + (uint64_t)i * rowB));
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
                            if (FHD_IN((size_t)d * RP + 4 * j + bb, (size_t)h * RP, kSiteStripSmem))
                                S[(size_t)d * RP + 4 * j + bb] = (uint8_t)(e[k] >> (8 * bb));
                        }
                    }
                }
            }
        }
    } else {
        const uint32_t RT = nthr / QC;
        if (tid < QC * RT) {
            const uint32_t q = tid % QC, tr = tid / QC;
            const uint32_t jj = q / C, c = q - jj * C;
            const uint64_t dv = (uint64_t)c * w + j0 + jj;
            const uint32_t t = FHD_IN(dv, (uint64_t)C * w, kSiteStripShift) ? modH.mod(pass_ld<kL2>(Dv + dv)) : 0;
            const uint32_t ht = kEnc ? t : h - t;
            for (uint32_t i = tr; i < h; i += RT) {
                const uint64_t o = (uint64_t)i * rowB + base + q;
                uint8_t e = 0;
                if (FHD_IN(o, fd.N, kSiteStripLoad)) {
                    e = pass_ld<kL2>(src + o);
                    if (!kEnc) e ^= pass_ld<kL2>(fd.B + o);
                }
                uint32_t d = i + ht;
                d = d >= h ? d - h : d;
                if (FHD_IN((size_t)d * RP + q, (size_t)h * RP, kSiteStripSmem)) S[(size_t)d * RP + q] = e;
            }
        }
    }
    sync();

    // ---- phase 2: the strip leaves row by row (XORed with B when encrypting)
    const uint32_t nv = QC / vec;
    const uint32_t RT = nthr / nv;
    if (tid >= nv * RT) return;
    const uint32_t tv = tid % nv, tr = tid / nv;
    if (vec == 16) {
        for (uint32_t ib = tr; ib < h; ib += kRowsV * RT) {
            uint4 g[kRowsV], k4[kRowsV];
#pragma unroll
            for (int k = 0; k < kRowsV; ++k) {
                const uint32_t i = ib + k * RT;
                if (i < h && FHD_IN((size_t)i * RP + 16 * tv + 15, (size_t)h * RP, kSiteStripSmem) &&
                    FHD_IN((uint64_t)i * rowB + base + 16 * tv + 15, fd.N, kSiteStripLoad)) {
                    g[k] = *reinterpret_cast<const uint4 *>(S + (size_t)i * RP + 16 * tv);
                    if (kEnc) k4[k] = pass_ld<kL2>(reinterpret_cast<const uint4 *>(fd.B + (uint64_t)i * rowB + base + 16 * tv));
                }
            }
#pragma unroll
            for (int k = 0; k < kRowsV; ++k) {
                const uint32_t i = ib + k * RT;
                if (i < h && FHD_IN((uint64_t)i * rowB + base + 16 * tv + 15, fd.N, kSiteStripStore)) {
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
            if (!FHD_IN((size_t)i * RP + 4 * tv + 3, (size_t)h * RP, kSiteStripSmem) || !FHD_IN(o + 3, fd.N, kSiteStripStore))
                continue;
            uint32_t g = *reinterpret_cast<const uint32_t *>(S + (size_t)i * RP + 4 * tv);
            if (kEnc) g ^= pass_ld<kL2>(reinterpret_cast<const uint32_t *>(fd.B + o));
            *reinterpret_cast<uint32_t *>(out + o) = g;
        }
    } else {
        for (uint32_t i = tr; i < h; i += RT) {
            const uint64_t o = (uint64_t)i * rowB + base + tv;
            if (!FHD_IN((size_t)i * RP + tv, (size_t)h * RP, kSiteStripSmem) || !FHD_IN(o, fd.N, kSiteStripStore)) continue;
            uint8_t g = S[(size_t)i * RP + tv];
            if (kEnc) g ^= pass_ld<kL2>(fd.B + o);
            out[o] = g;
        }
    }
}

// Plane word of channel c (pixels 4j .. 4j+3) from the three interleaved words 3j .. 3j+2 of an RGB row.
__device__ __forceinline__ uint32_t rgb_plane_word(uint32_t w0, uint32_t w1, uint32_t w2, int c) {
    if (c == 0) return __byte_perm(__byte_perm(w0, w1, 0x0630), w2, 0x5210);
    if (c == 1) return __byte_perm(__byte_perm(w0, w1, 0x0741), w2, 0x6210);
    return __byte_perm(__byte_perm(w0, w1, 0x0052), w2, 0x7410);
}

// Row pass of interleaved RGB rows with w % 16 == 0 and 16-byte aligned rows, staged as channel planes: each
// 48-byte group of a source row (16 pixels, three 16-byte loads) is deinterleaved once, while it is staged,
// into four plane words per channel (shared memory: row r, plane c at r * pitch + c * w).  A thread then
// builds one output 4-pixel group: per channel the two plane words that hold its source bytes (two 32-bit
// shared loads, consecutive across the threads), one funnel shift, and the three channels' words
// interleaved back into the three output words, stored straight to the frame.
template <bool kEnc, bool kL2, class Sync>
__device__ void row_pass_planar(const FrameDesc &fd, uint32_t i0, uint32_t nr, const uint8_t *src, uint8_t *dst,
                                uint8_t *In, uint32_t *sh, uint32_t tid, uint32_t nthr, Sync sync) {
    const uint32_t h = fd.h, w = fd.w, RB = fd.RB, rowB = 3 * w, pitch = rowB, W4 = w >> 2, W16 = w >> 4;
    [[maybe_unused]] const size_t band_bytes = (size_t)RB * pitch;
    const FastMod modW8(8 * w);
    for (uint32_t k = tid; k < nr * W16; k += nthr) {
        const uint32_t r = k / W16, g = k - r * W16;
        if (!FHD_IN((uint64_t)(i0 + r) * rowB + 48 * g + 47, fd.N, kSiteRowLoad) ||
            !FHD_IN((size_t)r * pitch + 2 * w + 16 * g + 15, band_bytes, kSiteRowSmem))
            continue;
        const uint4 *sp = reinterpret_cast<const uint4 *>(src + (uint64_t)r * rowB + 48 * g);
        const uint4 x0 = pass_ld<kL2>(sp), x1 = pass_ld<kL2>(sp + 1), x2 = pass_ld<kL2>(sp + 2);
        const uint32_t wd[12] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w, x2.x, x2.y, x2.z, x2.w};
#pragma unroll
        for (int c = 0; c < 3; ++c)
            *reinterpret_cast<uint4 *>(In + (size_t)r * pitch + (size_t)c * w + 16 * g) =
                make_uint4(rgb_plane_word(wd[0], wd[1], wd[2], c), rgb_plane_word(wd[3], wd[4], wd[5], c),
                           rgb_plane_word(wd[6], wd[7], wd[8], c), rgb_plane_word(wd[9], wd[10], wd[11], c));
    }
    for (uint32_t k = tid; k < nr * 3; k += nthr) {
        const uint32_t r = k / 3, c = k - r * 3;
        const uint64_t di = (uint64_t)c * h + i0 + r;
        if (FHD_IN(k, (uint64_t)RB * 3, kSiteRowSmem))
            sh[k] = FHD_IN(di, 3ull * h, kSiteRowShift) ? modW8.mod(pass_ld<kL2>(fd.D + di)) : 0;
    }
    sync();
    for (uint32_t r = 0; r < nr; ++r) {
        uint32_t du[3], fs[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint32_t sc = sh[r * 3 + c];
            const uint32_t a = sc >> 3, rr = sc & 7;
            // first source pixel of output pixel 0: -a-1 (encrypt) or a (decrypt), mod w
            int s0 = kEnc ? -(int)a - 1 : (int)a;
            if (s0 < 0) s0 += (int)w;
            du[c] = (uint32_t)s0 >> 2;
            const uint32_t o = (uint32_t)s0 & 3;
            fs[c] = kEnc ? 8 * o + 8 - rr : 8 * o + rr;
        }
        const uint32_t *plane = reinterpret_cast<const uint32_t *>(In + (size_t)r * pitch);
        uint32_t *orow = reinterpret_cast<uint32_t *>(dst + (uint64_t)r * rowB);
        for (uint32_t g = tid; g < W4; g += nthr) {
            uint32_t q[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                uint32_t u = g + du[c];
                u = u >= W4 ? u - W4 : u;
                uint32_t u1 = u + 1 == W4 ? 0 : u + 1;
                if (!FHD_IN(u, W4, kSiteRowSmem) || !FHD_IN(u1, W4, kSiteRowSmem)) u = u1 = 0;
                q[c] = __funnelshift_rc(plane[c * W4 + u], plane[c * W4 + u1], fs[c]);
            }
            if (!FHD_IN((uint64_t)(i0 + r) * rowB + 12 * g + 11, fd.N, kSiteRowStore)) continue;
            uint32_t *wp = orow + 3 * g;
            wp[0] = __byte_perm(__byte_perm(q[0], q[1], 0x1040), q[2], 0x3410);
            wp[1] = __byte_perm(__byte_perm(q[1], q[0], 0x2601), q[2], 0x3250);
            wp[2] = __byte_perm(__byte_perm(q[2], q[0], 0x3072), q[1], 0x3710);
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
template <bool kEnc, bool kL2 = false, class Sync>
__device__ void row_pass(const FrameDesc &fd, uint32_t band, uint8_t *smem, uint32_t tid, uint32_t nthr, Sync sync) {
    const uint32_t h = fd.h, w = fd.w, C = fd.C, RB = fd.RB;
    const uint32_t i0 = band * RB;
    const uint32_t nr = min(RB, h - i0);
    const uint32_t rowB = w * C;
    const uint32_t pitch = (rowB + 15) & ~15u;
    const uint8_t *src = (kEnc ? fd.src : fd.G) + (uint64_t)i0 * rowB;
    uint8_t *dst = (kEnc ? fd.G : fd.dst) + (uint64_t)i0 * rowB;
    uint8_t *In = smem;                                          // RB rows
    uint8_t *Out = smem + (size_t)RB * pitch;                    // RB rows
    uint32_t *sh = reinterpret_cast<uint32_t *>(smem + 2 * (size_t)RB * pitch);   // row shifts [r * C + c]
    const FastMod modW8(8 * w);
    [[maybe_unused]] const size_t band_bytes = (size_t)RB * pitch;   // extent of In and of Out
    if (!FHD_IN(i0, h, kSiteRowSmem)) return;   // a band past the frame (the same for the whole group)

    // ---- load the band (rows are contiguous in global memory)
    const bool v16 = rowB % 16 == 0 && aligned(src, 16) && aligned(dst, 16);
    if (C == 3 && (w & 15) == 0 && v16) {
        row_pass_planar<kEnc, kL2>(fd, i0, nr, src, dst, In, sh, tid, nthr, sync);
        return;
    }
    if (v16) {
        const uint32_t nvr = rowB / 16;
        for (uint32_t k = tid; k < nr * nvr; k += nthr) {
            const uint32_t r = k / nvr, v = k - r * nvr;
            if (FHD_IN((size_t)r * pitch + 16 * v + 15, band_bytes, kSiteRowSmem) &&
                FHD_IN((uint64_t)(i0 + r) * rowB + 16 * v + 15, fd.N, kSiteRowLoad))
                *reinterpret_cast<uint4 *>(In + (size_t)r * pitch + 16 * v) =
                    pass_ld<kL2>(reinterpret_cast<const uint4 *>(src + (uint64_t)r * rowB + 16 * v));
        }
    } else {
        for (uint32_t k = tid; k < nr * rowB; k += nthr) {
            const uint32_t r = k / rowB, q = k - r * rowB;
            if (FHD_IN((size_t)r * pitch + q, band_bytes, kSiteRowSmem) &&
                FHD_IN((uint64_t)(i0 + r) * rowB + q, fd.N, kSiteRowLoad))
                In[(size_t)r * pitch + q] = pass_ld<kL2>(src + (uint64_t)r * rowB + q);
        }
    }
    for (uint32_t k = tid; k < nr * C; k += nthr) {
        const uint32_t r = k / C, c = k - r * C;
        const uint64_t di = (uint64_t)c * h + i0 + r;
        if (FHD_IN(k, (uint64_t)RB * C, kSiteRowSmem))
            sh[k] = FHD_IN(di, (uint64_t)C * h, kSiteRowShift) ? modW8.mod(pass_ld<kL2>(fd.D + di)) : 0;
    }
    sync();

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
            for (uint32_t g = tid; g < W4; g += nthr) {
                uint32_t q[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    uint32_t u = g + du[c];
                    u = u >= W4 ? u - W4 : u;
                    uint32_t u1 = u + 1 == W4 ? 0 : u + 1;
                    if (!FHD_IN(u, W4, kSiteRowSmem) || !FHD_IN(u1, W4, kSiteRowSmem)) u = u1 = 0;
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
        sync();
        const uint32_t nvr = rowB / 16;
        for (uint32_t r = 0; r < nr; ++r)
            for (uint32_t v = tid; v < nvr; v += nthr)
                if (FHD_IN((size_t)r * pitch + 16 * v + 15, band_bytes, kSiteRowSmem) &&
                    FHD_IN((uint64_t)(i0 + r) * rowB + 16 * v + 15, fd.N, kSiteRowStore))
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
        for (uint32_t k = tid; k < nq; k += nthr) {
            const uint32_t j = 4 * k;
            const uint32_t nm = min(4u, w - j);
            // first source pixel: j - a - 1 (encrypt) or j + a (decrypt), mod w
            int p0 = kEnc ? (int)j - (int)a - 1 : (int)(j + a);
            if (p0 < 0) p0 += (int)w;
            if (p0 >= (int)w) p0 -= (int)w;
            if (!FHD_IN(p0, w, kSiteRowSmem)) p0 = 0;
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
    sync();

    // ---- store the band
    if (v16) {
        const uint32_t nvr = rowB / 16;
        for (uint32_t k = tid; k < nr * nvr; k += nthr) {
            const uint32_t r = k / nvr, v = k - r * nvr;
            if (FHD_IN((size_t)r * pitch + 16 * v + 15, band_bytes, kSiteRowSmem) &&
                FHD_IN((uint64_t)(i0 + r) * rowB + 16 * v + 15, fd.N, kSiteRowStore))
                *reinterpret_cast<uint4 *>(dst + (uint64_t)r * rowB + 16 * v) =
                    *reinterpret_cast<const uint4 *>(Out + (size_t)r * pitch + 16 * v);
        }
    } else {
        for (uint32_t k = tid; k < nr * rowB; k += nthr) {
            const uint32_t r = k / rowB, q = k - r * rowB;
            if (FHD_IN((size_t)r * pitch + q, band_bytes, kSiteRowSmem) &&
                FHD_IN((uint64_t)(i0 + r) * rowB + q, fd.N, kSiteRowStore))
                dst[(uint64_t)r * rowB + q] = Out[(size_t)r * pitch + q];
        }
    }
}

}  // namespace
}  // namespace fhd
