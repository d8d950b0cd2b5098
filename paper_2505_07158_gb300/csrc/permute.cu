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
#include "permute_dev.cuh"

namespace fhd {
namespace {

// CTA shapes.  Column pass: 512 threads at two CTAs per SM (the default) or 256 at four; row pass: 256
// threads held to six CTAs per SM (40 registers) or 128 at twelve.  The autotuner picks per frame shape
// (fhd_set_cta_threads); on the 30-frame 1080p clip the defaults measured 0.269 / 0.259 ms per encrypt /
// decrypt permutation call, 256-thread column-pass CTAs 0.326 / 0.368.
constexpr int kStripThreads = 512;
constexpr int kRowThreads = 256;
template <int kT>
constexpr int strip_ctas_per_sm() { return kT == 512 ? 2 : 4; }
template <int kT>
constexpr int row_ctas_per_sm() { return kT == 256 ? 6 : 12; }
template <bool kRow>
__device__ __forceinline__ uint32_t find_frame(const Batch &b, uint32_t cta) {
    uint32_t lo = 0, hi = b.count;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if ((kRow ? b.f[mid].rcta0 : b.f[mid].cta0) <= cta) lo = mid; else hi = mid;
    }
    return lo;
}

template <bool kEnc, int kT = kStripThreads>
__global__ void __launch_bounds__(kT, strip_ctas_per_sm<kT>()) strip_kernel(const __grid_constant__ Batch b,
                                                                            uint32_t cta_base) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t cta = cta_base + blockIdx.x;
    const FrameDesc &fd = b.f[find_frame<false>(b, cta)];
    strip_pass<kEnc>(fd, cta - fd.cta0, smem, threadIdx.x, blockDim.x, [] { __syncthreads(); });
}

template <bool kEnc, int kT = kRowThreads>
__global__ void __launch_bounds__(kT, row_ctas_per_sm<kT>()) row_kernel(const __grid_constant__ Batch b,
                                                                        uint32_t cta_base) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t cta = cta_base + blockIdx.x;
    const FrameDesc &fd = b.f[find_frame<true>(b, cta)];
    row_pass<kEnc>(fd, cta - fd.rcta0, smem, threadIdx.x, blockDim.x, [] { __syncthreads(); });
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
        ab[m] = (unit && FHD_IN((uint64_t)c * w + j0 + 8 * g + m, 3ull * w, kSiteGatherShift)
                     ? modH.mod(fd.D[3ull * h + (uint64_t)c * w + j0 + 8 * g + m])
                     : 0) * RP + (8 * g + m) * 3 + c;
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
            const bool ok = FHD_IN(wc * h + i, 3 * h, kSiteGatherShift);
            if (tab) {
                const uint32_t v = ok ? tab[wc * h + i] : 0;
                r.du = v >> 5;
                r.fs = (v & 31) + 1;
            } else {
                r = row_rot(ok ? fd.D[(uint64_t)wc * h + i] : 0, w, modW8);
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
                if (FHD_IN((uint64_t)i * rowB + o + 15, fd.N, kSiteGatherLoad))
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
        if (unit && i < h && FHD_IN(uwi * GS::NC * 16 + uoff + 24 * g + 35, GS::NCH * 16, kSiteGatherSmem)) {
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
                if (FHD_IN(a, hRP, kSiteGatherSmem)) S[a] = (uint8_t)((m < 4 ? q0 : q1) >> (8 * (m & 3)));
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
    if (!FHD_IN(j0, w, kSiteGatherSmem)) return;   // a strip past the frame (the whole CTA)
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
            if (i < h && FHD_IN((size_t)i * RP + 16 * tv + 15, (size_t)h * RP, kSiteGatherSmem) &&
                FHD_IN((uint64_t)i * rowB + base + 15, fd.N, kSiteGatherStore)) {
                v[k] = *reinterpret_cast<const uint4 *>(S + (size_t)i * RP + 16 * tv);
                k4[k] = __ldcs(reinterpret_cast<const uint4 *>(fd.B + (uint64_t)i * rowB + base));
            }
        }
#pragma unroll
        for (int k = 0; k < kRowsV; ++k) {
            const uint32_t i = ib + k * RT;
            if (i < h && FHD_IN((uint64_t)i * rowB + base + 15, fd.N, kSiteGatherStore)) {
                uint4 o = v[k];
                o.x ^= k4[k].x; o.y ^= k4[k].y; o.z ^= k4[k].z; o.w ^= k4[k].w;
                __stcs(reinterpret_cast<uint4 *>(fd.dst + (uint64_t)i * rowB + base), o);
            }
        }
    }
}

}  // namespace

size_t strip_smem_bytes(uint32_t h, uint32_t P, uint32_t C) { return ((size_t)h * P * C + 15) & ~(size_t)15; }

// Two row-sized buffers per row (input and output) and the row shifts.
size_t row_smem_bytes(uint32_t w, uint32_t C, uint32_t RB) {
    const size_t pitch = ((size_t)w * C + 15) & ~(size_t)15;
    return 2 * (size_t)RB * pitch + 4 * (size_t)RB * C;
}

uint32_t permute_strips(uint32_t w, uint32_t P) { return (w + P - 1) / P; }

// Autotuner overrides per frame shape: strip width P of the column pass and rows per CTA RB of the row
// pass (0: the built-in choice).
static uint32_t g_override_key[64][3];
static uint32_t g_override_P[64];
static uint32_t g_override_RB[64];
static uint32_t g_override_ST[64];   // column-pass threads per CTA (0: kStripThreads)
static uint32_t g_override_RT[64];   // row-pass threads per CTA (0: kRowThreads)
static int g_overrides = 0;

static int override_slot(uint32_t h, uint32_t w, uint32_t C) {
    for (int k = 0; k < g_overrides; ++k)
        if (g_override_key[k][0] == h && g_override_key[k][1] == w && g_override_key[k][2] == C) return k;
    if (g_overrides >= 64) return -1;
    g_override_key[g_overrides][0] = h;
    g_override_key[g_overrides][1] = w;
    g_override_key[g_overrides][2] = C;
    g_override_P[g_overrides] = g_override_RB[g_overrides] = 0;
    g_override_ST[g_overrides] = g_override_RT[g_overrides] = 0;
    return g_overrides++;
}

int set_cta_threads_override(uint32_t h, uint32_t w, uint32_t C, uint32_t st, uint32_t rt) {
    const int k = override_slot(h, w, C);
    if (k < 0) return -1;
    g_override_ST[k] = st;
    g_override_RT[k] = rt;
    return 0;
}

void cta_threads(uint32_t h, uint32_t w, uint32_t C, uint32_t *st, uint32_t *rt) {
    *st = kStripThreads;
    *rt = kRowThreads;
    for (int k = 0; k < g_overrides; ++k)
        if (g_override_key[k][0] == h && g_override_key[k][1] == w && g_override_key[k][2] == C) {
            if (g_override_ST[k]) *st = g_override_ST[k];
            if (g_override_RT[k]) *rt = g_override_RT[k];
        }
}

int set_strip_override(uint32_t h, uint32_t w, uint32_t C, uint32_t P) {
    const int k = override_slot(h, w, C);
    if (k < 0) return -1;
    g_override_P[k] = P;
    return 0;
}

int set_row_band_override(uint32_t h, uint32_t w, uint32_t C, uint32_t RB) {
    const int k = override_slot(h, w, C);
    if (k < 0) return -1;
    g_override_RB[k] = RB;
    return 0;
}

// Bands of about kRowSmemTarget bytes of shared memory (2 rows at 1080p), 1..16 rows; an autotuner override
// (if any and if it fits) wins.
uint32_t row_band(uint32_t h, uint32_t w, uint32_t C) {
    for (int k = 0; k < g_overrides; ++k)
        if (g_override_key[k][0] == h && g_override_key[k][1] == w && g_override_key[k][2] == C && g_override_RB[k] &&
            g_override_RB[k] <= 64 && row_smem_bytes(w, C, g_override_RB[k]) <= kSmemLimit)
            return g_override_RB[k];
    const size_t pitch = ((size_t)w * C + 15) & ~(size_t)15;
    size_t rb = kRowSmemTarget / (2 * pitch + 16);
    if (rb < 1) rb = 1;
    if (rb > 16) rb = 16;
    return (uint32_t)rb;
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
    const void *fns[9] = {(const void *)strip_kernel<true>, (const void *)strip_kernel<false>,
                          (const void *)strip_kernel<true, 256>, (const void *)strip_kernel<false, 256>,
                          (const void *)row_kernel<true>, (const void *)row_kernel<false>,
                          (const void *)row_kernel<true, 128>, (const void *)row_kernel<false, 128>,
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
    // CTA shapes of the batch: those of its largest frame's shape
    uint32_t big = 0;
    for (uint32_t k = 1; k < b.count; ++k)
        if (b.f[k].N > b.f[big].N) big = k;
    uint32_t st, rt;
    cta_threads(b.f[big].h, b.f[big].w, b.f[big].C, &st, &rt);
    auto rows = [&](bool enc) {
        if (rt == 128) {
            if (enc) row_kernel<true, 128><<<b.row_ctas, 128, rsm, s>>>(b, 0);
            else row_kernel<false, 128><<<b.row_ctas, 128, rsm, s>>>(b, 0);
        } else {
            if (enc) row_kernel<true><<<b.row_ctas, kRowThreads, rsm, s>>>(b, 0);
            else row_kernel<false><<<b.row_ctas, kRowThreads, rsm, s>>>(b, 0);
        }
        note_launch();
        return cudaGetLastError();
    };
    auto strips = [&](bool enc) {
        if (st == 256) {
            if (enc) strip_kernel<true, 256><<<b.perm_ctas, 256, ssm, s>>>(b, 0);
            else strip_kernel<false, 256><<<b.perm_ctas, 256, ssm, s>>>(b, 0);
        } else {
            if (enc) strip_kernel<true><<<b.perm_ctas, kStripThreads, ssm, s>>>(b, 0);
            else strip_kernel<false><<<b.perm_ctas, kStripThreads, ssm, s>>>(b, 0);
        }
        note_launch();
        return cudaGetLastError();
    };
    if (encrypt) {
        if ((e = rows(true)) != cudaSuccess) return e;
        return strips(true);
    }
    if ((e = strips(false)) != cudaSuccess) return e;
    return rows(false);
}

}  // namespace fhd

FHD_BOUNDS_TAKER(take_bounds_permute)
