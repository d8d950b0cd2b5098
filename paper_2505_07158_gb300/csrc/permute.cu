// K3 / K4: the bit-level confusion + XOR of Sec. II-C (Algos 3-7) fused into
// one gather pass per frame, and its exact inverse.
//
// The paper expands every pixel into 8 bits of an [8w x h] matrix (Algo 3),
// rotates each row's bitstring by d_h (Algo 4), rotates each pixel column by
// d_v rows (Algo 5), XORs with B (Algo 6) and packs the bits (Algo 7).  With
// the least-significant-bit-first expansion of Algo 3, a channel row's
// bitstring is its little-endian byte string, so a row rotation by
// s = 8a + r bits is a byte rotation by a plus a funnel shift by r.  For four
// consecutive output bytes of one channel row, with A[0..4] the source bytes
// at pixels j - a - 1 .. j - a + 3 (mod w) packed little-endian into a 40-bit
// value V, the four rotated bytes are the low 32 bits of V >> (8 - r): one
// funnel shift.  No bit matrix is materialised.  For output (i, j, c):
//   E[i,j,c] = B[i,j,c] ^ rowrot(F[i', :, c], s_h(i', c))[j],
//   i' = (i - s_v(j, c)) mod h,
// with s_h(i, c) = D[c*h + i] mod 8w and s_v(j, c) = D[C*h + c*w + j] mod h.
//
// A CTA owns a full-height strip of P pixel columns (P chosen so the strip
// fits the 227 KB of shared memory).  Encrypt: (1) every thread owns four
// columns of one channel, walks the rows, gathers + funnel-shifts its source
// bytes and scatters each byte straight into its vertically rotated row of
// the shared strip; (2) the strip is streamed out row by row with 16-byte
// loads of B and 16-byte stores of E.  Decrypt mirrors it: (1) 16-byte loads
// of E and B, XOR, each byte scattered into its un-rotated row of the shared
// strip (plus one column of the next strip, the funnel's right neighbour);
// (2) every thread funnel-shifts four columns of a row right and writes them
// at the row's pixel offset.
#include "common.cuh"

namespace fhd {
namespace {

constexpr int kPermThreads = 384;      // two CTAs per SM when the strip fits twice
constexpr int kRows = 8;              // rows per batch of independent loads
constexpr int kRowsV = 4;             // the same for 16-byte row vectors
constexpr size_t kSmemLimit = 232448;   // opt-in dynamic shared memory per CTA on sm_100/sm_103

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

__device__ __forceinline__ uint32_t find_frame(const Batch &b, uint32_t cta) {
    uint32_t lo = 0, hi = b.count;   // last frame with cta0 <= cta
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (b.f[mid].cta0 <= cta) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool aligned(const void *p, uintptr_t a) {
    return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0;
}

// Vector width (1, 4 or 16 bytes) usable for contiguous strip rows.
__device__ __forceinline__ uint32_t strip_vec(uint64_t rowB, uint32_t P, uint32_t C, uint32_t Pe,
                                              const void *p0, const void *p1) {
    if (rowB % 16 == 0 && (P * C) % 16 == 0 && (Pe * C) % 16 == 0 && aligned(p0, 16) && aligned(p1, 16)) return 16;
    if (rowB % 4 == 0 && (P * C) % 4 == 0 && (Pe * C) % 4 == 0 && aligned(p0, 4) && aligned(p1, 4)) return 4;
    return 1;
}

__global__ void __launch_bounds__(kPermThreads, 2) permute_encrypt_kernel(const __grid_constant__ Batch b) {
    extern __shared__ __align__(16) uint8_t smem[];
    const FrameDesc &fd = b.f[find_frame(b, blockIdx.x)];
    const uint32_t h = fd.h, w = fd.w, C = fd.C, P = fd.P;
    const uint32_t j0 = (blockIdx.x - fd.cta0) * P;
    const uint32_t Pe = min(P, w - j0);
    const uint32_t RP = P * C;             // shared row pitch
    const uint64_t rowB = (uint64_t)w * C;
    uint8_t *G = smem;                     // G[(i' + s_v) mod h][jj*C + c] = rowrot(F)[i'][j0 + jj][c]
    const uint16_t *D = fd.D;
    const FastMod modW8(8 * w), modH(h);
    uint16_t *Ds = reinterpret_cast<uint16_t *>(smem + (((size_t)h * RP + 15) & ~(size_t)15));
    for (uint32_t k = threadIdx.x; k < C * h; k += blockDim.x) Ds[k] = D[k];   // row shifts d_h
    __syncthreads();

    // ---- phase 1: gather, funnel, scatter into the vertically rotated strip.
    // Rows go in batches of kRows with every global load of a batch issued
    // before its shared-memory stores, so a thread keeps several loads in flight.
    const uint32_t nq = (Pe + 3) >> 2;     // quads per channel
    const uint32_t U = nq * C;             // column units (<= 128)
    const uint32_t RT = blockDim.x / U;    // row lanes
    if (threadIdx.x < U * RT) {
        const uint32_t u = threadIdx.x % U, r0 = threadIdx.x / U;
        const uint32_t c = u % C, jq = 4 * (u / C);
        const uint32_t nm = min(4u, Pe - jq);
        uint32_t tv[4];
#pragma unroll
        for (int m = 0; m < 4; ++m)
            tv[m] = (uint32_t)m < nm ? modH.mod(D[(uint64_t)C * h + (uint64_t)c * w + j0 + jq + m]) : 0;
        const uint8_t *Fc = fd.src + c;
        uint8_t *Gc = G + jq * C + c;
        const uint16_t *Dh = Ds + c * h;
        for (uint32_t ipb = r0; ipb < h; ipb += kRows * RT) {
            uint32_t sh[kRows];
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const uint32_t ip = ipb + k * RT;
                sh[k] = ip < h ? modW8.mod(Dh[ip]) : 0;
            }
            uint32_t X[kRows], A4[kRows];
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const uint32_t ip = ipb + k * RT;
                X[k] = 0; A4[k] = 0;
                if (ip < h) {
                    int s = (int)(j0 + jq) - (int)(sh[k] >> 3);   // pixel of A[1]
                    if (s < 0) s += (int)w;
                    const uint8_t *row = Fc + (uint64_t)ip * rowB;
                    uint32_t A0, A1, A2, A3, A4v;
                    if (s >= 1 && (uint32_t)s + 3 < w) {
                        const uint8_t *p = row + (uint64_t)(s - 1) * C;
                        A0 = p[0]; A1 = p[C]; A2 = p[2 * C]; A3 = p[3 * C]; A4v = p[4 * C];
                    } else {
                        uint32_t pm = s == 0 ? w - 1 : (uint32_t)s - 1;
                        uint32_t k1 = (uint32_t)s, k2 = k1 + 1 >= w ? k1 + 1 - w : k1 + 1;
                        uint32_t k3 = k2 + 1 >= w ? k2 + 1 - w : k2 + 1, k4 = k3 + 1 >= w ? k3 + 1 - w : k3 + 1;
                        A0 = row[(uint64_t)pm * C]; A1 = row[(uint64_t)k1 * C];
                        A2 = nm > 1 ? row[(uint64_t)k2 * C] : 0;
                        A3 = nm > 2 ? row[(uint64_t)k3 * C] : 0;
                        A4v = nm > 3 ? row[(uint64_t)k4 * C] : 0;
                    }
                    X[k] = A0 | (A1 << 8) | (A2 << 16) | (A3 << 24);
                    A4[k] = A4v;
                }
            }
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const uint32_t ip = ipb + k * RT;
                if (ip < h) {
                    const uint32_t out = __funnelshift_r(X[k], A4[k], 8 - (sh[k] & 7));
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        uint32_t d = ip + tv[m];
                        d = d >= h ? d - h : d;
                        if ((uint32_t)m < nm) Gc[(size_t)d * RP + m * C] = (uint8_t)(out >> (8 * m));
                    }
                }
            }
        }
    }
    __syncthreads();

    // ---- phase 2: E = B ^ strip, row by row, contiguous
    const uint32_t QC = Pe * C;
    const uint64_t base = (uint64_t)j0 * C;
    const uint32_t vec = strip_vec(rowB, P, C, Pe, fd.dst, fd.B);
    const uint32_t nv = QC / vec;
    const uint32_t RT2 = blockDim.x / nv;
    if (threadIdx.x >= nv * RT2) return;
    const uint32_t tv = threadIdx.x % nv, tr = threadIdx.x / nv;
    if (vec == 16) {
        for (uint32_t ib = tr; ib < h; ib += kRows * RT2) {
            uint4 g[kRows], k4[kRows];
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const uint32_t i = ib + k * RT2;
                if (i < h) {
                    k4[k] = __ldcs(reinterpret_cast<const uint4 *>(fd.B + (uint64_t)i * rowB + base + 16 * tv));
                    g[k] = *reinterpret_cast<const uint4 *>(G + (size_t)i * RP + 16 * tv);
                }
            }
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const uint32_t i = ib + k * RT2;
                if (i < h) {
                    uint4 v = g[k];
                    v.x ^= k4[k].x; v.y ^= k4[k].y; v.z ^= k4[k].z; v.w ^= k4[k].w;
                    __stcs(reinterpret_cast<uint4 *>(fd.dst + (uint64_t)i * rowB + base + 16 * tv), v);
                }
            }
        }
    } else if (vec == 4) {
        for (uint32_t i = tr; i < h; i += RT2) {
            const uint64_t o = (uint64_t)i * rowB + base + 4 * tv;
            uint32_t g = *reinterpret_cast<const uint32_t *>(G + (size_t)i * RP + 4 * tv);
            *reinterpret_cast<uint32_t *>(fd.dst + o) = g ^ *reinterpret_cast<const uint32_t *>(fd.B + o);
        }
    } else {
        for (uint32_t i = tr; i < h; i += RT2) {
            const uint64_t o = (uint64_t)i * rowB + base + tv;
            fd.dst[o] = G[(size_t)i * RP + tv] ^ fd.B[o];
        }
    }
}

__global__ void __launch_bounds__(kPermThreads, 2) permute_decrypt_kernel(const __grid_constant__ Batch b) {
    extern __shared__ __align__(16) uint8_t smem[];
    const FrameDesc &fd = b.f[find_frame(b, blockIdx.x)];
    const uint32_t h = fd.h, w = fd.w, C = fd.C, P = fd.P;
    const uint32_t j0 = (blockIdx.x - fd.cta0) * P;
    const uint32_t Pe = min(P, w - j0);
    const uint32_t RP = (P + 1) * C;       // strip plus the next strip's first column
    const uint64_t rowB = (uint64_t)w * C;
    uint8_t *A = smem;                     // A[i'][q] = (E ^ B)[(i' + s_v(q)) mod h][q]
    const uint16_t *D = fd.D;
    const FastMod modW8(8 * w), modH(h);
    uint16_t *Ds = reinterpret_cast<uint16_t *>(smem + (((size_t)h * RP + 15) & ~(size_t)15));
    for (uint32_t k = threadIdx.x; k < C * h; k += blockDim.x) Ds[k] = D[k];   // row shifts d_h
    const uint32_t QC = Pe * C;
    const uint64_t base = (uint64_t)j0 * C;
    const uint16_t *Dv = D + (uint64_t)C * h;

    // ---- phase 1: E ^ B, each byte scattered to its un-rotated row
    const uint32_t vec = strip_vec(rowB, P, C, Pe, fd.src, fd.B);
    const uint32_t nv = QC / vec;
    const uint32_t RT = blockDim.x / nv;
    if (threadIdx.x < nv * RT) {
        const uint32_t tv = threadIdx.x % nv, tr = threadIdx.x / nv;
        if (vec == 16) {
            uint32_t ht[16];   // h - s_v of the thread's 16 columns
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const uint32_t q = 16 * tv + k, jj = q / C, c = q - jj * C;
                ht[k] = h - modH.mod(Dv[(uint64_t)c * w + j0 + jj]);
            }
            for (uint32_t ib = tr; ib < h; ib += kRowsV * RT) {
                uint4 e[kRowsV];
#pragma unroll
                for (int k = 0; k < kRowsV; ++k) {
                    const uint32_t i = ib + k * RT;
                    if (i < h) {
                        const uint64_t o = (uint64_t)i * rowB + base + 16 * tv;
                        e[k] = __ldcs(reinterpret_cast<const uint4 *>(fd.src + o));
                        const uint4 kb = __ldcs(reinterpret_cast<const uint4 *>(fd.B + o));
                        e[k].x ^= kb.x; e[k].y ^= kb.y; e[k].z ^= kb.z; e[k].w ^= kb.w;
                    }
                }
#pragma unroll
                for (int k = 0; k < kRowsV; ++k) {
                    const uint32_t i = ib + k * RT;
                    if (i < h) {
                        const uint32_t wd[4] = {e[k].x, e[k].y, e[k].z, e[k].w};
#pragma unroll
                        for (int b = 0; b < 16; ++b) {
                            uint32_t d = i + ht[b];
                            d = d >= h ? d - h : d;
                            A[(size_t)d * RP + 16 * tv + b] = (uint8_t)(wd[b >> 2] >> (8 * (b & 3)));
                        }
                    }
                }
            }
        } else {
            const uint32_t q0 = vec * tv;
            uint32_t d[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t q = q0 + k, jj = q / C, c = q - jj * C;
                const uint32_t t = (uint32_t)k < vec ? modH.mod(Dv[(uint64_t)c * w + j0 + jj]) : 0;
                const uint32_t x = tr + h - t;
                d[k] = x >= h ? x - h : x;
            }
            for (uint32_t i = tr; i < h; i += RT) {
                const uint64_t o = (uint64_t)i * rowB + base + q0;
                uint32_t e;
                if (vec == 4) e = *reinterpret_cast<const uint32_t *>(fd.src + o) ^ *reinterpret_cast<const uint32_t *>(fd.B + o);
                else e = (uint32_t)(fd.src[o] ^ fd.B[o]);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if ((uint32_t)k < vec) A[(size_t)d[k] * RP + q0 + k] = (uint8_t)(e >> (8 * k));
                    const uint32_t x = d[k] + RT;
                    d[k] = x >= h ? x - h : x;
                }
            }
        }
    }
    // the next strip's first column (wrapping to column 0 after the last strip)
    {
        const uint32_t jx = (j0 + Pe) % w;
        for (uint32_t L = threadIdx.x; L < h * C; L += blockDim.x) {
            const uint32_t i = L / C, c = L - i * C;
            const uint64_t o = (uint64_t)i * rowB + (uint64_t)jx * C + c;
            const uint32_t t = modH.mod(Dv[(uint64_t)c * w + jx]);
            const uint32_t x = i + h - t;
            A[(size_t)(x >= h ? x - h : x) * RP + QC + c] = fd.src[o] ^ fd.B[o];
        }
    }
    __syncthreads();

    // ---- phase 2: rotate each row right by s_h, write at the row's offset
    const uint32_t nq = (Pe + 3) >> 2;
    const uint32_t U = nq * C;
    const uint32_t RT2 = blockDim.x / U;
    if (threadIdx.x >= U * RT2) return;
    const uint32_t u = threadIdx.x % U, r0 = threadIdx.x / U;
    const uint32_t c = u % C, jq = 4 * (u / C);
    const uint32_t nm = min(4u, Pe - jq);
    const uint16_t *Dh = Ds + c * h;
    uint8_t *Pc = fd.dst + c;
    // A columns jq .. jq + nm (the last one may be the extra column)
    const uint32_t q0 = jq * C + c;
    const uint32_t cl1 = min(jq + 1, Pe) * C + c, cl2 = min(jq + 2, Pe) * C + c;
    const uint32_t cl3 = min(jq + 3, Pe) * C + c, cl4 = min(jq + 4, Pe) * C + c;
    for (uint32_t ipb = r0; ipb < h; ipb += kRows * RT2) {
        uint32_t sh[kRows];
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
            const uint32_t ip = ipb + k * RT2;
            sh[k] = ip < h ? modW8.mod(Dh[ip]) : 0;
        }
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
            const uint32_t ip = ipb + k * RT2;
            if (ip >= h) continue;
            const uint8_t *arow = A + (size_t)ip * RP;
            const uint32_t X = arow[q0] | ((uint32_t)arow[cl1] << 8) | ((uint32_t)arow[cl2] << 16) |
                               ((uint32_t)arow[cl3] << 24);
            const uint32_t out = __funnelshift_r(X, arow[cl4], sh[k] & 7);
            int s = (int)(j0 + jq) - (int)(sh[k] >> 3);
            if (s < 0) s += (int)w;
            uint8_t *row = Pc + (uint64_t)ip * rowB;
            if ((uint32_t)s + nm <= w) {
                uint8_t *p = row + (uint64_t)s * C;
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if ((uint32_t)m < nm) p[(uint32_t)m * C] = (uint8_t)(out >> (8 * m));
            } else {
                uint32_t j = (uint32_t)s;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if ((uint32_t)m < nm) row[(uint64_t)j * C] = (uint8_t)(out >> (8 * m));
                    j = j + 1 >= w ? 0 : j + 1;
                }
            }
        }
    }
}

}  // namespace

size_t permute_smem_bytes(uint32_t h, uint32_t P, uint32_t C, bool encrypt) {
    size_t cols = encrypt ? P : P + 1;
    return (((size_t)h * cols * C + 15) & ~(size_t)15) + (((size_t)2 * C * h + 15) & ~(size_t)15);
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
// whose decrypt working set fits the opt-in shared memory; an autotuner
// override (if any and if it fits) wins.
uint32_t strip_width(uint32_t h, uint32_t w, uint32_t C) {
    for (int k = 0; k < g_overrides; ++k)
        if (g_override_key[k][0] == h && g_override_key[k][1] == w && g_override_key[k][2] == C && g_override_P[k] &&
            g_override_P[k] <= 128 && permute_smem_bytes(h, g_override_P[k], C, false) <= kSmemLimit)
            return g_override_P[k];
    uint32_t P = 128;
    while (P > 1 && (P / 2 >= w || permute_smem_bytes(h, P, C, false) > kSmemLimit)) P /= 2;
    return permute_smem_bytes(h, P, C, false) <= kSmemLimit ? P : 0;
}

cudaError_t permute_prepare() {
    cudaError_t e = cudaFuncSetAttribute(permute_encrypt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemLimit);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(permute_decrypt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmemLimit);
}

cudaError_t launch_permute(const Batch &b, bool encrypt, cudaStream_t s) {
    if (!b.count || !b.perm_ctas) return cudaSuccess;
    size_t smem = 0;
    for (uint32_t k = 0; k < b.count; ++k) {
        size_t need = permute_smem_bytes(b.f[k].h, b.f[k].P, b.f[k].C, encrypt);
        if (need > smem) smem = need;
    }
    if (encrypt)
        permute_encrypt_kernel<<<b.perm_ctas, kPermThreads, smem, s>>>(b);
    else
        permute_decrypt_kernel<<<b.perm_ctas, kPermThreads, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace fhd
