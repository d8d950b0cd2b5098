// K3 / K4: the bit-level confusion + XOR of Sec. II-C (Algos 3-7) fused into
// one gather pass per frame, and its exact inverse.
//
// The paper expands every pixel into 8 bits of an [8w x h] matrix (Algo 3),
// rotates each row's bitstring by d_h (Algo 4), rotates each pixel column by
// d_v rows (Algo 5), XORs with B (Algo 6) and packs the bits (Algo 7).  With
// the least-significant-bit-first expansion of Algo 3, a channel row's
// bitstring is its little-endian byte string, so a row rotation by
// s = 8a + r bits is a byte rotation by a plus a funnel shift by r:
//   out[j] = (in[j - a] << r | in[j - a - 1] >> (8 - r)) & 0xff   (mod w).
// No bit matrix is materialised.  For output (i, j, c):
//   E[i,j,c] = B[i,j,c] ^ rowrot(F[i', :, c], s_h(i', c))[j],
//   i' = (i - s_v(j, c)) mod h,
// with s_h(i, c) = D[c*h + i] mod 8w and s_v(j, c) = D[C*h + c*w + j] mod h.
//
// A CTA owns a full-height strip of P pixel columns.  Encrypt: (1) build the
// row-rotated strip G[h][P*C] in shared memory (each source row segment is
// fetched at its own byte offset a(i', c) and funnel-shifted), (2) emit the
// output rows of the strip: each byte gathers G at its own column shift and is
// XORed with B; output rows are written contiguously.  Decrypt mirrors it:
// (1) load E ^ B for the strip plus one column of the next strip (the funnel
// needs a right neighbour), (2) un-rotate columns while reading shared memory
// and write each row segment, funnel-shifted right, at its row's offset.
#include "common.cuh"

namespace fhd {
namespace {

constexpr int kPermThreads = 512;
constexpr size_t kSmemLimit = 232448;   // opt-in dynamic shared memory per CTA on sm_100/sm_103

__device__ __forceinline__ uint32_t find_frame(const Batch &b, uint32_t cta) {
    uint32_t lo = 0, hi = b.count;   // last frame with cta0 <= cta
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (b.f[mid].cta0 <= cta) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kPermThreads) permute_encrypt_kernel(const __grid_constant__ Batch b) {
    extern __shared__ __align__(16) uint8_t smem[];
    const FrameDesc &fd = b.f[find_frame(b, blockIdx.x)];
    const uint32_t h = fd.h, w = fd.w, C = fd.C, P = fd.P;
    const uint32_t strip = blockIdx.x - fd.cta0;
    const uint32_t j0 = strip * P;
    const uint32_t Pe = min(P, w - j0);
    const uint32_t RP = P * C;             // shared row pitch
    const uint32_t QC = Pe * C;            // bytes of a strip row
    uint8_t *G = smem;
    uint32_t *tv = reinterpret_cast<uint32_t *>(smem + (((size_t)h * RP + 15) & ~(size_t)15));
    const uint8_t *F = fd.src;
    const uint16_t *D = fd.D;
    const uint64_t rowB = (uint64_t)w * C;

    for (uint32_t q = threadIdx.x; q < QC; q += blockDim.x) {
        uint32_t jj = q / C, c = q - jj * C;
        tv[q] = D[(uint64_t)C * h + (uint64_t)c * w + j0 + jj] % h;
    }
    // Phase 1: G[i'][jj*C + c] = row-rotated F at pixel column j0 + jj.
    const uint32_t W8 = 8 * w;
    const uint64_t total1 = (uint64_t)h * C * Pe;
    for (uint64_t L = threadIdx.x; L < total1; L += blockDim.x) {
        uint32_t jj = (uint32_t)(L % Pe);
        uint32_t rc = (uint32_t)(L / Pe);
        uint32_t c = rc % C, ip = rc / C;
        uint32_t sh = D[(uint64_t)c * h + ip] % W8;
        uint32_t a = sh >> 3, r = sh & 7;
        uint32_t jc = (j0 + jj + w - a) % w;
        uint32_t jp = (jc + w - 1) % w;
        const uint8_t *row = F + (uint64_t)ip * rowB + c;
        uint32_t cur = row[(uint64_t)jc * C], prev = row[(uint64_t)jp * C];
        G[(size_t)ip * RP + jj * C + c] = (uint8_t)(((cur << r) | (prev >> (8 - r))) & 0xffu);
    }
    __syncthreads();
    // Phase 2: E[i, j0 + jj, c] = B ^ G[(i - s_v) mod h][jj*C + c].
    const uint64_t total2 = (uint64_t)h * QC;
    for (uint64_t L = threadIdx.x; L < total2; L += blockDim.x) {
        uint32_t q = (uint32_t)(L % QC);
        uint32_t i = (uint32_t)(L / QC);
        uint32_t src = i + h - tv[q];
        src = src >= h ? src - h : src;
        uint64_t o = (uint64_t)i * rowB + (uint64_t)j0 * C + q;
        fd.dst[o] = fd.B[o] ^ G[(size_t)src * RP + q];
    }
}

__global__ void __launch_bounds__(kPermThreads) permute_decrypt_kernel(const __grid_constant__ Batch b) {
    extern __shared__ __align__(16) uint8_t smem[];
    const FrameDesc &fd = b.f[find_frame(b, blockIdx.x)];
    const uint32_t h = fd.h, w = fd.w, C = fd.C, P = fd.P;
    const uint32_t strip = blockIdx.x - fd.cta0;
    const uint32_t j0 = strip * P;
    const uint32_t Pe = min(P, w - j0);
    const uint32_t RP = (P + 1) * C;
    const uint32_t QX = (Pe + 1) * C;      // strip row plus the next strip's first column
    uint8_t *A = smem;
    uint32_t *tv = reinterpret_cast<uint32_t *>(smem + (((size_t)h * RP + 15) & ~(size_t)15));
    const uint16_t *D = fd.D;
    const uint64_t rowB = (uint64_t)w * C;

    for (uint32_t q = threadIdx.x; q < QX; q += blockDim.x) {
        uint32_t jj = q / C, c = q - jj * C;
        uint32_t j = (j0 + jj) % w;
        tv[q] = D[(uint64_t)C * h + (uint64_t)c * w + j] % h;
    }
    // Phase 1: A[i][q] = E ^ B at pixel column (j0 + jj) mod w.
    const uint64_t total1 = (uint64_t)h * QX;
    for (uint64_t L = threadIdx.x; L < total1; L += blockDim.x) {
        uint32_t q = (uint32_t)(L % QX);
        uint32_t i = (uint32_t)(L / QX);
        uint32_t jj = q / C, c = q - jj * C;
        uint32_t j = (j0 + jj) % w;
        uint64_t o = (uint64_t)i * rowB + (uint64_t)j * C + c;
        A[(size_t)i * RP + q] = fd.src[o] ^ fd.B[o];
    }
    __syncthreads();
    // Phase 2: un-rotate columns (read row (i' + s_v) mod h), then rotate the
    // row right by s_h: output pixel (j0 + jj - a) mod w.
    const uint32_t W8 = 8 * w;
    const uint64_t total2 = (uint64_t)h * C * Pe;
    for (uint64_t L = threadIdx.x; L < total2; L += blockDim.x) {
        uint32_t jj = (uint32_t)(L % Pe);
        uint32_t rc = (uint32_t)(L / Pe);
        uint32_t c = rc % C, ip = rc / C;
        uint32_t sh = D[(uint64_t)c * h + ip] % W8;
        uint32_t a = sh >> 3, r = sh & 7;
        uint32_t q0 = jj * C + c, q1 = q0 + C;
        uint32_t s0 = ip + tv[q0]; s0 = s0 >= h ? s0 - h : s0;
        uint32_t s1 = ip + tv[q1]; s1 = s1 >= h ? s1 - h : s1;
        uint32_t lo = A[(size_t)s0 * RP + q0], hi = A[(size_t)s1 * RP + q1];
        uint32_t j = (j0 + jj + w - a) % w;
        fd.dst[(uint64_t)ip * rowB + (uint64_t)j * C + c] = (uint8_t)(((lo >> r) | (hi << (8 - r))) & 0xffu);
    }
}

}  // namespace

size_t permute_smem_bytes(uint32_t h, uint32_t P, uint32_t C, bool encrypt) {
    size_t cols = encrypt ? P : P + 1;
    size_t g = ((size_t)h * cols * C + 15) & ~(size_t)15;
    return g + 4 * cols * C;
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
            permute_smem_bytes(h, g_override_P[k], C, false) <= kSmemLimit)
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
