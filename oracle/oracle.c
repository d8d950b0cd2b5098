/*
 * Plain single-threaded CPU oracle of the diffusion-free bit-level video
 * cipher of arXiv 2505.07158 ("Real-Time Bit-Level Encryption of Full
 * High-Definition Video Without Diffusion").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the cipher computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg load it.  It shares no code,
 * header, table or constant generator with the CUDA library: the SHA-256
 * round constants below are *derived* here from their FIPS 180-4 definition
 * (integer cube and square roots of the first primes), while the CUDA side
 * carries its own table.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fno-fast-math -fPIC -shared.
 * -ffp-contract=off is required: the chaotic iteration must round every
 * multiply and add separately (no fused multiply-add), also on aarch64.
 *
 * Every function cites the passage of the paper it follows.  Where the paper
 * is silent or garbled, the reading taken is stated at the function.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* SHA-256 (FIPS 180-4), used by Sec. II-A to digest each sub-frame.        */
/* ------------------------------------------------------------------------ */

static uint32_t sha_k[64];
static uint32_t sha_h0[8];
static int sha_ready = 0;

/* floor(cbrt(x)) for x < 2^105, by bisection on integers. */
static uint64_t icbrt128(unsigned __int128 x) {
    uint64_t lo = 0, hi = (uint64_t)1 << 36;
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        unsigned __int128 c = (unsigned __int128)mid * mid * mid;
        if (c <= x) lo = mid; else hi = mid;
    }
    return lo;
}

/* floor(sqrt(x)) for x < 2^70, by bisection on integers. */
static uint64_t isqrt128(unsigned __int128 x) {
    uint64_t lo = 0, hi = (uint64_t)1 << 36;
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        unsigned __int128 c = (unsigned __int128)mid * mid;
        if (c <= x) lo = mid; else hi = mid;
    }
    return lo;
}

/* FIPS 180-4 Sec. 4.2.2 / 5.3.3: K_t = first 32 bits of the fractional part
 * of the cube root of the t-th prime; H0_i = first 32 bits of the fractional
 * part of the square root of the i-th prime.  floor(r * 2^32) mod 2^32 with
 * r = p^(1/3) equals floor(cbrt(p * 2^96)) mod 2^32 exactly. */
static void sha_init_constants(void) {
    uint32_t primes[64];
    int cnt = 0;
    for (uint32_t c = 2; cnt < 64; ++c) {
        int is_p = 1;
        for (uint32_t d = 2; d * d <= c; ++d)
            if (c % d == 0) { is_p = 0; break; }
        if (is_p) primes[cnt++] = c;
    }
    for (int t = 0; t < 64; ++t)
        sha_k[t] = (uint32_t)icbrt128((unsigned __int128)primes[t] << 96);
    for (int i = 0; i < 8; ++i)
        sha_h0[i] = (uint32_t)isqrt128((unsigned __int128)primes[i] << 64);
    sha_ready = 1;
}

static uint32_t rotr32(uint32_t x, int n) { return (x >> n) | (x << (32 - n)); }

/* FIPS 180-4 Sec. 6.2.2: one compression of a 64-byte block. */
static void sha_compress(uint32_t H[8], const uint8_t blk[64]) {
    uint32_t W[64];
    for (int t = 0; t < 16; ++t)
        W[t] = ((uint32_t)blk[4 * t] << 24) | ((uint32_t)blk[4 * t + 1] << 16) |
               ((uint32_t)blk[4 * t + 2] << 8) | (uint32_t)blk[4 * t + 3];
    for (int t = 16; t < 64; ++t) {
        uint32_t s0 = rotr32(W[t - 15], 7) ^ rotr32(W[t - 15], 18) ^ (W[t - 15] >> 3);
        uint32_t s1 = rotr32(W[t - 2], 17) ^ rotr32(W[t - 2], 19) ^ (W[t - 2] >> 10);
        W[t] = s1 + W[t - 7] + s0 + W[t - 16];
    }
    uint32_t a = H[0], b = H[1], c = H[2], d = H[3];
    uint32_t e = H[4], f = H[5], g = H[6], h = H[7];
    for (int t = 0; t < 64; ++t) {
        uint32_t S1 = rotr32(e, 6) ^ rotr32(e, 11) ^ rotr32(e, 25);
        uint32_t ch = (e & f) ^ (~e & g);
        uint32_t T1 = h + S1 + ch + sha_k[t] + W[t];
        uint32_t S0 = rotr32(a, 2) ^ rotr32(a, 13) ^ rotr32(a, 22);
        uint32_t maj = (a & b) ^ (a & c) ^ (b & c);
        uint32_t T2 = S0 + maj;
        h = g; g = f; f = e; e = d + T1;
        d = c; c = b; b = a; a = T1 + T2;
    }
    H[0] += a; H[1] += b; H[2] += c; H[3] += d;
    H[4] += e; H[5] += f; H[6] += g; H[7] += h;
}

/* FIPS 180-4 Sec. 5.1.1 padding + Sec. 6.2 hash computation. */
void oracle_sha256(const uint8_t *msg, uint64_t len, uint8_t out[32]) {
    if (!sha_ready) sha_init_constants();
    uint32_t H[8];
    memcpy(H, sha_h0, sizeof H);
    uint64_t full = len / 64;
    for (uint64_t b = 0; b < full; ++b) sha_compress(H, msg + 64 * b);
    uint8_t tail[128];
    memset(tail, 0, sizeof tail);
    uint64_t rem = len - 64 * full;
    if (rem) memcpy(tail, msg + 64 * full, rem);
    tail[rem] = 0x80;
    uint64_t tail_len = (rem + 1 + 8 <= 64) ? 64 : 128;
    uint64_t bits = len * 8;
    for (int i = 0; i < 8; ++i) tail[tail_len - 1 - i] = (uint8_t)(bits >> (8 * i));
    sha_compress(H, tail);
    if (tail_len == 128) sha_compress(H, tail + 64);
    for (int i = 0; i < 8; ++i) {
        out[4 * i] = (uint8_t)(H[i] >> 24);
        out[4 * i + 1] = (uint8_t)(H[i] >> 16);
        out[4 * i + 2] = (uint8_t)(H[i] >> 8);
        out[4 * i + 3] = (uint8_t)H[i];
    }
}

/* Sec. II-A, Algorithm 1 (partition, hash, fold): the frame's N bytes are
 * split into n sub-frames f_i; H = h_1 xor ... xor h_n with h_i = SHA-256(f_i).
 * Reading (partition not given by the paper): sub-frame i is the contiguous
 * byte range [floor(i*N/n), floor((i+1)*N/n)) of the raw H x W x C buffer. */
void oracle_frame_digest(const uint8_t *frame, uint64_t N, uint32_t n, uint8_t H[32]) {
    memset(H, 0, 32);
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t lo = (uint64_t)(((unsigned __int128)N * i) / n);
        uint64_t hi = (uint64_t)(((unsigned __int128)N * (i + 1)) / n);
        uint8_t hi_dig[32];
        oracle_sha256(frame + lo, hi - lo, hi_dig);
        for (int b = 0; b < 32; ++b) H[b] ^= hi_dig[b];
    }
}

/* Tree digest: an option of this implementation, not of the paper.  With the
 * XOR fold above, identical sub-frames cancel (a flat frame split into an even
 * number of equal sub-frames has H = 0) and the order of the sub-frames does
 * not matter.  This mode keeps the same partition and sub-frame digests and
 * hashes their concatenation instead: H = SHA-256(h_1 || h_2 || ... || h_n),
 * 32 n bytes in sub-frame order.  Sender and receiver must use the same mode. */
void oracle_frame_digest_tree(const uint8_t *frame, uint64_t N, uint32_t n, uint8_t H[32]) {
    uint8_t *cat = (uint8_t *)malloc(32ull * n);
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t lo = (uint64_t)(((unsigned __int128)N * i) / n);
        uint64_t hi = (uint64_t)(((unsigned __int128)N * (i + 1)) / n);
        oracle_sha256(frame + lo, hi - lo, cat + 32ull * i);
    }
    oracle_sha256(cat, 32ull * n, H);
    free(cat);
}

/* ------------------------------------------------------------------------ */
/* Key and initial-condition reconstruction (Sec. II-A, Fig. 1a).           */
/* ------------------------------------------------------------------------ */

static uint64_t le64(const uint8_t *p) {
    uint64_t v = 0;
    for (int i = 7; i >= 0; --i) v = (v << 8) | p[i];
    return v;
}

/* The paper's key is the five doubles x0, y0, z0, w0, gamma (Sec. IV-A).
 * Reading for a 256-bit key: k_m = little-endian uint64 of key bytes
 * [8m, 8m+8); v_m = (k_m >> 11) * 2^-53 * u_m for m = x, y, z, w, and
 * gamma = -1.52 + 1.46 * ((k0^k1^k2^k3) >> 11) * 2^-53, inside the
 * hyperchaotic range -1.52 <= gamma <= -0.06 of Eq. (1). */
void oracle_key_to_ic(const uint8_t key[32], const uint32_t u[4], double ic[5]) {
    uint64_t k[4];
    for (int m = 0; m < 4; ++m) k[m] = le64(key + 8 * m);
    for (int m = 0; m < 4; ++m) {
        double unit = (double)(k[m] >> 11) * 0x1p-53;
        ic[m] = unit * (double)u[m];
    }
    double g = (double)((k[0] ^ k[1] ^ k[2] ^ k[3]) >> 11) * 0x1p-53;
    ic[4] = -1.52 + 1.46 * g;
}

/* Sec. II-A, Fig. 1a: reconstruct one initial condition v from 8 bytes of H.
 * (1) integer: the two least significant bytes of v's integer part XOR two
 *     bytes of H, reduced mod the predefined upper bound u;
 * (2) fraction: the six least significant bytes of v's fractional part XOR
 *     six bytes of H;
 * (3) combine the two.
 * Readings: v is taken by magnitude; "the six least significant bytes of the
 * fractional part" are the 48-bit fixed-point fraction floor(frac * 2^48);
 * H bytes are consumed little-endian (hb[0..1] integer, hb[2..7] fraction);
 * a non-finite v or |v| >= 2^52 contributes integer 0 and fraction 0. */
double oracle_reconstruct(double v, const uint8_t hb[8], uint32_t u) {
    double a = fabs(v);
    uint64_t I = 0, F48 = 0;
    if (a < 0x1p52) {           /* false for NaN too */
        I = (uint64_t)a;         /* truncation toward zero */
        double F = a - (double)I; /* exact: the fractional part of a double */
        F48 = (uint64_t)(F * 0x1p48);
    }
    uint64_t hi16 = (uint64_t)hb[0] | ((uint64_t)hb[1] << 8);
    uint64_t h48 = 0;
    for (int i = 5; i >= 0; --i) h48 = (h48 << 8) | hb[2 + i];
    uint64_t ip = ((I & 0xFFFFu) ^ hi16) % u;
    double fp = (double)(F48 ^ h48) * 0x1p-48;
    return (double)ip + fp;
}

/* ------------------------------------------------------------------------ */
/* Lorenz hyperchaotic system, Eq. (1), integrated by classical RK4.        */
/* ------------------------------------------------------------------------ */

/* Eq. (1) with sigma = 10, rho = 28, beta = 8/3 (Sec. II-A). */
static void lhcs_f(const double s[4], double gamma, double out[4]) {
    const double sigma = 10.0, rho = 28.0, beta = 8.0 / 3.0;
    double x = s[0], y = s[1], z = s[2], w = s[3];
    out[0] = sigma * (y - x) + w;
    out[1] = (rho * x - y) - x * z;
    out[2] = x * y - beta * z;
    out[3] = gamma * w - y * z;
}

/* Reading (the paper names no integrator or step): classical fourth-order
 * Runge-Kutta with step h, every operation rounded to nearest in binary64,
 * no contraction, in this order:
 *   k1 = f(s); k2 = f(s + (h/2) k1); k3 = f(s + (h/2) k2); k4 = f(s + h k3);
 *   s' = s + (h/6) * (((k1 + 2 k2) + 2 k3) + k4),
 * with h/2 and h/6 each rounded once. */
void oracle_rk4_step(double s[4], double gamma, double h) {
    double hh = h / 2.0, h6 = h / 6.0;
    double k1[4], k2[4], k3[4], k4[4], t[4];
    lhcs_f(s, gamma, k1);
    for (int v = 0; v < 4; ++v) t[v] = s[v] + hh * k1[v];
    lhcs_f(t, gamma, k2);
    for (int v = 0; v < 4; ++v) t[v] = s[v] + hh * k2[v];
    lhcs_f(t, gamma, k3);
    for (int v = 0; v < 4; ++v) t[v] = s[v] + h * k3[v];
    lhcs_f(t, gamma, k4);
    for (int v = 0; v < 4; ++v) {
        double acc = ((k1[v] + 2.0 * k2[v]) + 2.0 * k3[v]) + k4[v];
        s[v] = s[v] + h6 * acc;
    }
}

/* Sec. II-A and Algorithm 1 (reconstruct, initialise LHCS_m, iterate):
 * v = the stream's chaining state (the user's x0..w0 for the first frame,
 * x_2n..w_2n of the previous frame's LHCS_m run afterwards).  Each of x, y,
 * z, w is reconstructed with 8 bytes of H (x: H[0..7], y: H[8..15], ...),
 * LHCS_m is iterated 2n times, IR[t] = state after step t+1 (t = 0..2n-1),
 * and the new chaining state is the last iterate. */
void oracle_master(const double v[4], const uint8_t H[32], const uint32_t u[4],
                   double gamma, double h, uint32_t n, double *IR, double new_state[4]) {
    double s[4];
    for (int m = 0; m < 4; ++m) s[m] = oracle_reconstruct(v[m], H + 8 * m, u[m]);
    for (uint32_t t = 0; t < 2 * n; ++t) {
        oracle_rk4_step(s, gamma, h);
        for (int m = 0; m < 4; ++m) IR[4 * t + m] = s[m];
    }
    for (int m = 0; m < 4; ++m) new_state[m] = s[m];
}

/* Sec. II-B and Algorithm 2 (data generation by worker i, 0-based here).
 * Readings: LHCS_w^{i,1} starts from IR[2i], LHCS_w^{i,2} from IR[2i+1]; a
 * worker iterates both, and each iterate (the state after a step) yields, for
 * x, y, z, w in turn, the six low bytes of the 52-bit mantissa, least
 * significant first.  The worker's byte stream S_i is the byte-wise XOR of
 * the two systems' bytes (per-element XOR of 16-bit distances equals XOR of
 * their bytes).  Worker i owns D[floor(i*L_D/n), floor((i+1)*L_D/n)) and
 * B[floor(i*N/n), floor((i+1)*N/n)) with L_D = C*(h+w), N = h*w*C; it fills
 * its D slice first, one 16-bit distance from every two bytes (little-endian),
 * then its B slice, one byte per byte.  D layout: D[c*h + i] is the
 * horizontal distance of row i, channel c; D[C*h + c*w + j] the vertical
 * distance of pixel column j, channel c. */
void oracle_keystream(const double *IR, uint32_t n, double gamma, double hstep,
                      uint32_t hgt, uint32_t wid, uint32_t C, uint16_t *D, uint8_t *B) {
    uint64_t LD = (uint64_t)C * (hgt + wid);
    uint64_t LB = (uint64_t)hgt * wid * C;
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t d0 = (uint64_t)(((unsigned __int128)LD * i) / n);
        uint64_t d1 = (uint64_t)(((unsigned __int128)LD * (i + 1)) / n);
        uint64_t b0 = (uint64_t)(((unsigned __int128)LB * i) / n);
        uint64_t b1 = (uint64_t)(((unsigned __int128)LB * (i + 1)) / n);
        uint64_t need = 2 * (d1 - d0) + (b1 - b0);
        double s1[4], s2[4];
        for (int m = 0; m < 4; ++m) { s1[m] = IR[4 * (2 * i) + m]; s2[m] = IR[4 * (2 * i + 1) + m]; }
        uint8_t *S = (uint8_t *)malloc(need + 24);
        uint64_t pos = 0;
        while (pos < need) {
            oracle_rk4_step(s1, gamma, hstep);
            oracle_rk4_step(s2, gamma, hstep);
            for (int m = 0; m < 4; ++m) {
                uint64_t u1, u2;
                memcpy(&u1, &s1[m], 8);
                memcpy(&u2, &s2[m], 8);
                for (int b = 0; b < 6; ++b)
                    S[pos++] = (uint8_t)((u1 >> (8 * b)) ^ (u2 >> (8 * b)));
            }
        }
        for (uint64_t m = 0; m < d1 - d0; ++m)
            D[d0 + m] = (uint16_t)(S[2 * m] | ((uint16_t)S[2 * m + 1] << 8));
        for (uint64_t m = 0; m < b1 - b0; ++m)
            B[b0 + m] = S[2 * (d1 - d0) + m];
        free(S);
    }
}

/* ------------------------------------------------------------------------ */
/* Frame encryption on the expanded bit matrices (Sec. II-C, Algos 3-7).    */
/* ------------------------------------------------------------------------ */

/* bit k of byte x, k = 0 the least significant (the order of Algo 3). */
static uint8_t bit_of(uint8_t x, int k) { return (uint8_t)((x >> k) & 1u); }

/* A byte from its eight bits, bits[k] the coefficient of 2^k (Algo 7 packs
 * the bits back in the order Algo 3 took them out). */
static uint8_t byte_of(const uint8_t *bits) {
    uint32_t v = 0;
    for (int k = 0; k < 8; ++k) v += (uint32_t)bits[k] << k;
    return (uint8_t)v;
}

/* The confusion of Sec. II-C on one channel c, stated on the paper's
 * [8w x h] bit matrix, one byte per bit, row i of length 8w:
 *   M (i, 8j + k)                   = bit k of F(i, j, c)               (Algo 3)
 *   M1(i, (p + d_h(i)) mod 8w)      = M (i, p)                          (Algo 4)
 *   M2((i + d_v(p / 8)) mod h, p)   = M1(i, p)                          (Algo 5)
 *   M3(i, 8j + k)                   = M2(i, 8j + k) xor bit k of B(i, j, c)   (Algo 6)
 *   E (i, j, c)                     = sum over k of M3(i, 8j + k) 2^k    (Algo 7)
 * Readings: Algorithm 1's "M_t <- M_e" is a buffer swap after Algos 4, 5 and
 * 6 (after Algo 3 the extracted bits are already the matrix the shifts act
 * on); d_h(i) of (row i, channel c) is D[c*h + i]; d_v of (pixel column j,
 * channel c) is D[C*h + c*w + j] -- Algo 5 gives one d_v per thread, shared
 * by its eight bits, and Eq. (3)'s unbalanced parentheses are read as
 * Algo 5's ((i + (d_v mod h)) mod h); the byte of Algo 6 for pixel (i, j) of
 * channel c is B[(i*w + j)*C + c]. */
void oracle_permute_encrypt(const uint8_t *F, uint32_t h, uint32_t w, uint32_t C,
                            const uint16_t *D, const uint8_t *B, uint8_t *E) {
    uint64_t W8 = 8ull * w;
    uint8_t *M = (uint8_t *)malloc(h * W8);
    uint8_t *M1 = (uint8_t *)malloc(h * W8);
    for (uint32_t c = 0; c < C; ++c) {
        for (uint32_t i = 0; i < h; ++i)
            for (uint32_t j = 0; j < w; ++j)
                for (int k = 0; k < 8; ++k)
                    M[i * W8 + 8ull * j + k] = bit_of(F[((uint64_t)i * w + j) * C + c], k);
        for (uint32_t i = 0; i < h; ++i) {
            uint64_t dh = D[(uint64_t)c * h + i] % W8;
            for (uint64_t p = 0; p < W8; ++p) M1[i * W8 + (p + dh) % W8] = M[i * W8 + p];
        }
        /* M2 reuses M's storage: every position of M is written once. */
        uint8_t *M2 = M;
        for (uint64_t p = 0; p < W8; ++p) {
            uint64_t dv = D[(uint64_t)C * h + (uint64_t)c * w + p / 8] % h;
            for (uint32_t i = 0; i < h; ++i) M2[((i + dv) % h) * W8 + p] = M1[i * W8 + p];
        }
        uint8_t *M3 = M1;
        for (uint32_t i = 0; i < h; ++i)
            for (uint32_t j = 0; j < w; ++j)
                for (int k = 0; k < 8; ++k)
                    M3[i * W8 + 8ull * j + k] =
                        M2[i * W8 + 8ull * j + k] ^ bit_of(B[((uint64_t)i * w + j) * C + c], k);
        for (uint32_t i = 0; i < h; ++i)
            for (uint32_t j = 0; j < w; ++j)
                E[((uint64_t)i * w + j) * C + c] = byte_of(M3 + i * W8 + 8ull * j);
    }
    free(M);
    free(M1);
}

/* Decryption: the paper gives it only as "the inverse transformation of the
 * encryption procedure" (Sec. II-D).  On the same bit matrices, each map of
 * the encryption undone in reverse order:
 *   A (i, 8j + k)  = bit k of E(i, j, c)
 *   A2(i, 8j + k)  = A(i, 8j + k) xor bit k of B(i, j, c)      (Algo 6 is an involution)
 *   A1(i, p)       = A2((i + d_v(p / 8)) mod h, p)             (inverse of Algo 5)
 *   A0(i, p)       = A1(i, (p + d_h(i)) mod 8w)                (inverse of Algo 4)
 *   F (i, j, c)    = sum over k of A0(i, 8j + k) 2^k */
void oracle_permute_decrypt(const uint8_t *E, uint32_t h, uint32_t w, uint32_t C,
                            const uint16_t *D, const uint8_t *B, uint8_t *F) {
    uint64_t W8 = 8ull * w;
    uint8_t *A = (uint8_t *)malloc(h * W8);
    uint8_t *A1 = (uint8_t *)malloc(h * W8);
    for (uint32_t c = 0; c < C; ++c) {
        for (uint32_t i = 0; i < h; ++i)
            for (uint32_t j = 0; j < w; ++j) {
                uint8_t e = E[((uint64_t)i * w + j) * C + c], b = B[((uint64_t)i * w + j) * C + c];
                for (int k = 0; k < 8; ++k) A[i * W8 + 8ull * j + k] = bit_of(e, k) ^ bit_of(b, k);
            }
        for (uint64_t p = 0; p < W8; ++p) {
            uint64_t dv = D[(uint64_t)C * h + (uint64_t)c * w + p / 8] % h;
            for (uint32_t i = 0; i < h; ++i) A1[i * W8 + p] = A[((i + dv) % h) * W8 + p];
        }
        uint8_t *A0 = A;
        for (uint32_t i = 0; i < h; ++i) {
            uint64_t dh = D[(uint64_t)c * h + i] % W8;
            for (uint64_t p = 0; p < W8; ++p) A0[i * W8 + p] = A1[i * W8 + (p + dh) % W8];
        }
        for (uint32_t i = 0; i < h; ++i)
            for (uint32_t j = 0; j < w; ++j)
                F[((uint64_t)i * w + j) * C + c] = byte_of(A0 + i * W8 + 8ull * j);
    }
    free(A);
    free(A1);
}

/* ------------------------------------------------------------------------ */
/* Whole frame, Algorithm 1: digest -> reconstruct -> LHCS_m -> workers ->  */
/* confusion + XOR.  `state` is the stream's chaining state (in/out).       */
/* ------------------------------------------------------------------------ */

void oracle_frame_keystream(double state[4], double gamma, double hstep, uint32_t n,
                            const uint32_t u[4], const uint8_t H[32], uint32_t h,
                            uint32_t w, uint32_t C, uint16_t *D, uint8_t *B) {
    double *IR = (double *)malloc(sizeof(double) * 8 * n);
    double ns[4];
    oracle_master(state, H, u, gamma, hstep, n, IR, ns);
    oracle_keystream(IR, n, gamma, hstep, h, w, C, D, B);
    for (int m = 0; m < 4; ++m) state[m] = ns[m];
    free(IR);
}

/* Digest transport: an option of this implementation.  Sec. V sends the
 * SHA-256 hashes encrypted over the public channel but gives no mechanism.
 * Masked transport sends H xor M, with
 *   M = SHA-256("FHDMASK1" || LE64(x) || LE64(y) || LE64(z) || LE64(w) || LE64(gamma)),
 * the bit patterns of the stream's chaining state before the frame (the key's
 * x0..w0 for the first frame) and its gamma: 48 bytes, one SHA-256 block.  The
 * receiver holds the same state and recovers H = (H xor M) xor M.  A hash and
 * not further RK4 steps of the state: those would coincide with the previous
 * frame's last worker chain, which seeds from the same iterate. */
void oracle_digest_mask(const double state[4], double gamma, uint8_t M[32]) {
    uint8_t msg[48];
    memcpy(msg, "FHDMASK1", 8);
    const double v[5] = {state[0], state[1], state[2], state[3], gamma};
    for (int m = 0; m < 5; ++m) {
        uint64_t bits;
        memcpy(&bits, &v[m], 8);
        for (int i = 0; i < 8; ++i) msg[8 + 8 * m + i] = (uint8_t)(bits >> (8 * i));
    }
    oracle_sha256(msg, 48, M);
}

/* digest_mode 0: the paper's XOR fold; 1: the tree digest (not the paper's).
 * masked != 0: H_out is the transmitted digest H xor M (see oracle_digest_mask);
 * the keystream is still derived from H itself. */
void oracle_encrypt_frame(double state[4], double gamma, double hstep, uint32_t n,
                          const uint32_t u[4], const uint8_t *F, uint32_t h, uint32_t w,
                          uint32_t C, uint8_t *E, uint8_t H_out[32], uint32_t digest_mode, uint32_t masked) {
    uint64_t N = (uint64_t)h * w * C;
    uint64_t LD = (uint64_t)C * (h + w);
    uint8_t H[32], M[32];
    if (digest_mode == 1) oracle_frame_digest_tree(F, N, n, H);
    else oracle_frame_digest(F, N, n, H);
    if (masked) oracle_digest_mask(state, gamma, M);
    for (int i = 0; i < 32; ++i) H_out[i] = masked ? (uint8_t)(H[i] ^ M[i]) : H[i];
    uint16_t *D = (uint16_t *)malloc(sizeof(uint16_t) * (LD ? LD : 1));
    uint8_t *B = (uint8_t *)malloc(N ? N : 1);
    oracle_frame_keystream(state, gamma, hstep, n, u, H, h, w, C, D, B);
    oracle_permute_encrypt(F, h, w, C, D, B, E);
    free(D);
    free(B);
}

/* masked != 0: H_in is the transmitted digest H xor M. */
void oracle_decrypt_frame(double state[4], double gamma, double hstep, uint32_t n,
                          const uint32_t u[4], const uint8_t *E, uint32_t h, uint32_t w,
                          uint32_t C, const uint8_t H_in[32], uint8_t *F, uint32_t masked) {
    uint64_t N = (uint64_t)h * w * C;
    uint64_t LD = (uint64_t)C * (h + w);
    uint8_t H[32], M[32];
    if (masked) oracle_digest_mask(state, gamma, M);
    for (int i = 0; i < 32; ++i) H[i] = masked ? (uint8_t)(H_in[i] ^ M[i]) : H_in[i];
    uint16_t *D = (uint16_t *)malloc(sizeof(uint16_t) * (LD ? LD : 1));
    uint8_t *B = (uint8_t *)malloc(N ? N : 1);
    oracle_frame_keystream(state, gamma, hstep, n, u, H, h, w, C, D, B);
    oracle_permute_decrypt(E, h, w, C, D, B, F);
    free(D);
    free(B);
}
