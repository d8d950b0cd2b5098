// K2a (master) and K2b (workers): the Lorenz hyperchaotic iterations.
//
// Eq. (1) of the paper with sigma = 10, rho = 28, beta = 8/3 and the stream's
// gamma, integrated by classical RK4 with step h (the paper names no
// integrator; this reading is fixed with the oracle):
//   k1 = f(s); k2 = f(s + (h/2) k1); k3 = f(s + (h/2) k2); k4 = f(s + h k3);
//   s' = s + (h/6) (((k1 + 2 k2) + 2 k3) + k4),
// every operation an explicit round-to-nearest binary64 intrinsic (no FMA
// contraction; the library is also built with -fmad=false), so the iterates
// are bit-identical to a plain C implementation.  2 k is an exact doubling
// done on the bit pattern.
//
// GPU mapping.  On this GPU a binary64 warp instruction occupies the SM
// sub-partition's FP64 pipe for ~64 cycles whatever the number of active
// lanes, and every chain is strictly sequential, so the time per step is set
// by the binary64 instructions one warp issues per step.  A warp carries 32
// independent chains and one chain's four variables are spread over four
// warps on four sub-partitions: a CTA is 4 warps, warp v owns variable v
// (x, y, z, w) of 32 chains (lane = chain), and the stage inputs are exchanged
// through shared memory with one barrier per RK4 stage.  (Measured on GB300:
// ~3.5k cycles per step; one warp per 8 chains with lane-local variables and
// shuffles, and moving off-path operations to exact integer emulation, were
// both slower.)
#include "common.cuh"

namespace fhd {
namespace {

constexpr double kSigma = 10.0;
constexpr double kRho = 28.0;
constexpr double kBeta = 8.0 / 3.0;

// Exact 2*k on the IEEE-754 encoding (zero, subnormal and normal inputs).
__device__ __forceinline__ double twice(double k) {
    unsigned long long b = (unsigned long long)__double_as_longlong(k);
    unsigned long long mag = b & 0x7fffffffffffffffull;
    if (mag == 0) return k;
    if (mag < (1ull << 52)) return __longlong_as_double((long long)((b & 0x8000000000000000ull) | (mag << 1)));
    if (mag >= 0x7fe0000000000000ull) return __dmul_rn(2.0, k);   // overflow, inf, nan: hardware
    return __longlong_as_double((long long)(b + (1ull << 52)));
}

// Component v of Eq. (1) at (x, y, z, w); v is warp-uniform.
__device__ __forceinline__ double lhcs_f(int v, double x, double y, double z, double w, double gamma) {
    switch (v) {
        case 0: return __dadd_rn(__dmul_rn(kSigma, __dsub_rn(y, x)), w);
        case 1: return __dsub_rn(__dsub_rn(__dmul_rn(kRho, x), y), __dmul_rn(x, z));
        case 2: return __dsub_rn(__dmul_rn(x, y), __dmul_rn(kBeta, z));
        default: return __dsub_rn(__dmul_rn(gamma, w), __dmul_rn(y, z));
    }
}

struct Rk4 {
    double h, hh, h6;
};

// One RK4 step of 32 chains by 4 cooperating warps.  On entry buf[0][*][lane]
// holds every variable of the current state (visible to all warps); on exit
// buf[0] holds the new state and `s` this warp's component of it.
__device__ __forceinline__ void rk4_step_coop(double &s, int v, int lane, double gamma, const Rk4 &c,
                                              double (*buf)[4][32]) {
    double k, acc, t;
    k = lhcs_f(v, buf[0][0][lane], buf[0][1][lane], buf[0][2][lane], buf[0][3][lane], gamma);
    acc = k;
    t = __dadd_rn(s, __dmul_rn(c.hh, k));
    buf[1][v][lane] = t;
    __syncthreads();
    k = lhcs_f(v, buf[1][0][lane], buf[1][1][lane], buf[1][2][lane], buf[1][3][lane], gamma);
    t = __dadd_rn(s, __dmul_rn(c.hh, k));
    acc = __dadd_rn(acc, twice(k));
    buf[0][v][lane] = t;
    __syncthreads();
    k = lhcs_f(v, buf[0][0][lane], buf[0][1][lane], buf[0][2][lane], buf[0][3][lane], gamma);
    t = __dadd_rn(s, __dmul_rn(c.h, k));
    acc = __dadd_rn(acc, twice(k));
    buf[1][v][lane] = t;
    __syncthreads();
    k = lhcs_f(v, buf[1][0][lane], buf[1][1][lane], buf[1][2][lane], buf[1][3][lane], gamma);
    acc = __dadd_rn(acc, k);
    s = __dadd_rn(s, __dmul_rn(c.h6, acc));
    buf[0][v][lane] = s;
    __syncthreads();
}

// Sec. II-A, Fig. 1a: reconstruct one initial condition from 8 digest bytes
// (two for the integer part mod u, six for the 48-bit fraction), v by
// magnitude; non-finite or |v| >= 2^52 contributes 0 and 0.
__device__ __forceinline__ double reconstruct(double v, const uint8_t *hb, uint32_t u) {
    double a = fabs(v);
    unsigned long long I = 0, F48 = 0;
    if (a < 0x1p52) {
        I = __double2ull_rz(a);
        double F = __dsub_rn(a, __ull2double_rn(I));
        F48 = __double2ull_rz(__dmul_rn(F, 0x1p48));
    }
    unsigned long long hi16 = (unsigned long long)hb[0] | ((unsigned long long)hb[1] << 8);
    unsigned long long h48 = 0;
#pragma unroll
    for (int i = 5; i >= 0; --i) h48 = (h48 << 8) | hb[2 + i];
    unsigned long long ip = ((I & 0xffffull) ^ hi16) % u;
    double fp = __dmul_rn(__ull2double_rn(F48 ^ h48), 0x1p-48);
    return __dadd_rn(__ull2double_rn(ip), fp);
}

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

// Reconstruct from (state, H), run LHCS_m 2n steps writing IR, return the
// last iterate in `s` (this warp's component).  All lanes carry the chain.
__device__ void master_frame(double &s, int v, int lane, double gamma, const uint8_t *H_smem,
                             const uint32_t *u, uint32_t n, const Rk4 &c, double *IR, double (*buf)[4][32]) {
    s = reconstruct(s, H_smem + 8 * v, u[v]);
    buf[0][v][lane] = s;
    __syncthreads();
    for (uint32_t t = 0; t < 2 * n; ++t) {
        rk4_step_coop(s, v, lane, gamma, c, buf);
        if (lane == 0) IR[4 * t + v] = s;
    }
}

// K2a: one CTA per stream of the batch; the stream's frames in call order.
__global__ void __launch_bounds__(128) master_kernel(const __grid_constant__ Batch b, StreamState *states,
                                                     int encrypt, unsigned *status) {
    __shared__ double buf[2][4][32];
    __shared__ __align__(16) uint8_t H[32];
    const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t g = blockIdx.x;
    if (g >= b.groups) return;
    const Rk4 c{b.hstep, b.hhalf, b.hsixth};
    const uint32_t first = b.group_begin[g], last = b.group_begin[g + 1];
    const uint32_t slot = b.f[b.order[first]].slot;
    StreamState *st = states + slot;
    double s = st->v[v];
    const double gamma = b.f[b.order[first]].gamma;
    for (uint32_t k = first; k < last; ++k) {
        const FrameDesc &fd = b.f[b.order[k]];
        if (threadIdx.x < 8) {
            uint32_t word;
            if (encrypt) {
                const uint32_t *p = reinterpret_cast<const uint32_t *>(fd.part);
                word = 0;
                for (uint32_t i = 0; i < b.n; ++i) word ^= p[8 * i + threadIdx.x];
                reinterpret_cast<uint32_t *>(fd.digest)[threadIdx.x] = word;
            } else {
                word = reinterpret_cast<const uint32_t *>(fd.digest)[threadIdx.x];
            }
            reinterpret_cast<uint32_t *>(H)[threadIdx.x] = word;
        }
        __syncthreads();
        master_frame(s, v, lane, gamma, H, b.u, b.n, c, fd.IR, buf);
        __syncthreads();
    }
    if (lane == 0) {
        st->v[v] = s;
        if (!finite(s)) atomicOr(status, kStatusNonFinite);
        if (v == 0) st->frames += (last - first);
    }
}

// fhd_master: one CTA, one state of 5 doubles (x, y, z, w, gamma).
__global__ void __launch_bounds__(128) master_raw_kernel(double *state5, const uint8_t *Hg, uint32_t n,
                                                         Rk4 c, uint4 u4, double *IR, unsigned *status) {
    __shared__ double buf[2][4][32];
    __shared__ __align__(16) uint8_t H[32];
    const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < 32) H[threadIdx.x] = Hg[threadIdx.x];
    __syncthreads();
    const uint32_t u[4] = {u4.x, u4.y, u4.z, u4.w};
    double s = state5[v];
    const double gamma = state5[4];
    master_frame(s, v, lane, gamma, H, u, n, c, IR, buf);
    if (lane == 0) {
        state5[v] = s;
        if (!finite(s) && status) atomicOr(status, kStatusNonFinite);
    }
}

// K2b worker geometry of one frame.
struct WorkerSlice {
    uint64_t d0, nd, b0, nb;
};
__device__ __forceinline__ WorkerSlice worker_slice(uint64_t LD, uint64_t LB, uint32_t n, uint32_t p) {
    WorkerSlice w;
    w.d0 = (uint64_t)(((unsigned __int128)LD * p) / n);
    w.nd = (uint64_t)(((unsigned __int128)LD * (p + 1)) / n) - w.d0;
    w.b0 = (uint64_t)(((unsigned __int128)LB * p) / n);
    w.nb = (uint64_t)(((unsigned __int128)LB * (p + 1)) / n) - w.b0;
    return w;
}

constexpr uint32_t kPairsPerCta = 16;   // 32 chains = 16 worker pairs

__device__ void keystream_cta(const FrameDesc &fd, uint32_t n, uint32_t pg, double gamma, const Rk4 &c,
                              double (*buf)[4][32]) {
    const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t p = pg * kPairsPerCta + (lane >> 1);
    const bool active = p < n;
    const uint64_t LD = (uint64_t)fd.C * (fd.h + fd.w);
    const uint64_t LB = fd.N;
    WorkerSlice ws{0, 0, 0, 0};
    if (active) ws = worker_slice(LD, LB, n, p);
    const uint64_t need = 2 * ws.nd + ws.nb;
    // Uniform trip count: the longest slice of the frame.
    const uint64_t need_max = 2 * ((LD + n - 1) / n) + (LB + n - 1) / n;
    const uint64_t T = (need_max + 23) / 24;
    double s = active ? fd.IR[4 * (2 * p + (lane & 1)) + v] : 0.0;
    buf[0][v][lane] = s;
    __syncthreads();
    uint8_t *Dbytes = reinterpret_cast<uint8_t *>(fd.D) + 2 * ws.d0;
    uint8_t *Bp = fd.B + ws.b0;
    const uint64_t ndb = 2 * ws.nd;
    const int half = (lane & 1) * 3;
    for (uint64_t t = 0; t < T; ++t) {
        rk4_step_coop(s, v, lane, gamma, c, buf);
        unsigned long long mine = (unsigned long long)__double_as_longlong(s) & 0xffffffffffffull;
        unsigned long long other = __shfl_xor_sync(0xffffffffu, mine, 1);
        unsigned long long x = mine ^ other;
        uint64_t pos0 = 24 * t + 6 * v;
        if (active && pos0 < need) {
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) {
                uint64_t pos = pos0 + half + bb;
                uint8_t byte = (uint8_t)(x >> (8 * (half + bb)));
                if (pos < ndb) Dbytes[pos] = byte;
                else if (pos < need) Bp[pos - ndb] = byte;
            }
        }
    }
}

// K2b: ceil(n/16) CTAs per frame, each 16 worker pairs of one frame.
__global__ void __launch_bounds__(128) keystream_kernel(const __grid_constant__ Batch b) {
    __shared__ double buf[2][4][32];
    const uint32_t cpf = (b.n + kPairsPerCta - 1) / kPairsPerCta;
    const uint32_t f = blockIdx.x / cpf, pg = blockIdx.x % cpf;
    if (f >= b.count) return;
    const FrameDesc &fd = b.f[f];
    const Rk4 c{b.hstep, b.hhalf, b.hsixth};
    keystream_cta(fd, b.n, pg, fd.gamma, c, buf);
}

}  // namespace

cudaError_t launch_master(const Batch &b, StreamState *states, bool encrypt, unsigned *status, cudaStream_t s) {
    if (!b.groups) return cudaSuccess;
    master_kernel<<<b.groups, 128, 0, s>>>(b, states, encrypt ? 1 : 0, status);
    return cudaGetLastError();
}

cudaError_t launch_master_raw(double *state5, const uint8_t *H, uint32_t n, double hstep, const uint32_t u[4],
                              double *IR, unsigned *status, cudaStream_t s) {
    Rk4 c{hstep, hstep / 2.0, hstep / 6.0};   // host arithmetic: IEEE round-to-nearest
    master_raw_kernel<<<1, 128, 0, s>>>(state5, H, n, c, make_uint4(u[0], u[1], u[2], u[3]), IR, status);
    return cudaGetLastError();
}

cudaError_t launch_keystream(const Batch &b, cudaStream_t s) {
    if (!b.count) return cudaSuccess;
    const uint32_t cpf = (b.n + kPairsPerCta - 1) / kPairsPerCta;
    keystream_kernel<<<b.count * cpf, 128, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace fhd
