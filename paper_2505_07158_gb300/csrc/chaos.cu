// K2a (master) and K2b (workers): the Lorenz hyperchaotic iterations.
//
// Eq. (1) of the paper with sigma = 10, rho = 28, beta = 8/3 and the stream's
// gamma, integrated by classical RK4 with step h (the paper names no
// integrator; this reading is fixed with the oracle):
//   k1 = f(s); k2 = f(s + (h/2) k1); k3 = f(s + (h/2) k2); k4 = f(s + h k3);
//   s' = s + (h/6) (((k1 + 2 k2) + 2 k3) + k4),
// every operation an explicit round-to-nearest binary64 intrinsic (no FMA
// contraction; the library is also built with -fmad=false), so the iterates
// are bit-identical to a plain C implementation.  The term acc + 2 k of the
// combination is one fma(k, 2, acc) (see below).
//
// GPU mapping.  On this GPU a binary64 instruction occupies the SM
// sub-partition's FP64 pipe for ~64 cycles whatever the number of active
// lanes, one after another (no overlap, dependent or not), and handing a
// binary64 result to another unit (shuffle, shared memory, integer select)
// costs ~15-40 more cycles per hand-off; every chain is strictly sequential.
// So the time per step is the binary64 instructions one warp issues per step
// plus its hand-offs.  A warp carries six chains, one variable per lane
// (lane = 4 chain + v, v = x, y, z, w), and every component of Eq. (1) is the
// same four fused multiply-adds with per-lane operands:
//   p = fma(Pa, Pb, -Pc); q = fma(Qa, Qb, -0); p2 = fma(p, B2, -P2); k = fma(q, kS, p2)
//   v = x: p = Y*1 - X, q = W*1, p2 = sigma p,     k = q + p2  = sigma (y - x) + w
//   v = y: p = X rho,   q = X Z, p2 = p*1 - Y,     k = p2 - q  = (rho x - y) - x z
//   v = z: p = Z beta,  q = X Y, p2 = -p,          k = q + p2  = x y - beta z
//   v = w: p = W gamma, q = Y Z, p2 = p,           k = p2 - q  = gamma w - y z
// Each fma rounds once, a product with addend -0 or a sum with a factor of
// +-1, so k is bit-identical to the dmul/dadd/dsub sequence of the plain
// definition.  The variable operands Pa, Pc, Qa, Qb, P2 arrive by five warp
// shuffles per stage; a constant operand (the 1 of v = x, the 0 addends) is
// shuffled from lane 24 (+0) or lane 25 (1.0), which stay fixed points of the
// update because their own k is +0.  No selects and no barriers remain: a
// step takes 27 binary64 instructions and ~2.0k cycles on GB300 (the earlier
// mapping, one warp per variable with a shared-memory exchange and one barrier
// per stage, took ~3.5k).  In the combination, acc + 2 k is one fma(k, 2, acc):
// 2 k is exact, so it equals the separate doubling and add whenever 2 k is
// finite (an overflowing 2 k makes the definition's state non-finite anyway).
#include "chaos_dev.cuh"

namespace fhd {
namespace {

// K2a: one warp per stream of the batch; the stream's frames in call order.
__global__ void __launch_bounds__(32) master_kernel(const __grid_constant__ Batch b, StreamState *states,
                                                    unsigned *status) {
    __shared__ __align__(16) uint8_t H[32];
    if (blockIdx.x >= b.groups) return;
    master_stream(b, blockIdx.x, states, status, H, threadIdx.x, [](uint32_t) { return true; }, [](uint32_t) {});
}

// fhd_master: one warp, one state of 5 doubles (x, y, z, w, gamma).
__global__ void __launch_bounds__(32) master_raw_kernel(double *state5, const uint8_t *Hg, uint32_t n, Rk4 c,
                                                        uint4 u4, double *IR, unsigned *status) {
    __shared__ __align__(16) uint8_t H[32];
    const int lane = threadIdx.x;
    H[lane] = Hg[lane];
    __syncwarp();
    const uint32_t u[4] = {u4.x, u4.y, u4.z, u4.w};
    const double gamma = state5[4];
    const LaneRole role = lane_role(lane, gamma);
    double s = lane_init(lane, lane < 4 ? state5[lane] : 0.0);
    master_frame(s, lane, role, H, u, n, c, IR);
    if (lane < 4) {
        state5[lane] = s;
        if (!finite(s) && status) atomicOr(status, kStatusNonFinite);
    }
}

// K2b: one warp per kPairs worker pairs of one frame (three with the six-chain step, four with the
// eight-chain step); a CTA carries blockDim.x / 32 consecutive such warps (warps of one CTA are spread over
// the SM's sub-partitions).
// kMix (eight-chain step only): b.int_mix of every 8 consecutive warps step on the integer pipes instead of
// the binary64 pipe (the same bytes: rk4_step_lanes8_int).  A separate instantiation, so that the binary64-only
// kernel keeps its own register allocation.
template <int kPairs, bool kMix = false>
__global__ void __launch_bounds__(256) keystream_kernel(const __grid_constant__ Batch b) {
    const uint32_t wpf = (b.n + kPairs - 1) / kPairs;
    const uint32_t task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint32_t f = task / wpf, pg = task % wpf;
    if (f >= b.count) return;
    const Rk4 c{b.hstep, b.hhalf, b.hsixth};
    if constexpr (kMix) {
        if ((task & 7) < b.int_mix) {
            keystream_warp<kPairs, true>(b.f[f], b.n, c, pg, threadIdx.x & 31);
            return;
        }
    }
    keystream_warp<kPairs>(b.f[f], b.n, c, pg, threadIdx.x & 31);
}

// ---- One-trajectory route (see traj_records in common.cuh).
//
// K2t: the records of six frames per warp, one chain per frame, in the six-chain layout of LHCS_m (lane
// 4c + v holds variable v of frame 6 blockIdx.x + c; lanes 24..31 hold the constants).  Steps k = 1, 2, ...
// take the state from s_k to s_{k+1}: while k < 2n it is LHCS_m's iterate IR[k], read back, and from k = 2n
// on one RK4 step.  After step k >= 2 the warp writes record k - 2 = (s_k, s_{k+1}): the 48-bit XOR of each
// variable's two bit patterns (its six low mantissa bytes) is packed with the next variable's by one
// shuffle, and lanes v = 0, 1, 2 store the record's three 64-bit words.  A chain is strictly sequential, so
// its time is the number of steps times the step's latency (27 binary64 instructions back to back, plus the
// hand-offs); the warp runs to its longest frame.
__device__ __forceinline__ unsigned long long low48(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0xffffffffffffull;
}

__global__ void __launch_bounds__(32) trajectory_kernel(const __grid_constant__ Batch b) {
    const int lane = threadIdx.x, v = lane & 3, ch = lane >> 2;
    const uint32_t f = blockIdx.x * kChainsPerWarp + ch;
    const bool active = ch < kChainsPerWarp && f < b.count;
    const uint32_t n = b.n;
    uint64_t R = 0;
    double gamma = 0.0;
    const double *IR = nullptr;
    uint64_t *rec = nullptr;
    if (active) {
        const FrameDesc &fd = b.f[f];
        R = traj_records((uint64_t)fd.C * (fd.h + fd.w), fd.N, n);
        gamma = fd.gamma;
        IR = fd.IR;
        rec = reinterpret_cast<uint64_t *>(fd.T);
    }
    unsigned long long Rmax = R;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, Rmax, o);
        Rmax = t > Rmax ? t : Rmax;
    }
    const Rk4 c{b.hstep, b.hhalf, b.hsixth};
    const LaneRole role = lane_role(lane, gamma);
    double s = lane_init(lane, active && FHD_IN(v, 8ull * n, kSiteTrajIR) ? __ldcg(IR + v) : 0.0);   // s_1
    unsigned long long prev = low48(s);
    for (uint64_t k = 1; k <= Rmax + 1; ++k) {
        if (k < 2ull * n) {   // s_{k+1} = IR[k] (uniform over the warp)
            if (active && FHD_IN(4 * k + v, 8ull * n, kSiteTrajIR)) s = __ldcg(IR + 4 * k + v);
        } else {
            rk4_step_lanes(s, role, c);
        }
        const unsigned long long cur = low48(s);
        const unsigned long long x = prev ^ cur;
        const unsigned long long nx = __shfl_down_sync(0xffffffffu, x, 1);
        const uint64_t r = k - 2;
        if (k >= 2 && active && v < 3 && r < R && FHD_IN(3 * r + v, 3 * R, kSiteTrajRecord))
            rec[3 * r + v] = (x >> (16 * v)) | (nx << (48 - 16 * v));
        prev = cur;
    }
}

// K2e: D and B of every frame from its records.  CTA (x, f) takes worker slice i = x / cps of frame f, and
// part j = x % cps of it: part 0 also writes the slice's D bytes (byte q of the slice's D bytes is record
// byte 48 i + q), and the parts split the slice's B bytes (B[b0 + m] is record byte 48 i + 2 nd + m) in
// 16-byte chunks of B, kEmitChunks per thread.  A chunk inside the slice is one 16-byte store of bytes
// o .. o + 15 of two aligned 16-byte record loads (o = the source offset mod 16, the same for the whole
// slice); the chunks at the slice's ends, and every chunk of an unaligned B, go byte by byte.
constexpr int kEmitThreads = 256;
constexpr int kEmitChunks = 4;

__device__ __forceinline__ uint32_t word8(const uint4 &a, const uint4 &b, int i) {
    switch (i) {
        case 0: return a.x;
        case 1: return a.y;
        case 2: return a.z;
        case 3: return a.w;
        case 4: return b.x;
        case 5: return b.y;
        case 6: return b.z;
        default: return b.w;
    }
}

__global__ void __launch_bounds__(kEmitThreads) emit_kernel(const __grid_constant__ Batch b, uint32_t cps) {
    const uint32_t f = blockIdx.y, i = blockIdx.x / cps, j = blockIdx.x % cps;
    if (f >= b.count || i >= b.n) return;
    const FrameDesc &fd = b.f[f];
    const uint64_t LD = (uint64_t)fd.C * (fd.h + fd.w), LB = fd.N;
    __shared__ WorkerSlice ws_s;
    if (threadIdx.x == 0) ws_s = worker_slice(LD, LB, b.n, i);
    __syncthreads();
    const WorkerSlice ws = ws_s;
    const uint8_t *T = fd.T;
    const uint64_t tlim = traj_bytes(LD, LB, b.n);
    const uint64_t s0 = 48ull * i;   // worker i's stream in the records
    if (j == 0) {
        uint8_t *Db = reinterpret_cast<uint8_t *>(fd.D);
        for (uint64_t q = threadIdx.x; q < 2 * ws.nd; q += kEmitThreads) {
            const uint8_t byte = FHD_IN(s0 + q, tlim, kSiteEmitLoad) ? T[s0 + q] : 0;
            if (FHD_IN(2 * ws.d0 + q, 2 * LD, kSiteEmitStore)) Db[2 * ws.d0 + q] = byte;
        }
    }
    if (!ws.nb) return;
    uint8_t *B = fd.B;
    const uint64_t sb = s0 + 2 * ws.nd;   // record byte of B[b0]
    const uint64_t lo = ws.b0, hi = ws.b0 + ws.nb;
    const bool aligned = (reinterpret_cast<uintptr_t>(B) & 15) == 0;
    const uint64_t c_lo = lo >> 4, c_hi = (hi + 15) >> 4;   // chunks [16 c, 16 c + 16) meeting the slice
    const uint32_t o = (uint32_t)((sb - lo) & 15), q = o >> 2, r = 8 * (o & 3);
#pragma unroll
    for (int u = 0; u < kEmitChunks; ++u) {
        const uint64_t cidx = c_lo + ((uint64_t)j * kEmitChunks + u) * kEmitThreads + threadIdx.x;
        if (cidx >= c_hi) break;
        const uint64_t p0 = 16 * cidx;
        if (aligned && p0 >= lo && p0 + 16 <= hi) {
            const uint64_t sp = sb + (p0 - lo);   // sp mod 16 = o
            const uint64_t a = sp & ~15ull;
            uint4 w0 = make_uint4(0, 0, 0, 0), w1 = w0;
            if (FHD_IN(a + 31, tlim, kSiteEmitLoad)) {
                w0 = __ldcg(reinterpret_cast<const uint4 *>(T + a));
                w1 = __ldcg(reinterpret_cast<const uint4 *>(T + a) + 1);
            }
            uint4 out;
            out.x = __funnelshift_r(word8(w0, w1, q), word8(w0, w1, q + 1), r);
            out.y = __funnelshift_r(word8(w0, w1, q + 1), word8(w0, w1, q + 2), r);
            out.z = __funnelshift_r(word8(w0, w1, q + 2), word8(w0, w1, q + 3), r);
            out.w = __funnelshift_r(word8(w0, w1, q + 3), word8(w0, w1, q + 4), r);
            if (FHD_IN(p0 + 15, LB, kSiteEmitStore)) *reinterpret_cast<uint4 *>(B + p0) = out;
        } else {
            const uint64_t e = p0 + 16 < hi ? p0 + 16 : hi;
            for (uint64_t p = p0 > lo ? p0 : lo; p < e; ++p) {
                const uint64_t sp = sb + (p - lo);
                const uint8_t byte = FHD_IN(sp, tlim, kSiteEmitLoad) ? T[sp] : 0;
                if (FHD_IN(p, LB, kSiteEmitStore)) B[p] = byte;
            }
        }
    }
}

int g_ks_route = FHD_KS_ROUTE_TRAJECTORY;

}  // namespace

int set_keystream_route(int route) {
    if (route != FHD_KS_ROUTE_TRAJECTORY && route != FHD_KS_ROUTE_PAIRS) return -1;
    const int old = g_ks_route;
    g_ks_route = route;
    return old;
}

int keystream_route() { return g_ks_route; }

cudaError_t launch_trajectory_keystream(const Batch &b, cudaStream_t s) {
    if (!b.count) return cudaSuccess;
    uint64_t nb_max = 0;
    for (uint32_t k = 0; k < b.count; ++k) {
        const uint64_t nb = (b.f[k].N + b.n - 1) / b.n;
        nb_max = nb > nb_max ? nb : nb_max;
    }
    trajectory_kernel<<<(b.count + kChainsPerWarp - 1) / kChainsPerWarp, 32, 0, s>>>(b);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t chunks = nb_max / 16 + 2;   // chunks of B one slice meets
    const uint64_t per_cta = (uint64_t)kEmitThreads * kEmitChunks;
    const uint64_t cps = (chunks + per_cta - 1) / per_cta;
    const uint64_t gx = cps * b.n;
    if (gx > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    emit_kernel<<<dim3((unsigned)gx, b.count), kEmitThreads, 0, s>>>(b, (uint32_t)cps);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_master(const Batch &b, StreamState *states, unsigned *status, cudaStream_t s) {
    if (!b.groups) return cudaSuccess;
    master_kernel<<<b.groups, 32, 0, s>>>(b, states, status);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_master_raw(double *state5, const uint8_t *H, uint32_t n, double hstep, const uint32_t u[4],
                              double *IR, unsigned *status, cudaStream_t s) {
    Rk4 c{hstep, hstep / 2.0, hstep / 6.0};   // host arithmetic: IEEE round-to-nearest
    master_raw_kernel<<<1, 32, 0, s>>>(state5, H, n, c, make_uint4(u[0], u[1], u[2], u[3]), IR, status);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_keystream(const Batch &b, cudaStream_t s, bool dense, uint32_t warps_per_cta, uint32_t smem) {
    if (!b.count) return cudaSuccess;
    const uint32_t k = warps_per_cta ? warps_per_cta : 1;
    if (smem > 48 * 1024) {
        const void *fns[3] = {(const void *)keystream_kernel<4>, (const void *)keystream_kernel<4, true>,
                              (const void *)keystream_kernel<kPairsPerWarp>};
        for (const void *f : fns) {
            cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
    }
    if (dense) {
        const uint32_t warps = b.count * ((b.n + 3) / 4);
        if (b.int_mix)
            keystream_kernel<4, true><<<(warps + k - 1) / k, 32 * k, smem, s>>>(b);
        else
            keystream_kernel<4><<<(warps + k - 1) / k, 32 * k, smem, s>>>(b);
        note_launch();
        return cudaGetLastError();
    }
    const uint32_t warps = b.count * ((b.n + kPairsPerWarp - 1) / kPairsPerWarp);
    keystream_kernel<kPairsPerWarp><<<(warps + k - 1) / k, 32 * k, smem, s>>>(b);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fhd

FHD_BOUNDS_TAKER(take_bounds_chaos)
