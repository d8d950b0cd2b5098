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

// ---- One-trajectory route (see traj_records in common.cuh; the warp and chunk bodies are in chaos_dev.cuh).

// K2t: the records of six frames per warp, one chain per frame (lane 4c + v: variable v of frame
// 6 blockIdx.x + c).
__global__ void __launch_bounds__(32) trajectory_kernel(const __grid_constant__ Batch b) {
    const int lane = threadIdx.x;
    const uint32_t f = blockIdx.x * kChainsPerWarp + (lane >> 2);
    const bool active = (lane >> 2) < kChainsPerWarp && f < b.count;
    trajectory_warp(active ? &b.f[f] : nullptr, b.n, Rk4{b.hstep, b.hhalf, b.hsixth}, lane);
}

// K2e: D and B of every frame from its records.  CTA (x, f) takes worker slice i = x / cps of frame f and
// part j = x % cps of it: part 0 also writes the slice's D bytes, and the parts split the slice's B bytes
// in runs of kEmitChunks x kEmitThreads 16-byte chunks of B.
constexpr int kEmitThreads = 256;
constexpr int kEmitChunks = 4;

__global__ void __launch_bounds__(kEmitThreads) emit_kernel(const __grid_constant__ Batch b, uint32_t cps) {
    const uint32_t f = blockIdx.y, i = blockIdx.x / cps, j = blockIdx.x % cps;
    if (f >= b.count || i >= b.n) return;
    const FrameDesc &fd = b.f[f];
    __shared__ WorkerSlice ws_s;
    if (threadIdx.x == 0) ws_s = worker_slice((uint64_t)fd.C * (fd.h + fd.w), fd.N, b.n, i);
    __syncthreads();
    const WorkerSlice ws = ws_s;
    if (j == 0) emit_d_slice(fd, b.n, i, ws, threadIdx.x, kEmitThreads);
    if (!ws.nb) return;
    const uint64_t per = 16ull * kEmitThreads * kEmitChunks;
    const uint64_t base = (ws.b0 >> 4) << 4;   // the slice's first chunk
    const uint64_t lo = base + j * per, hi = lo + per;
    const uint64_t a = lo > ws.b0 ? lo : ws.b0, e = hi < ws.b0 + ws.nb ? hi : ws.b0 + ws.nb;
    if (a < e) emit_b_part(fd, b.n, i, ws, a, e, threadIdx.x, kEmitThreads);
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
