// Device code of the Lorenz hyperchaotic iterations (Eq. (1), RK4) shared by the chaining and worker kernels
// and the persistent batch kernel: the lane-packed RK4 steps, the reconstruction, LHCS_m of one stream and
// one warp of worker pairs.  See chaos.cu for the design.
#pragma once
#include "binary64_int.cuh"
#include "bounds.cuh"
#include "common.cuh"
#include "sha256_core.cuh"

namespace fhd {
namespace {

constexpr double kSigma = 10.0;
constexpr double kRho = 28.0;
constexpr double kBeta = 8.0 / 3.0;

struct Rk4 {
    double h, hh, h6;
};

constexpr int kChainsPerWarp = 6;   // lanes 0..23
constexpr int kPairsPerWarp = 3;
constexpr int kLaneZero = 24;       // holds +0
constexpr int kLaneOne = 25;        // holds 1.0

// Per-lane operand sources and coefficients of the component template.
struct LaneRole {
    double Pb, B2, kS;
    int sPa, sPc, sQa, sQb, sP2;
};

__device__ __forceinline__ LaneRole lane_role(int lane, double gamma) {
    LaneRole r;
    const int v = lane & 3, base = lane & ~3;
    if (lane >= 4 * kChainsPerWarp) {   // constant lanes: every operand +0, k = +0
        r.Pb = r.B2 = r.kS = 0.0;
        r.sPa = r.sPc = r.sQa = r.sQb = r.sP2 = kLaneZero;
        return r;
    }
    r.Pb = v == 0 ? 1.0 : v == 1 ? kRho : v == 2 ? kBeta : gamma;
    r.B2 = v == 0 ? kSigma : v == 2 ? -1.0 : 1.0;
    r.kS = (v == 0 || v == 2) ? 1.0 : -1.0;
    r.sPa = base + (v == 0 ? 1 : v == 1 ? 0 : v);                 // Y, X, Z, W
    r.sPc = v == 0 ? base : kLaneZero;                            // X, +0, +0, +0
    r.sQa = base + (v == 0 ? 3 : v == 3 ? 1 : 0);                 // W, X, X, Y
    r.sQb = v == 0 ? kLaneOne : base + (v == 2 ? 1 : 2);          // 1, Z, Y, Z
    r.sP2 = v == 1 ? base + 1 : kLaneZero;                        // +0, Y, +0, +0
    return r;
}

// Initial value of a lane: the chain variable, or the constant a constant lane holds.
__device__ __forceinline__ double lane_init(int lane, double chain_value) {
    return lane < 4 * kChainsPerWarp ? chain_value : (lane == kLaneOne ? 1.0 : 0.0);
}

// One RK4 step of the warp's six chains; s is this lane's variable.  All 32
// lanes of the warp must call it together.
__device__ __forceinline__ void rk4_step_lanes(double &s, const LaneRole &r, const Rk4 &c) {
    double tin = s, acc = 0.0;
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        const double Pa = __shfl_sync(0xffffffffu, tin, r.sPa);
        const double Pc = __shfl_sync(0xffffffffu, tin, r.sPc);
        const double Qa = __shfl_sync(0xffffffffu, tin, r.sQa);
        const double Qb = __shfl_sync(0xffffffffu, tin, r.sQb);
        const double P2 = __shfl_sync(0xffffffffu, tin, r.sP2);
        const double p = __fma_rn(Pa, r.Pb, -Pc);
        const double q = __fma_rn(Qa, Qb, -0.0);
        const double p2 = __fma_rn(p, r.B2, -P2);
        const double k = __fma_rn(q, r.kS, p2);
        if (st < 3) {
            tin = __dadd_rn(s, __dmul_rn(st == 2 ? c.h : c.hh, k));
            acc = st == 0 ? k : __fma_rn(k, 2.0, acc);
        } else {
            acc = __dadd_rn(acc, k);
            s = __dadd_rn(s, __dmul_rn(c.h6, acc));
        }
    }
}

// The same step with eight chains per warp (all 32 lanes carry variables, so
// no lane holds a constant): three shuffles per stage, and the operands that
// are a variable on some lanes and a constant on others are selected:
//   v = x: p = fma(Y, 1, -X), q = fma(W, 1, -0);  v = y: p = fma(X, rho, -0), p2 = fma(p, 1, -Y);
//   v = z: p = fma(Z, beta, -0), p2 = -p;          v = w: p = fma(W, gamma, -0);
// q = X Z, X Y, Y Z for y, z, w.  The first fma's shuffled operand is a factor
// on every lane and its addend a select on the lane's own value (-X or -0),
// so no select sits between the shuffles and the first fma.  Fewer binary64
// instructions per chain step (27 per eight chains), a longer step (selects).
struct LaneRole8 {
    double Pb, B2, kS;
    int s1, s2, s3;
    bool vx, vy;
};

__device__ __forceinline__ LaneRole8 lane_role8(int lane, double gamma) {
    LaneRole8 r;
    const int v = lane & 3, base = lane & ~3;
    r.Pb = v == 0 ? 1.0 : v == 1 ? kRho : v == 2 ? kBeta : gamma;
    r.B2 = v == 0 ? kSigma : v == 2 ? -1.0 : 1.0;
    r.kS = (v == 0 || v == 2) ? 1.0 : -1.0;
    r.s1 = base + (v == 0 ? 1 : v == 1 ? 0 : v);           // Y, X, Z, W
    r.s2 = base + (v == 0 ? 3 : v == 3 ? 1 : 0);           // W, X, X, Y
    r.s3 = base + ((v == 0 || v == 2) ? 1 : 2);            // Y, Z, Y, Z
    r.vx = v == 0;
    r.vy = v == 1;
    return r;
}

// `after_fetch(s)` runs once the first stage's operands are fetched, with the state at the start of the
// step: the worker kernel emits the previous step's stream bytes there, so that their integer work follows
// the shuffles that start this step instead of delaying them.
template <class F>
__device__ __forceinline__ void rk4_step_lanes8(double &s, const LaneRole8 &r, const Rk4 &c, F &&after_fetch) {
    double tin = s, acc = 0.0;
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        const double a = __shfl_sync(0xffffffffu, tin, r.s1);
        const double b = __shfl_sync(0xffffffffu, tin, r.s2);
        const double d = __shfl_sync(0xffffffffu, tin, r.s3);
        if (st == 0) after_fetch(tin);
        const double Pc = r.vx ? tin : 0.0;
        const double Qb = r.vx ? 1.0 : d;
        const double P2 = r.vy ? tin : 0.0;
        const double p = __fma_rn(a, r.Pb, -Pc);
        const double q = __fma_rn(b, Qb, -0.0);
        const double p2 = __fma_rn(p, r.B2, -P2);
        const double k = __fma_rn(q, r.kS, p2);
        if (st < 3) {
            tin = __dadd_rn(s, __dmul_rn(st == 2 ? c.h : c.hh, k));
            acc = st == 0 ? k : __fma_rn(k, 2.0, acc);
        } else {
            acc = __dadd_rn(acc, k);
            s = __dadd_rn(s, __dmul_rn(c.h6, acc));
        }
    }
}

// Integer-pipe operations of one lane without a vote: the fast path's result and, in `sp`, whether the
// lane needs the binary64 instruction instead.
__device__ __forceinline__ double lane_mul(double a, double b, bool &sp) {
    bool x;
    const uint64_t r = b64_mul((uint64_t)__double_as_longlong(a), (uint64_t)__double_as_longlong(b), x);
    sp = sp || x;
    return __longlong_as_double((long long)r);
}
__device__ __forceinline__ double lane_add(double a, double b, bool &sp) {
    bool x;
    const uint64_t r = b64_add((uint64_t)__double_as_longlong(a), (uint64_t)__double_as_longlong(b), x);
    sp = sp || x;
    return __longlong_as_double((long long)r);
}
// 2 k, exactly: one more in the exponent field while the double stays normal and finite.
__device__ __forceinline__ double lane_twice(double k, bool &sp) {
    const uint64_t K = (uint64_t)__double_as_longlong(k);
    sp = sp || ((uint32_t)(K >> 52) & 0x7ff) - 1 >= 0x7fd;
    return __longlong_as_double((long long)(K + (1ull << 52)));
}

// The eight-chain step with every rounded operation on the integer pipes (binary64_int.cuh): bit-identical
// to rk4_step_lanes8.  Each fused multiply-add of that step is split into its multiply and its add, which
// rounds the same way because in every use one of the two is exact: a factor of +-1 (Pb = 1, B2 = +-1,
// kS = +-1), a factor 2 (the combination), or an addend of -0.  The products by kS = +-1 are sign flips and
// the addends -0 after a rounded product are dropped (x + (-0) = x for every x the product can be, +0
// included).  The operations take no vote: a lane whose operands leave the integer fast path marks the
// step, and a marked step is done again, from its starting state, by rk4_step_lanes8 (one vote per step;
// the step's stream bytes, those of the state before it, are emitted once).
template <class F>
__device__ __forceinline__ void rk4_step_lanes8_int(double &s, const LaneRole8 &r, const Rk4 &c, F &&after_fetch) {
    const long long kneg = r.kS < 0.0 ? (long long)kSign : 0;
    const double s0 = s;
    bool sp = false;
    double tin = s, acc = 0.0;
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        const double a = __shfl_sync(0xffffffffu, tin, r.s1);
        const double b = __shfl_sync(0xffffffffu, tin, r.s2);
        const double d = __shfl_sync(0xffffffffu, tin, r.s3);
        if (st == 0) after_fetch(tin);
        const double Pc = r.vx ? tin : 0.0;
        const double Qb = r.vx ? 1.0 : d;
        const double P2 = r.vy ? tin : 0.0;
        const double p = lane_add(lane_mul(a, r.Pb, sp), -Pc, sp);
        const double q = lane_mul(b, Qb, sp);
        const double p2 = lane_add(lane_mul(p, r.B2, sp), -P2, sp);
        const double k = lane_add(__longlong_as_double(__double_as_longlong(q) ^ kneg), p2, sp);
        if (st < 3) {
            tin = lane_add(s, lane_mul(st == 2 ? c.h : c.hh, k, sp), sp);
            acc = st == 0 ? k : lane_add(acc, lane_twice(k, sp), sp);
        } else {
            acc = lane_add(acc, k, sp);
            s = lane_add(s, lane_mul(c.h6, acc, sp), sp);
        }
    }
    if (__any_sync(0xffffffffu, sp)) {
        s = s0;
        rk4_step_lanes8(s, r, c, [](double) {});
    }
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

// Reconstruct from (state, H), run LHCS_m 2n steps writing IR.  The chain
// lives in lanes 0..3 of the warp (lane = variable); s is this lane's value.
__device__ void master_frame(double &s, int lane, const LaneRole &role, const uint8_t *H_smem, const uint32_t *u,
                             uint32_t n, const Rk4 &c, double *IR) {
    if (lane < 4) s = reconstruct(s, H_smem + 8 * lane, u[lane]);
    __syncwarp();
    for (uint32_t t = 0; t < 2 * n; ++t) {
        rk4_step_lanes(s, role, c);
        if (lane < 4 && FHD_IN(4 * t + lane, 8ull * n, kSiteMasterIR)) IR[4 * t + lane] = s;
    }
}

// Mask of the transmitted digest (masked transport, an option of this library; Sec. V sends the hashes
// encrypted without giving the mechanism): M = SHA-256("FHDMASK1" || LE64(x) || LE64(y) || LE64(z) ||
// LE64(w) || LE64(gamma)) of the chaining state before the frame, 48 bytes in one block.  M is returned as
// the 8 little-endian words of its big-endian byte string, ready to XOR with the stored digest words.
__device__ void digest_mask(double x, double y, double z, double w, double gamma, uint32_t M[8]) {
    uint32_t wd[16];
    wd[0] = 0x4648444Du;   // "FHDM"
    wd[1] = 0x41534B31u;   // "ASK1"
    const double v[5] = {x, y, z, w, gamma};
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const unsigned long long bits = (unsigned long long)__double_as_longlong(v[m]);
        wd[2 + 2 * m] = __byte_perm((uint32_t)bits, 0, 0x0123);           // bytes 0..3, big-endian word
        wd[3 + 2 * m] = __byte_perm((uint32_t)(bits >> 32), 0, 0x0123);   // bytes 4..7
    }
    wd[12] = 0x80000000u;
    wd[13] = 0u;
    wd[14] = 0u;
    wd[15] = 48u * 8u;
    uint32_t h[8];
    sha256_init(h);
    sha256_compress(h, wd);
#pragma unroll
    for (int q = 0; q < 8; ++q) M[q] = __byte_perm(h[q], 0, 0x0123);
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

// Bytes of one step: the pair's XOR of the 6 low mantissa bytes of each
// variable; this lane writes its half (3 bytes) at stream position pos0 on.
// dlim and blim are the bytes of D and of B from Dbytes and Bp on (range checks of checked builds).
__device__ __forceinline__ void emit_bytes(double s, bool active, uint64_t pos0, uint64_t need, uint64_t ndb, int half,
                                           uint8_t *Dbytes, uint8_t *Bp, uint64_t dlim, uint64_t blim) {
    const unsigned long long mine = (unsigned long long)__double_as_longlong(s) & 0xffffffffffffull;
    const unsigned long long x = mine ^ __shfl_xor_sync(0xffffffffu, mine, 4);
    if (active && pos0 < need) {
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
            const uint64_t pos = pos0 + half + bb;
            const uint8_t byte = (uint8_t)(x >> (8 * (half + bb)));
            if (pos < ndb) {
                if (FHD_IN(pos, dlim, kSiteWorkerD)) Dbytes[pos] = byte;
            } else if (pos < need) {
                if (FHD_IN(pos - ndb, blim, kSiteWorkerB)) Bp[pos - ndb] = byte;
            }
        }
    }
}

// Worker pairs pg * kPairs .. pg * kPairs + kPairs - 1 of frame fd (Algorithm 2), run by one warp (lane = its
// lane): lane 4c + v holds variable v of chain c, chains 2q and 2q + 1 are pair q, so the partner of a lane
// is lane ^ 4.  Every warp of the frame runs the frame's uniform trip count (its longest slice).
template <int kPairs, bool kInt = false>
__device__ void keystream_warp(const FrameDesc &fd, uint32_t n, const Rk4 &c, uint32_t pg, int lane) {
    const int v = lane & 3, ch = lane >> 2;
    const uint32_t p = pg * kPairs + (ch >> 1);
    const bool active = lane < 8 * kPairs && p < n;
    const uint64_t LD = (uint64_t)fd.C * (fd.h + fd.w);
    const uint64_t LB = fd.N;
    WorkerSlice ws{0, 0, 0, 0};
    if (active) ws = worker_slice(LD, LB, n, p);
    const uint64_t need = 2 * ws.nd + ws.nb;
    // Uniform trip count: the longest slice of the frame.
    const uint64_t need_max = 2 * ((LD + n - 1) / n) + (LB + n - 1) / n;
    const uint64_t T = (need_max + 23) / 24;
    const uint32_t ir = 4 * (2 * p + (ch & 1)) + v;
    const double chain_value = active && FHD_IN(ir, 8ull * n, kSiteWorkerIR) ? __ldcg(fd.IR + ir) : 0.0;   // by LHCS_m
    uint8_t *Dbytes = reinterpret_cast<uint8_t *>(fd.D) + 2 * ws.d0;
    uint8_t *Bp = fd.B + ws.b0;
    const uint64_t ndb = 2 * ws.nd;
    const uint64_t dlim = 2 * LD - 2 * ws.d0, blim = LB - ws.b0;
    const int half = (ch & 1) * 3;
    if (kPairs == kPairsPerWarp) {
        const LaneRole role = lane_role(lane, fd.gamma);
        double s = lane_init(lane, chain_value);
        for (uint64_t t = 0; t < T; ++t) {
            rk4_step_lanes(s, role, c);
            emit_bytes(s, active, 24 * t + 6 * v, need, ndb, half, Dbytes, Bp, dlim, blim);
        }
    } else {
        // The bytes of step t (the state after it) are emitted during step t + 1, and the last step's after
        // the loop: the same bytes at the same positions.
        const LaneRole8 role = lane_role8(lane, fd.gamma);
        double s = chain_value;
        for (uint64_t t = 0; t < T; ++t) {
            auto emit = [&](double prev) {
                if (t) emit_bytes(prev, active, 24 * (t - 1) + 6 * v, need, ndb, half, Dbytes, Bp, dlim, blim);
            };
            if constexpr (kInt) rk4_step_lanes8_int(s, role, c, emit);
            else rk4_step_lanes8(s, role, c, emit);
        }
        if (T) emit_bytes(s, active, 24 * (T - 1) + 6 * v, need, ndb, half, Dbytes, Bp, dlim, blim);
    }
}

// ---- One-trajectory keystream route (traj_records in common.cuh).

__device__ __forceinline__ unsigned long long low48(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0xffffffffffffull;
}

// The records of one frame per chain of the warp, in the six-chain layout of LHCS_m (lane 4c + v holds
// variable v of chain c; lanes 24..31 hold the constants).  fd: this lane's frame (the four lanes of a chain
// share it), nullptr where the chain has none.  Steps k = 1, 2, ... take the state from s_k to s_{k+1}:
// while k < 2n it is LHCS_m's iterate IR[k], read back, and from k = 2n on one RK4 step.  After step k >= 2
// the warp writes record k - 2 = (s_k, s_{k+1}): the 48-bit XOR of each variable's two bit patterns (its six
// low mantissa bytes) is packed with the next variable's by one shuffle, and lanes v = 0, 1, 2 store the
// record's three 64-bit words.  A chain is strictly sequential, so its time is the number of steps times the
// step's latency (27 binary64 instructions back to back, plus the hand-offs); the warp runs to its longest
// frame.  All 32 lanes call it together.
__device__ void trajectory_warp(const FrameDesc *fd, uint32_t n, const Rk4 &c, int lane) {
    const int v = lane & 3;
    const bool active = fd != nullptr && lane < 4 * kChainsPerWarp;
    uint64_t R = 0;
    double gamma = 0.0;
    const double *IR = nullptr;
    uint64_t *rec = nullptr;
    if (active) {
        R = traj_records((uint64_t)fd->C * (fd->h + fd->w), fd->N, n);
        gamma = fd->gamma;
        IR = fd->IR;
        rec = reinterpret_cast<uint64_t *>(fd->T);
    }
    unsigned long long Rmax = R;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, Rmax, o);
        Rmax = t > Rmax ? t : Rmax;
    }
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

__device__ __forceinline__ uint32_t word8(const uint4 &a, const uint4 &b, uint32_t i) {
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

// Worker slice i's D bytes from the records (byte q of them is record byte 48 i + q), by threads tid of
// nthreads.
__device__ void emit_d_slice(const FrameDesc &fd, uint32_t n, uint32_t i, const WorkerSlice &ws, uint32_t tid,
                             uint32_t nthreads) {
    const uint64_t LD = (uint64_t)fd.C * (fd.h + fd.w);
    const uint64_t tlim = traj_bytes(LD, fd.N, n), s0 = 48ull * i;
    uint8_t *Db = reinterpret_cast<uint8_t *>(fd.D);
    for (uint64_t q = tid; q < 2 * ws.nd; q += nthreads) {
        const uint8_t byte = FHD_IN(s0 + q, tlim, kSiteEmitLoad) ? fd.T[s0 + q] : 0;
        if (FHD_IN(2 * ws.d0 + q, 2 * LD, kSiteEmitStore)) Db[2 * ws.d0 + q] = byte;
    }
}

// B[lo, hi) inside worker slice i (B[b0 + m] is record byte 48 i + 2 nd + m), by threads tid of nthreads in
// 16-byte chunks of B: a chunk inside [lo, hi) is one 16-byte store of bytes o .. o + 15 of two aligned
// 16-byte record loads (o = the source offset mod 16, the same for the whole slice); the chunks at the ends
// of [lo, hi), and every chunk of a B that is not 16-byte aligned, go byte by byte.
__device__ void emit_b_part(const FrameDesc &fd, uint32_t n, uint32_t i, const WorkerSlice &ws, uint64_t lo,
                            uint64_t hi, uint32_t tid, uint32_t nthreads) {
    const uint64_t LD = (uint64_t)fd.C * (fd.h + fd.w), LB = fd.N;
    const uint64_t tlim = traj_bytes(LD, LB, n);
    const uint8_t *T = fd.T;
    uint8_t *B = fd.B;
    const uint64_t sb = 48ull * i + 2 * ws.nd;   // record byte of B[b0]
    const bool aligned = (reinterpret_cast<uintptr_t>(B) & 15) == 0;
    const uint32_t o = (uint32_t)((sb - ws.b0) & 15), q = o >> 2, r = 8 * (o & 3);
    const uint64_t c_hi = (hi + 15) >> 4;
    for (uint64_t cidx = (lo >> 4) + tid; cidx < c_hi; cidx += nthreads) {
        const uint64_t p0 = 16 * cidx;
        if (aligned && p0 >= lo && p0 + 16 <= hi) {
            const uint64_t sp = sb + (p0 - ws.b0);   // sp mod 16 = o
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
                const uint64_t sp = sb + (p - ws.b0);
                const uint8_t byte = FHD_IN(sp, tlim, kSiteEmitLoad) ? T[sp] : 0;
                if (FHD_IN(p, LB, kSiteEmitStore)) B[p] = byte;
            }
        }
    }
}

// LHCS_m of stream group g of a batch (Algorithm 1), one warp (lane = its lane), the group's frames in call
// order: reconstruct from the chaining state and the frame's digest, 2n RK4 steps into the frame's IR, and
// chain on.  before(f) runs on every lane before frame f and may refuse it (false ends the group and keeps
// the state of the frames done); after(f) runs once frame f's iterates are written.  H is 32 bytes of
// shared memory of this warp.
template <class BatchT, class Before, class After>
__device__ void master_stream(const BatchT &b, uint32_t g, StreamState *states, unsigned *status, uint8_t *H,
                              int lane, Before before, After after) {
    const Rk4 c{b.hstep, b.hhalf, b.hsixth};
    const uint32_t first = b.group_begin[g], last = b.group_begin[g + 1];
    const uint32_t slot = b.f[b.order[first]].slot;
    StreamState *st = states + slot;
    const double gamma = b.f[b.order[first]].gamma;
    const LaneRole role = lane_role(lane, gamma);
    double s = lane_init(lane, lane < 4 ? st->v[lane] : 0.0);
    uint32_t done = 0;
    for (uint32_t k = first; k < last; ++k) {
        if (!FHD_IN(b.order[k], b.count, kSiteMasterFrame)) break;
        const FrameDesc &fd = b.f[b.order[k]];
        if (!before(b.order[k])) break;   // a dependency of the frame did not arrive (a bounded wait gave up)
        if (lane < 8)   // the frame's digest: folded by the digest stage, or the transmitted one
            reinterpret_cast<uint32_t *>(H)[lane] = __ldcg(reinterpret_cast<const uint32_t *>(fd.digest) + lane);
        __syncwarp();
        if (b.digest_masked) {
            // Lanes 0..3 hold the chaining state before this frame.  Encryption transmits H xor M (the
            // keystream still derives from H); decryption unmasks the transmitted digest and leaves H in
            // the frame's digest for the receiver-side check.
            const double x = __shfl_sync(0xffffffffu, s, 0), y = __shfl_sync(0xffffffffu, s, 1);
            const double z = __shfl_sync(0xffffffffu, s, 2), w = __shfl_sync(0xffffffffu, s, 3);
            if (lane == 0) {
                uint32_t M[8];
                digest_mask(x, y, z, w, gamma, M);
                uint32_t *hw = reinterpret_cast<uint32_t *>(H);
                uint32_t *dg = reinterpret_cast<uint32_t *>(fd.digest);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t t = hw[q] ^ M[q];
                    if (b.encrypt) {
                        dg[q] = t;
                    } else {
                        hw[q] = t;
                        dg[q] = t;
                    }
                }
            }
            __syncwarp();
        }
        master_frame(s, lane, role, H, b.u, b.n, c, fd.IR);
        __syncwarp();
        ++done;
        after(b.order[k]);
    }
    if (lane < 4) {
        st->v[lane] = s;
        if (!finite(s)) atomicOr(status, kStatusNonFinite);
        if (lane == 0) st->frames += done;
    }
}

}  // namespace
}  // namespace fhd
