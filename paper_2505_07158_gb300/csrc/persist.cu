// Persistent batch kernel: every step of a batch of frames in one launch.
//
// A batch of one direction, or an encryption and the decryption of its ciphertexts (a round trip of the
// same frames through a sender's and a receiver's streams), runs as one kernel of one CTA per SM.  Each CTA
// carries three kinds of workers, each pulling tasks from its own device queue (an atomic counter over a
// task order fixed by the launch descriptor):
//   * warps 0-1: a digest pipeline (the producer/consumer SHA-256 of Sec. II-A, 32 sub-frame messages per
//     task, largest frames first); the pipeline that completes a frame's messages folds (Algorithm 1) or
//     tree-hashes them into the frame digest and publishes it;
//   * warps 2-5: chain workers, one per SM sub-partition, so that a chain has the sub-partition's binary64
//     pipe to itself: first the LHCS_m task of every stream (Algorithm 1), then the worker warps of every
//     frame (Algorithm 2, three worker pairs each, largest frames first, the two sides interleaved);
//   * warps 6-17: a permutation group of 384 threads with the CTA's large shared memory: per frame,
//     smallest first, the row bands and column strips of the encryption, then the decryption's column
//     strips and row bands (Sec. II-C, Algos 3-7, and the inverse).
// A task waits for its inputs on per-frame counters: LHCS_m for the frame digest (the decryption's for the
// encryption's LHCS_m of the same frame, which writes the transmitted digest), a worker warp for its frame's
// LHCS_m, an encrypting row band for the frame's keystream (the row shifts), an encrypting strip for the
// frame's row bands, a decrypting strip for its keystream and the ciphertext, a decrypting row band for
// the frame's strips.  Tasks are dequeued in an order in
// which every dependency of a task was dequeued before it, by a worker that does not wait on anything
// later, so the launch completes whatever number of its CTAs is resident.  Every wait is bounded: past the
// launch's time limit (%globaltimer, and an iteration cap as a second bound) the waiting task sets the
// timeout bit of the status words and an abort flag that ends every other wait and every queue at once;
// the kernel then returns with the batch unfinished, and cipher_sync_status reports FHD_ERR_TIMEOUT.
#include "chaos_dev.cuh"
#include "permute_dev.cuh"
#include "sha256_dev.cuh"

namespace fhd {
namespace {

constexpr int kPWarps = 18;
constexpr int kPThreads = 32 * kPWarps;
constexpr int kChainWarp0 = 2, kChainWarps = 4;
constexpr int kMemWarp0 = 6, kMemThreads = 32 * (kPWarps - kMemWarp0);
constexpr unsigned kBarSha = 1, kBarMem = 2;
constexpr size_t kPFixedSmem = sizeof(ShaSmem) + 32 * kChainWarps + 64;   // + broadcast slots
constexpr size_t kPSmemLimit = 232448;

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Publish a task's results: the caller has fenced its (and its group's) writes before this.
__device__ __forceinline__ void release_add(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void bar_sync(unsigned id, unsigned n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// Bounded wait until *p >= target.  False once the launch's limit has passed (the waiter then marks the
// timeout in both sides' status words and raises the abort flag) or another wait has given up.
__device__ bool wait_geq(const unsigned *p, unsigned target, const PLaunch &L) {
    if (ld_acquire(p) >= target) return true;
    const unsigned long long t0 = globaltimer();
    const unsigned long long cap = L.timeout_ns / 64 + 65536;   // a bound that does not rely on the clock
    for (unsigned long long it = 0; it < cap; ++it) {
        __nanosleep(128);
        if (ld_acquire(p) >= target) return true;
        if (ld_acquire(&L.cnt->abort)) return false;
        if (globaltimer() - t0 > L.timeout_ns) break;
    }
    atomicOr(L.s[0].status, kStatusTimeout);
    if (L.sides > 1) atomicOr(L.s[1].status, kStatusTimeout);
    atomicExch(&L.cnt->abort, 1u);
    return false;
}

// Largest k with a[k] <= v (a ascending, a[0] = 0, m + 1 entries).
__device__ __forceinline__ uint32_t segment(const uint32_t *a, uint32_t m, uint32_t v) {
    uint32_t lo = 0, hi = m;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid; else hi = mid;
    }
    return lo;
}

// ---- digest pipeline (warps 0-1)
__device__ void digest_worker(const PLaunch &L, ShaSmem &sm, unsigned *slot) {
    const uint32_t rtid = threadIdx.x;   // 0..63
    const PSide &S = L.s[0];
    const uint32_t n = S.n, nmsg = S.count * n;
    for (;;) {
        if (rtid == 0) slot[0] = ld_acquire(&L.cnt->abort) ? L.sha_units : atomicAdd(&L.cnt->sha_next, 1u);
        bar_sync(kBarSha, 64);
        const uint32_t task = slot[0];
        bar_sync(kBarSha, 64);
        if (task >= L.sha_units) return;
        sha_pipeline(
            [&](uint32_t m, const uint8_t *&p, uint64_t &len, uint8_t *&out) {
                const FrameDesc &fd = S.f[L.prio[m / n]];
                const uint32_t i = m % n;
                const uint64_t lo = (uint64_t)(((unsigned __int128)fd.N * i) / n);
                const uint64_t hi = (uint64_t)(((unsigned __int128)fd.N * (i + 1)) / n);
                p = fd.src + lo;
                len = hi - lo;
                out = fd.part + 32ull * i;
            },
            nmsg, task, rtid, kBarSha, sm);
        __threadfence();
        bar_sync(kBarSha, 64);
        if (rtid == 0) {
            // the frames this task's messages belong to: count them in, and the task that completes a
            // frame forms its digest
            const uint32_t m0 = 32 * task, m1 = min(m0 + 32, nmsg);
            for (uint32_t r = m0 / n; r * n < m1; ++r) {
                const uint32_t lo = max(m0, r * n), hi = min(m1, (r + 1) * n);
                const uint32_t f = L.prio[r];
                const unsigned old = atomicAdd(&L.cnt->sha_msgs[f], hi - lo);
                if (old + (hi - lo) != n) continue;
                __threadfence();
                const FrameDesc &fd = S.f[f];
                uint32_t h[8];
                if (S.digest_mode == FHD_DIGEST_TREE) {
                    tree_digest(fd.part, n, h);
                    store_digest(fd.digest, h);
                } else {
                    const uint32_t *pp = reinterpret_cast<const uint32_t *>(fd.part);
                    uint32_t *dg = reinterpret_cast<uint32_t *>(fd.digest);
                    for (int q = 0; q < 8; ++q) {
                        uint32_t acc = 0;
                        for (uint32_t i = 0; i < n; ++i) acc ^= __ldcg(pp + 8 * i + q);   // other pipelines' digests
                        dg[q] = acc;
                    }
                }
                __threadfence();
                if ((int)f != L.hold_frame) release_add(&L.cnt->digest_ready[f], 1u);
            }
        }
    }
}

// ---- chain workers (warps 2-5): LHCS_m tasks, then worker warps
__device__ void chain_worker(const PLaunch &L, uint8_t *H) {
    const int lane = threadIdx.x & 31;
    const uint32_t G0 = L.s[0].groups, G1 = L.sides > 1 ? L.s[1].groups : 0;
    // One lane waits; the warp learns the outcome.
    auto wait = [&](const unsigned *p, unsigned target) {
        int ok = 1;
        if (lane == 0) ok = wait_geq(p, target, L) ? 1 : 0;
        return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };
    for (;;) {
        uint32_t task = 0;
        if (lane == 0) task = ld_acquire(&L.cnt->abort) ? L.chain_tasks : atomicAdd(&L.cnt->chain_next, 1u);
        task = __shfl_sync(0xffffffffu, task, 0);
        if (task >= L.chain_tasks) return;
        if (task < G0 + G1) {
            const uint32_t side = task < G0 ? 0 : 1, g = side ? task - G0 : task;
            const PSide &S = L.s[side];
            master_stream(
                S, g, S.states, S.status, H, lane,
                [&](uint32_t f) {
                    if (side == 0) return S.encrypt ? wait(&L.cnt->digest_ready[f], 1u) : true;
                    return wait(&L.cnt->master_done[0][f], 1u);   // the transmitted digest of the sender's frame
                },
                [&](uint32_t f) {
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) release_add(&L.cnt->master_done[side][f], 1u);
                });
        } else {
            const uint32_t k = task - G0 - G1, per = L.sides * L.wpf;
            const uint32_t r = k / per, rem = k - r * per, side = rem / L.wpf, pg = rem - side * L.wpf;
            const uint32_t f = L.prio[r];
            const PSide &S = L.s[side];
            if (wait(&L.cnt->master_done[side][f], 1u))
                keystream_warp<3>(S.f[f], S.n, Rk4{S.hstep, S.hhalf, S.hsixth}, pg, lane);
            __threadfence();
            __syncwarp();
            if (lane == 0) release_add(&L.cnt->ks_done[side][f], 1u);
        }
    }
}

// ---- permutation group (warps 6-17)
__device__ void mem_worker(const PLaunch &L, uint8_t *smem, unsigned *slot) {
    const uint32_t mtid = threadIdx.x - 32 * kMemWarp0;
    auto sync = [] { bar_sync(kBarMem, kMemThreads); };
    const PSide &S0 = L.s[0];
    for (;;) {
        // kind: 0 row pass (encrypting), 1 column pass (encrypting), 2 column pass (decrypting), 3 row pass
        // (decrypting); side, frame and strip or band index of the task.  A frame's tasks, in queue order:
        // encrypting: row bands (they read the row shifts of the keystream), column strips (the row-rotated
        // frame); decrypting: column strips (its keystream, and the ciphertext), row bands (the strips).
        if (mtid == 0) {
            const uint32_t t = ld_acquire(&L.cnt->abort) ? L.mem_tasks : atomicAdd(&L.cnt->mem_next, 1u);
            uint32_t kind = 0, side = 0, f = 0, idx = 0, ok = 0;
            if (t < L.mem_tasks) {
                const uint32_t r = segment(L.memb_begin, S0.count, t);
                f = L.mprio[r];
                uint32_t o = t - L.memb_begin[r];
                if (S0.encrypt) {
                    if (o < S0.bands[f]) {
                        idx = o;
                        ok = wait_geq(&L.cnt->ks_done[0][f], L.wpf, L);
                    } else if ((o -= S0.bands[f]) < S0.strips[f]) {
                        kind = 1;
                        idx = o;
                        ok = wait_geq(&L.cnt->rows_done[0][f], S0.bands[f], L);
                    } else {
                        o -= S0.strips[f];
                        side = 1;
                        if (o < L.s[1].strips[f]) {
                            kind = 2;
                            idx = o;
                            ok = wait_geq(&L.cnt->ks_done[1][f], L.wpf, L) &&
                                 wait_geq(&L.cnt->strips_done[0][f], S0.strips[f], L);
                        } else {
                            kind = 3;
                            idx = o - L.s[1].strips[f];
                            ok = wait_geq(&L.cnt->strips_done[1][f], L.s[1].strips[f], L);
                        }
                    }
                } else if (o < S0.strips[f]) {
                    kind = 2;
                    idx = o;
                    ok = wait_geq(&L.cnt->ks_done[0][f], L.wpf, L);
                } else {
                    kind = 3;
                    idx = o - S0.strips[f];
                    ok = wait_geq(&L.cnt->strips_done[0][f], S0.strips[f], L);
                }
            }
            slot[0] = t;
            slot[1] = kind | (side << 2) | (ok << 3);
            slot[2] = f;
            slot[3] = idx;
        }
        sync();
        const uint32_t t = slot[0], code = slot[1], f = slot[2], idx = slot[3];
        sync();
        if (t >= L.mem_tasks) return;
        const uint32_t kind = code & 3, side = (code >> 2) & 1;
        const FrameDesc &fd = L.s[side].f[f];
        if (code & 8) {
            if (kind == 0) row_pass<true, true>(fd, idx, smem, mtid, kMemThreads, sync);
            else if (kind == 1) strip_pass<true, true>(fd, idx, smem, mtid, kMemThreads, sync);
            else if (kind == 2) strip_pass<false, true>(fd, idx, smem, mtid, kMemThreads, sync);
            else row_pass<false, true>(fd, idx, smem, mtid, kMemThreads, sync);
        }
        __threadfence();
        sync();
        if (mtid == 0 && (code & 8)) {
            unsigned *c = kind == 0 || kind == 3 ? &L.cnt->rows_done[side][f] : &L.cnt->strips_done[side][f];
            release_add(c, 1u);
        }
    }
}

__global__ void __launch_bounds__(kPThreads, 1) persistent_kernel(const __grid_constant__ PLaunch L) {
    extern __shared__ __align__(16) uint8_t smem[];
    ShaSmem &sm = *reinterpret_cast<ShaSmem *>(smem);
    uint8_t *H = smem + sizeof(ShaSmem);
    unsigned *slot = reinterpret_cast<unsigned *>(H + 32 * kChainWarps);   // [0] digest, [4..7] permutation
    uint8_t *mem = smem + kPFixedSmem;
    const uint32_t warp = threadIdx.x >> 5;
    if (warp < kChainWarp0) {
        if (L.sha_units) digest_worker(L, sm, slot);
    } else if (warp < kMemWarp0) {
        chain_worker(L, H + 32 * (warp - kChainWarp0));
    } else {
        mem_worker(L, mem, slot + 4);
    }
}

}  // namespace

size_t persistent_mem_smem_limit() { return kPSmemLimit - kPFixedSmem; }

cudaError_t launch_persistent(const PLaunch &L, size_t mem_smem, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = kPFixedSmem + mem_smem;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPSmemLimit);
    if (e != cudaSuccess) return e;
    persistent_kernel<<<sms, kPThreads, smem, s>>>(L);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fhd
