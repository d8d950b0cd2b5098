// Persistent batch kernel: every step of a batch of frames in one launch.
//
// A batch of one direction, or an encryption and the decryption of its ciphertexts (a round trip of the
// same frames through a sender's and a receiver's streams), runs as one kernel of one CTA per SM.  Each CTA
// carries three kinds of workers, each pulling tasks from its own device queue (an atomic counter over a
// task order fixed by the launch descriptor):
//   * warps 0 and 1: a digest pipeline (the producer/consumer SHA-256 of Sec. II-A, 32 sub-frame messages
//     per task, largest frames first); the pipeline that completes a frame's messages folds (Algorithm 1)
//     or tree-hashes them into the frame digest and publishes it;
//   * warps 2, 3 and 5: chain workers, one on each of sub-partitions 1-3, so that a chain has its
//     sub-partition's binary64 pipe, and its issue port, to itself; per frame, smallest first
//     (the order in which their digests arrive): the LHCS_m task of every stream whose earliest frame it
//     is (Algorithm 1), then the frame's keystream tasks (Algorithm 2, the two sides interleaved): with the
//     one-trajectory route one task per frame and side, the frame's trajectory records (traj_records in
//     common.cuh); with the worker pairs one per three pairs;
//   * warps 4 and 6-15: a permutation group of 352 threads with the CTA's large shared memory: per frame,
//     smallest first, the encryption's emission tasks (one-trajectory route: D and B from the records, in
//     runs of kEmitTaskBytes of B), row bands and column strips, then the decryption's emission tasks,
//     column strips and row bands (Sec. II-C, Algos 3-7, and the inverse).
// A task waits for its inputs on per-frame counters: LHCS_m for the frame digest (the decryption's for the
// encryption's LHCS_m of the same frame, which writes the transmitted digest), a keystream task for its
// frame's LHCS_m, an emission task for its frame's trajectory, an encrypting row band for the frame's
// keystream (the row shifts: its worker warps, or its emission tasks), an encrypting strip for the frame's
// row bands, a decrypting strip for its keystream and the ciphertext, a decrypting row band for the
// frame's strips.  Tasks are dequeued in an order in
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

// Warp roles by SM sub-partition (warp w runs on sub-partition w mod 4): the digest pipeline's consumer
// (warp 0) and producer (warp 1) on sub-partitions 0 and 1; the chain workers (warps 2, 3 and 5) on
// sub-partitions 2, 3 and 1, one each -- in a digest CTA they start only after its pipeline (below), so
// the integer-bound digest rounds never share an issue port with a binary64 chain; warps 4 and 6-15 form
// the permutation group.  Four warps per sub-partition leave each of them 128 registers (a
// sub-partition's register file holds 16K).
constexpr int kPWarps = 16;
constexpr int kPThreads = 32 * kPWarps;
constexpr int kShaConsumer = 0, kShaProducer = 1;
constexpr int kChainWarps = 3;   // warps 2, 3, 5
constexpr int kMemThreads = 32 * (kPWarps - 2 - kChainWarps);
__device__ __forceinline__ int chain_index(uint32_t warp) { return warp == 2 ? 0 : warp == 3 ? 1 : warp == 5 ? 2 : -1; }
__device__ __forceinline__ uint32_t mem_index(uint32_t warp) { return warp == 4 ? 0 : warp - 5; }   // warps 4, 6..15
constexpr unsigned kBarSha = 1, kBarMem = 2;
constexpr size_t kPFixedSmem = sizeof(ShaSmem) + 32 * kChainWarps + 64 + 16;   // + broadcast slots, flag
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

// Publish a task's results (the caller has fenced its, and its group's, writes before this): a release-add
// that also stamps *t with %globaltimer when this add brings the counter to `target`.
__device__ __forceinline__ void publish(unsigned *p, unsigned v, unsigned target, unsigned long long *t) {
    unsigned old;
    asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    if (old + v == target) *t = globaltimer();
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

// One digest task (32 sub-frame messages, frames in prio order) as a function of its own: its register
// allocation is then that of the pipeline alone.
__device__ __noinline__ void digest_task(const PLaunch &L, uint32_t task, uint32_t rtid, ShaSmem &sm) {
    const PSide &S = L.s[0];
    const uint32_t n = S.n;
    sha_pipeline(
        [&](uint32_t m, const uint8_t *&p, uint64_t &len, uint8_t *&out) {
            if (!FHD_IN(m / n, S.count, kSiteShaDigest) || !FHD_IN(L.prio[m / n], S.count, kSitePersistTask))
                return false;
            const FrameDesc &fd = S.f[L.prio[m / n]];
            const uint32_t i = m % n;
            const uint64_t lo = (uint64_t)(((unsigned __int128)fd.N * i) / n);
            const uint64_t hi = (uint64_t)(((unsigned __int128)fd.N * (i + 1)) / n);
            if (!FHD_IN(hi, fd.N + 1, kSiteShaMessage)) return false;
            p = fd.src + lo;
            len = hi - lo;
            out = fd.part + 32ull * i;
            return true;
        },
        S.count * n, task, rtid, kBarSha, sm);
}

// ---- digest pipeline (warps 0-1)
__device__ void digest_worker(const PLaunch &L, ShaSmem &sm, unsigned *slot) {
    const uint32_t rtid = (threadIdx.x >> 5) == kShaConsumer ? (threadIdx.x & 31) : 32 + (threadIdx.x & 31);
    const PSide &S = L.s[0];
    const uint32_t n = S.n, nmsg = S.count * n;
    for (;;) {
        if (rtid == 0) slot[0] = ld_acquire(&L.cnt->abort) ? L.sha_units : atomicAdd(&L.cnt->sha_next, 1u);
        bar_sync(kBarSha, 64);
        const uint32_t task = slot[0];
        bar_sync(kBarSha, 64);
        if (task >= L.sha_units) return;
        digest_task(L, task, rtid, sm);
        __threadfence();
        bar_sync(kBarSha, 64);
        if (rtid == 0) {
            // the frames this task's messages belong to: count them in, and the task that completes a
            // frame forms its digest
            const uint32_t m0 = 32 * task, m1 = min(m0 + 32, nmsg);
            for (uint32_t r = m0 / n; r * n < m1; ++r) {
                const uint32_t lo = max(m0, r * n), hi = min(m1, (r + 1) * n);
                const uint32_t f = L.prio[r];
                if (!FHD_IN(f, S.count, kSitePersistTask)) continue;
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
                if ((int)f != L.hold_frame) publish(&L.cnt->digest_ready[f], 1u, 1u, &L.cnt->t_digest[f]);
            }
        }
    }
}

// The chain workers' two task bodies as separate functions, so that their register allocation is their own
// and not that of the whole kernel (inlined into it, the worker loop was allocated with the permutation and
// digest code's pressure).
__device__ __noinline__ void keystream_task(const FrameDesc &fd, uint32_t n, const Rk4 &c, uint32_t pg, int lane) {
    keystream_warp<3>(fd, n, c, pg, lane);
}

// One-trajectory route: the frame's trajectory on chain 0 of the warp (lanes 0..3).
__device__ __noinline__ void trajectory_task(const FrameDesc &fd, uint32_t n, const Rk4 &c, int lane) {
    trajectory_warp(lane < 4 ? &fd : nullptr, n, c, lane);
}

// Emission task idx of a frame (one-trajectory route): B bytes [idx kEmitTaskBytes, (idx + 1) kEmitTaskBytes)
// from the records, slice by slice, and for idx 0 also every slice's D bytes.
__device__ void emit_task(const FrameDesc &fd, uint32_t n, uint32_t idx, uint32_t mtid) {
    const uint64_t LD = (uint64_t)fd.C * (fd.h + fd.w), LB = fd.N;
    if (idx == 0)
        for (uint32_t i = 0; i < n; ++i) emit_d_slice(fd, n, i, worker_slice(LD, LB, n, i), mtid, kMemThreads);
    const uint64_t lo = (uint64_t)idx * kEmitTaskBytes;
    const uint64_t hi = lo + kEmitTaskBytes < LB ? lo + kEmitTaskBytes : LB;
    if (lo >= hi) return;
    // the slice holding B[lo]: the largest i with floor(i LB / n) <= lo
    uint32_t i = (uint32_t)(((lo + 1) * n - 1) / LB);
    for (; i < n; ++i) {
        const WorkerSlice ws = worker_slice(LD, LB, n, i);
        if (ws.b0 >= hi) break;
        const uint64_t a = lo > ws.b0 ? lo : ws.b0, e = hi < ws.b0 + ws.nb ? hi : ws.b0 + ws.nb;
        if (a < e) emit_b_part(fd, n, i, ws, a, e, mtid, kMemThreads);
    }
}

// The same for the permutation group's task bodies (kind 4: an emission task).
__device__ __noinline__ void mem_task(uint32_t kind, const FrameDesc &fd, uint32_t n, uint32_t idx, uint8_t *smem,
                                      uint32_t mtid) {
    auto sync = [] { bar_sync(kBarMem, kMemThreads); };
    if (kind == 0) row_pass<true, true>(fd, idx, smem, mtid, kMemThreads, sync);
    else if (kind == 1) strip_pass<true, true>(fd, idx, smem, mtid, kMemThreads, sync);
    else if (kind == 2) strip_pass<false, true>(fd, idx, smem, mtid, kMemThreads, sync);
    else if (kind == 3) row_pass<false, true>(fd, idx, smem, mtid, kMemThreads, sync);
    else emit_task(fd, n, idx, mtid);
}

// ---- chain workers (warps 2-5): LHCS_m tasks, then worker warps
__device__ void chain_worker(const PLaunch &L, uint8_t *H) {
    const int lane = threadIdx.x & 31;
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
        // first every LHCS_m task (the groups in the order of their earliest frame, side 0 then side 1),
        // then per frame (smallest first) its keystream tasks, the sides interleaved
        if (task < L.chain_masters_total) {
            const uint32_t r = segment(L.chain_begin, L.s[0].count, task);
            const uint32_t f = L.mprio[r], side = task - L.chain_begin[r];
            if (!FHD_IN(f, L.s[0].count, kSitePersistTask) || !FHD_IN(side, L.sides, kSitePersistTask)) continue;
            const uint32_t g = L.chain_group[f];
            if (!FHD_IN(g, L.s[side].groups, kSitePersistTask)) continue;
            const PSide &S = L.s[side];
            master_stream(
                S, g, S.states, S.status, H, lane,
                [&](uint32_t fr) {
                    if (side == 0) return S.encrypt ? wait(&L.cnt->digest_ready[fr], 1u) : true;
                    return wait(&L.cnt->master_done[0][fr], 1u);   // the transmitted digest of the sender's frame
                },
                [&](uint32_t fr) {
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) publish(&L.cnt->master_done[side][fr], 1u, 1u, &L.cnt->t_master[side][fr]);
                });
        } else {
            const uint32_t per = L.sides * L.wpf, t2 = task - L.chain_masters_total, r = t2 / per;
            const uint32_t f = L.mprio[r], k = t2 - r * per, side = k / L.wpf, pg = k - side * L.wpf;
            if (!FHD_IN(r, L.s[0].count, kSitePersistTask) || !FHD_IN(f, L.s[0].count, kSitePersistTask) ||
                !FHD_IN(side, L.sides, kSitePersistTask))
                continue;
            const PSide &S = L.s[side];
            if (wait(&L.cnt->master_done[side][f], 1u)) {
                if (L.traj) trajectory_task(S.f[f], S.n, Rk4{S.hstep, S.hhalf, S.hsixth}, lane);
                else keystream_task(S.f[f], S.n, Rk4{S.hstep, S.hhalf, S.hsixth}, pg, lane);
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) publish(&L.cnt->ks_done[side][f], 1u, L.wpf, &L.cnt->t_ks[side][f]);
        }
    }
}

// ---- permutation group (warps 6-17)
__device__ void mem_worker(const PLaunch &L, uint8_t *smem, unsigned *slot) {
    const uint32_t mtid = 32 * mem_index(threadIdx.x >> 5) + (threadIdx.x & 31);
    auto sync = [] { bar_sync(kBarMem, kMemThreads); };
    const PSide &S0 = L.s[0];
    // The frame's keystream of one side is ready: its worker warps are done (worker pairs), or its emission
    // tasks (one-trajectory route).
    auto keystream_ready = [&](uint32_t side, uint32_t f) {
        return L.traj ? wait_geq(&L.cnt->emit_done[side][f], L.s[side].emits[f], L)
                      : wait_geq(&L.cnt->ks_done[side][f], L.wpf, L);
    };
    for (;;) {
        // kind: 0 row pass (encrypting), 1 column pass (encrypting), 2 column pass (decrypting), 3 row pass
        // (decrypting), 4 emission (one-trajectory route); side, frame and strip, band or emission index of
        // the task.  A frame's tasks, in queue order: encrypting: emissions (they read the frame's
        // trajectory), row bands (they read the row shifts of the keystream), column strips (the row-rotated
        // frame); decrypting: emissions, column strips (its keystream, and the ciphertext), row bands (the
        // strips).
        if (mtid == 0) {
            const uint32_t t = ld_acquire(&L.cnt->abort) ? L.mem_tasks : atomicAdd(&L.cnt->mem_next, 1u);
            uint32_t kind = 0, side = 0, f = 0, idx = 0, ok = 0;
            if (t < L.mem_tasks) {
                const uint32_t r = segment(L.memb_begin, S0.count, t);
                f = L.mprio[r];
                uint32_t o = t - L.memb_begin[r];
                const bool emit0 = o < S0.emits[f];
                if (!emit0) o -= S0.emits[f];
                if (emit0) {
                    kind = 4;
                    idx = o;
                    ok = wait_geq(&L.cnt->ks_done[0][f], L.wpf, L);
                } else if (S0.encrypt) {
                    if (o < S0.bands[f]) {
                        idx = o;
                        ok = keystream_ready(0, f);
                    } else if ((o -= S0.bands[f]) < S0.strips[f]) {
                        kind = 1;
                        idx = o;
                        ok = wait_geq(&L.cnt->rows_done[0][f], S0.bands[f], L);
                    } else {
                        o -= S0.strips[f];
                        side = 1;
                        if (o < L.s[1].emits[f]) {
                            kind = 4;
                            idx = o;
                            ok = wait_geq(&L.cnt->ks_done[1][f], L.wpf, L);
                        } else if ((o -= L.s[1].emits[f]) < L.s[1].strips[f]) {
                            kind = 2;
                            idx = o;
                            ok = keystream_ready(1, f) && wait_geq(&L.cnt->strips_done[0][f], S0.strips[f], L);
                        } else {
                            kind = 3;
                            idx = o - L.s[1].strips[f];
                            ok = wait_geq(&L.cnt->strips_done[1][f], L.s[1].strips[f], L);
                        }
                    }
                } else if (o < S0.strips[f]) {
                    kind = 2;
                    idx = o;
                    ok = keystream_ready(0, f);
                } else {
                    kind = 3;
                    idx = o - S0.strips[f];
                    ok = wait_geq(&L.cnt->strips_done[0][f], S0.strips[f], L);
                }
            }
            slot[0] = t;
            slot[1] = kind | (side << 3) | (ok << 4);
            slot[2] = f;
            slot[3] = idx;
        }
        sync();
        const uint32_t t = slot[0], code = slot[1], f = slot[2], idx = slot[3];
        sync();
        if (t >= L.mem_tasks) return;
        const uint32_t kind = code & 7, side = (code >> 3) & 1;
        if (!FHD_IN(f, L.s[0].count, kSitePersistTask) || !FHD_IN(side, L.sides, kSitePersistTask) ||
            !FHD_IN(idx, kind == 4 ? L.s[side].emits[f] : kind == 0 || kind == 3 ? L.s[side].bands[f] : L.s[side].strips[f],
                    kSitePersistTask))
            continue;
        const FrameDesc &fd = L.s[side].f[f];
        if (code & 16) mem_task(kind, fd, L.s[side].n, idx, smem, mtid);
        __threadfence();
        sync();
        if (mtid == 0 && (code & 16)) {
            if (kind == 4)
                publish(&L.cnt->emit_done[side][f], 1u, L.s[side].emits[f], &L.cnt->t_emit[side][f]);
            else if (kind == 0 || kind == 3)
                publish(&L.cnt->rows_done[side][f], 1u, L.s[side].bands[f], &L.cnt->t_rows[side][f]);
            else
                publish(&L.cnt->strips_done[side][f], 1u, L.s[side].strips[f], &L.cnt->t_strips[side][f]);
        }
    }
}

// Digest CTAs: the first min(digest tasks, grid) CTAs run the digest pipelines, and their chain workers and
// permutation group start only once those pipelines have found the digest queue empty.  The digest rounds
// (integer work, shared-memory traffic) and binary64 chains slow each other down several times when they
// share an SM, so while the digests of the large frames run, the chains of the frames whose digests are
// done run on the other SMs; a digest CTA joins them when its last digest task ends.
__device__ bool wait_digest_cta(const PLaunch &L, volatile unsigned *flag) {
    const unsigned long long t0 = globaltimer();
    const unsigned long long cap = L.digest_wait_ns / 64 + 65536;
    for (unsigned long long it = 0; it < cap; ++it) {
        if (*flag) return true;
        if (ld_acquire(&L.cnt->abort)) return false;
        if (globaltimer() - t0 > L.digest_wait_ns) break;
        __nanosleep(256);
    }
    atomicOr(L.s[0].status, kStatusTimeout);
    if (L.sides > 1) atomicOr(L.s[1].status, kStatusTimeout);
    atomicExch(&L.cnt->abort, 1u);
    return false;
}

// 16 warps x 128 registers fill the SM's register file: one CTA per SM, and no spills in the task bodies.
__global__ void __maxnreg__(128) persistent_kernel(const __grid_constant__ PLaunch L) {
    extern __shared__ __align__(16) uint8_t smem[];
    ShaSmem &sm = *reinterpret_cast<ShaSmem *>(smem);
    uint8_t *H = smem + sizeof(ShaSmem);
    unsigned *slot = reinterpret_cast<unsigned *>(H + 32 * kChainWarps);   // [0] digest, [4..7] permutation,
    volatile unsigned *digest_cta_done = slot + 8;                          // [8] this CTA's digests finished
    uint8_t *mem = smem + kPFixedSmem;
    const uint32_t warp = threadIdx.x >> 5;
    const bool digest_cta = blockIdx.x < L.sha_units;
    if (threadIdx.x == 0) {
        *digest_cta_done = digest_cta ? 0u : 1u;
        if (blockIdx.x == 0) L.cnt->t0 = globaltimer();
    }
    __syncthreads();
    if (warp == kShaConsumer || warp == kShaProducer) {
        if (digest_cta) {
            digest_worker(L, sm, slot);
            if (threadIdx.x == 0) {
                __threadfence_block();
                *digest_cta_done = 1u;
            }
        }
    } else if (chain_index(warp) >= 0) {
        if (wait_digest_cta(L, digest_cta_done)) chain_worker(L, H + 32 * chain_index(warp));
    } else {
        if (wait_digest_cta(L, digest_cta_done)) mem_worker(L, mem, slot + 4);
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

FHD_BOUNDS_TAKER(take_bounds_persist)
