// Internal declarations shared by the CUDA translation units of libfhdcipher.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fhdcipher.h"

namespace fhd {

// Frames per launch: the per-frame descriptors travel as a kernel parameter
// (well under the 32 KB parameter limit of sm_70+ with CUDA 12.1+).
constexpr int kMaxBatch = 256;

// Per-frame launch descriptor.  All pointers are device pointers.
struct FrameDesc {
    const uint8_t *src;
    uint8_t *dst;
    uint8_t *digest;   // 32 bytes: written by encrypt (H), read by decrypt
    uint8_t *B;        // N bytes of XOR keystream (scratch)
    uint16_t *D;       // C*(h+w) shift distances (scratch)
    double *IR;        // 2n x 4 iterates of LHCS_m (scratch)
    uint8_t *part;     // n x 32 sub-frame digests (scratch)
    uint8_t *G;        // N bytes: frame between the row and the column pass (scratch)
    uint8_t *T;        // trajectory records of the one-trajectory keystream route (scratch, traj_bytes)
    uint64_t N;        // h*w*C
    double gamma;      // control parameter of the frame's stream
    uint32_t h, w, C;
    uint32_t slot;     // index of the stream's chaining state
    uint32_t P;        // strip width in pixels of the column pass
    uint32_t cta0;     // first column-pass CTA of this frame
    uint32_t RB;       // rows per CTA of the row pass
    uint32_t rcta0;    // first row-pass CTA of this frame
};

struct Batch {
    uint32_t count;
    uint32_t n;               // worker pairs / sub-frames per frame
    uint32_t groups;          // streams in this batch (master CTAs)
    uint32_t perm_ctas;       // total column-pass CTAs
    uint32_t row_ctas;        // total row-pass CTAs
    uint32_t digest_mode;     // FHD_DIGEST_XOR (the paper's fold) or FHD_DIGEST_TREE
    uint32_t digest_masked;   // transmitted digest is H xor M (FHD_TRANSPORT_MASKED)
    uint32_t encrypt;         // 1: this batch encrypts (LHCS_m masks the digest), 0: decrypts (unmasks)
    uint32_t int_mix;         // eight-chain worker warps per 8 that step on the integer pipes (0..8)
    double hstep, hhalf, hsixth;   // RK4 step h, h/2 and h/6 (rounded once, on the host)
    uint32_t u[4];            // reconstruction bounds
    uint16_t order[kMaxBatch];          // frame indices grouped by stream, in call order
    uint16_t group_begin[kMaxBatch + 1];
    FrameDesc f[kMaxBatch];
};

// One-trajectory keystream route (chaos.cu).  Worker pair i starts from the LHCS_m iterates IR[2i] and
// IR[2i+1] and iterates the same map with the same step (Algorithm 2), so its two systems are the frame's
// LHCS_m trajectory continued: with s_t the state after t steps from the reconstructed initial condition
// (IR[t-1] = s_t), step k of pair i yields the stream bytes of s_{2i+1+k} xor those of s_{2i+2+k}.  Record r
// of the frame is that 24-byte XOR for s_{r+2} and s_{r+3}; worker i's byte stream is the records from byte
// 48 i on.  traj_records is the number of records the frame's n workers read (a bound: the longest slice
// plus the offset of the last worker), traj_bytes the scratch they take with the emission's over-read.
__host__ __device__ inline uint64_t traj_records(uint64_t LD, uint64_t LB, uint32_t n) {
    const uint64_t need = 2 * ((LD + n - 1) / n) + (LB + n - 1) / n;
    return (48ull * (n - 1) + need + 23) / 24;
}
__host__ __device__ inline uint64_t traj_bytes(uint64_t LD, uint64_t LB, uint32_t n) {
    return 24 * traj_records(LD, LB, n) + 64;
}
// B bytes per emission task of a persistent launch (a multiple of 16; the frame's task 0 also writes D).
constexpr uint64_t kEmitTaskBytes = 180224;

// ---- Persistent batch launch (persist.cu): one kernel pulls the digest, chaining, worker and permutation
// tasks of a batch -- of one direction, or of an encryption and the decryption of its ciphertext -- from
// device queues with per-frame dependency counters.
constexpr int kPMax = 64;   // frames per side

// One direction of a persistent launch.  The fields master_stream reads have the names of Batch's.
struct PSide {
    uint32_t count, n, groups;
    uint32_t digest_mode, digest_masked, encrypt;
    double hstep, hhalf, hsixth;
    uint32_t u[4];
    uint16_t order[kPMax];
    uint16_t group_begin[kPMax + 1];
    uint32_t strips[kPMax];   // column-pass strips of frame k
    uint32_t bands[kPMax];    // row-pass bands of frame k
    uint32_t emits[kPMax];    // emission tasks of frame k (one-trajectory route; 0 with the worker pairs)
    struct StreamState *states;
    unsigned *status;
    FrameDesc f[kPMax];
};

// Dependency counters and queue heads of one launch (device memory, zeroed before it).
struct PCounters {
    unsigned sha_next, chain_next, mem_next, abort;
    unsigned sha_msgs[kPMax];          // side 0 (encrypting): sub-frame messages hashed, per frame
    unsigned digest_ready[kPMax];      // side 0: frame digest written
    unsigned master_done[2][kPMax];    // LHCS_m iterates of the frame written
    unsigned ks_done[2][kPMax];        // worker warps of the frame done
    unsigned rows_done[2][kPMax];      // row-pass bands of the frame done
    unsigned strips_done[2][kPMax];    // column-pass strips of the frame done
    unsigned emit_done[2][kPMax];      // emission tasks of the frame done (one-trajectory route)
    // %globaltimer at the launch's start and when each of the counters above reached its target
    // (instrumentation: cipher_persistent_trace)
    unsigned long long t0;
    unsigned long long t_digest[kPMax];
    unsigned long long t_master[2][kPMax], t_ks[2][kPMax], t_rows[2][kPMax], t_strips[2][kPMax];
    unsigned long long t_emit[2][kPMax];
};

struct PLaunch {
    uint32_t sides;            // 1: one direction; 2: side 0 encrypts, side 1 decrypts side 0's ciphertexts
    uint32_t traj;             // 1: the one-trajectory route (a frame's keystream task is its trajectory,
                               // then emission tasks in the permutation queue); 0: worker pairs
    uint32_t wpf;              // keystream tasks per frame: worker warps (three worker pairs each), or 1
    uint32_t sha_units;        // digest pipelines of side 0 when it encrypts (32 messages each), else 0
    uint32_t chain_tasks;      // the LHCS_m tasks, then per frame (mprio order) its worker warps
    uint32_t chain_masters_total;
    uint32_t mem_tasks;
    uint32_t prio[kPMax];      // frame indices by decreasing size: digest and worker order
    uint32_t mprio[kPMax];     // frame indices by increasing size: permutation order
    uint32_t memb_begin[kPMax + 1];   // permutation queue: first task of each frame (mprio order)
    uint32_t chain_begin[kPMax + 1];  // chain queue: first LHCS_m task of the groups starting at each frame
    uint16_t chain_masters[kPMax];    // LHCS_m tasks of the stream group whose earliest frame is f (0, 1 or 2)
    uint16_t chain_group[kPMax];      // that stream group
    unsigned long long timeout_ns;    // limit of every dependency wait
    unsigned long long digest_wait_ns;   // limit of a digest CTA's other workers' wait for its digest pipeline
    int hold_frame;            // test hook: side 0's digest of this frame is never published (-1: none)
    PCounters *cnt;
    PSide s[2];
};

cudaError_t launch_persistent(const PLaunch &L, size_t mem_smem, cudaStream_t s);
size_t persistent_mem_smem_limit();   // shared memory the permutation tasks of a persistent launch may use

// Chaining state of one video stream (Sec. II-A): x, y, z, w, gamma, frames done.
struct StreamState {
    double v[4];
    double gamma;
    unsigned long long frames;
};
static_assert(sizeof(StreamState) == FHD_STATE_BYTES, "state layout");

// Device status word bits (cipher_sync_status).
enum : unsigned {
    kStatusNonFinite = 1u << 0,  // a chaotic state became NaN/Inf
    kStatusTimeout = 1u << 1,    // a bounded wait gave up
    kStatusBounds = 1u << 2,     // a bounds check failed (checked builds)
};

// Bounds record of a checked build (-DFHD_BOUNDS_CHECK; bounds.cuh): how many accesses failed their range
// check, and the first one's site, index and extent.  Each translation unit with kernels keeps its own.
struct BoundsRecord {
    unsigned count, site;
    unsigned long long index, limit;
};

// Sites of the range checks (the buffer and the access that failed).
enum : unsigned {
    kSiteShaMessage = 1,     // a sub-frame message outside its frame
    kSiteShaBlock = 2,       // a message block load past the message
    kSiteShaDigest = 3,      // a sub-frame digest slot past the frame's n slots, or a frame index past the batch
    kSiteMasterIR = 10,      // an LHCS_m iterate past the frame's 2n x 4
    kSiteMasterFrame = 11,   // a stream group's frame index past the batch
    kSiteWorkerIR = 12,      // a worker chain's initial value past the frame's iterates
    kSiteWorkerD = 13,       // a shift-distance byte past C (h + w) entries
    kSiteWorkerB = 14,       // an XOR byte past the frame
    kSiteTrajIR = 15,        // trajectory: an LHCS_m iterate past the frame's 2n x 4
    kSiteTrajRecord = 16,    // trajectory: a record past the frame's traj_records
    kSiteEmitLoad = 17,      // emission: a record byte past the frame's traj_bytes
    kSiteEmitStore = 18,     // emission: a D byte past 2 C (h + w) or a B byte past the frame
    kSiteRowLoad = 20,       // row pass: frame (F or G) load
    kSiteRowShift = 21,      // row pass: row shift distance (D) load
    kSiteRowSmem = 22,       // row pass: shared-memory band or shift table
    kSiteRowStore = 23,      // row pass: frame (G or output) store
    kSiteStripShift = 30,    // column pass: column shift distance (D) load
    kSiteStripLoad = 31,     // column pass: frame (G or E) or B load
    kSiteStripSmem = 32,     // column pass: shared-memory strip
    kSiteStripStore = 33,    // column pass: frame store
    kSiteGatherShift = 40,   // single pass: shift distance or rotation table
    kSiteGatherLoad = 41,    // single pass: F load
    kSiteGatherSmem = 42,    // single pass: staging buffer or strip
    kSiteGatherStore = 43,   // single pass: B load or E store
    kSitePersistTask = 50,   // persistent launch: a task's frame, side or index outside the launch
    kSiteStats = 60,         // statistics: a frame load past the batch
};
const char *bounds_site_name(unsigned site);

// Read and clear the bounds record of each translation unit with kernels, added into *acc (the first
// violation kept is the first unit's).  Without FHD_BOUNDS_CHECK they add nothing.
cudaError_t take_bounds_sha(BoundsRecord *acc);
cudaError_t take_bounds_chaos(BoundsRecord *acc);
cudaError_t take_bounds_permute(BoundsRecord *acc);
cudaError_t take_bounds_persist(BoundsRecord *acc);
cudaError_t take_bounds_stats(BoundsRecord *acc);

// Launchers (one per kernel family); each returns the launch error.
cudaError_t launch_sha_subframes(const Batch &b, cudaStream_t s);
cudaError_t launch_verify(const Batch &b, uint8_t *ok, cudaStream_t s);   // ok[f.slot] per frame
cudaError_t launch_sha_plain(const uint8_t *data, uint64_t nbytes, uint32_t n, uint32_t count,
                             uint8_t *part, cudaStream_t s);
cudaError_t launch_fold(const uint8_t *part, uint32_t n, uint32_t count, uint8_t *digest, cudaStream_t s);
cudaError_t launch_tree_batch(const Batch &b, cudaStream_t s);
cudaError_t launch_tree(const uint8_t *part, uint32_t n, uint32_t count, uint8_t *digest, cudaStream_t s);
cudaError_t launch_fold_batch(const Batch &b, cudaStream_t s);
// Counts one kernel launch of this library (read by fhd_launch_count).
void note_launch();

// Frame statistics (stats.cu); frames are a contiguous batch [count][h][w][C].
cudaError_t launch_stats_histogram(const uint8_t *frames, uint32_t count, uint64_t frame_bytes, uint32_t C,
                                   unsigned long long *hist64, uint32_t *hist32, double *out, cudaStream_t s);
cudaError_t launch_stats_npcr(const uint8_t *a, const uint8_t *b, uint32_t count, uint64_t frame_bytes, uint32_t C,
                              uint64_t wh, unsigned long long *acc, double *out, cudaStream_t s);
cudaError_t launch_stats_correlation(const uint8_t *frames, uint32_t count, uint32_t h, uint32_t w, uint32_t C,
                                     const uint32_t *pairs, uint32_t npairs, long long *sums, double *out,
                                     unsigned *status, cudaStream_t s);
cudaError_t launch_stats_local_entropy(const uint8_t *frames, uint32_t count, uint32_t h, uint32_t w, uint32_t C,
                                       const uint32_t *blocks, uint32_t k, uint32_t bs, double *ent, double *out,
                                       unsigned *status, cudaStream_t s);
cudaError_t noalloc_scratch(uint8_t **out);   // fixed sub-frame digest array of fhd_frame_digest_noalloc
uint32_t noalloc_max_digests();
cudaError_t launch_master(const Batch &b, StreamState *states, unsigned *status, cudaStream_t s);
cudaError_t launch_master_raw(double *state5, const uint8_t *H, uint32_t n, double hstep, const uint32_t u[4],
                              double *IR, unsigned *status, cudaStream_t s);
// smem: dynamic shared memory each worker CTA requests (unused by the kernel: it caps the worker CTAs an SM
// holds at once).
cudaError_t launch_keystream(const Batch &b, cudaStream_t s, bool dense = false, uint32_t warps_per_cta = 1,
                             uint32_t smem = 0);
cudaError_t launch_permute(const Batch &b, bool encrypt, cudaStream_t s);
// The one-trajectory route: every frame's records (one chain per frame, six frames per warp), then D and B
// from them.  Each frame needs f.T (traj_bytes).
cudaError_t launch_trajectory_keystream(const Batch &b, cudaStream_t s);
int set_keystream_route(int route);   // FHD_KS_ROUTE_TRAJECTORY or FHD_KS_ROUTE_PAIRS; -1 on a bad value
int keystream_route();

// Geometry of the permutation passes: strip width (column pass) and rows per
// CTA (row pass), and their dynamic shared memory.
uint32_t strip_width(uint32_t h, uint32_t w, uint32_t C);
size_t strip_smem_bytes(uint32_t h, uint32_t P, uint32_t C);
uint32_t permute_strips(uint32_t w, uint32_t P);
uint32_t row_band(uint32_t h, uint32_t w, uint32_t C);
size_t row_smem_bytes(uint32_t w, uint32_t C, uint32_t RB);
cudaError_t permute_prepare();   // opt in to large dynamic shared memory
// Binary64 pipe probe (probe.cu): one CTA of 4 * warps_per_subpartition warps per SM; *lane_ops = binary64
// lane-operations the launch executes.
cudaError_t launch_fp64_probe(uint32_t warps_per_subpartition, uint32_t iters, double *sink, uint64_t *lane_ops,
                              cudaStream_t s);
// Integer-pipe binary64 check (probe.cu): `pairs` operand pairs from a counter-based generator, products and
// sums compared bit for bit with the binary64 instructions; counts[0..3] (device) += mismatched products,
// mismatched sums, products and sums taken by the integer fast path.
cudaError_t launch_binary64_check(uint64_t pairs, uint64_t seed, unsigned long long *counts, cudaStream_t s);
int set_strip_override(uint32_t h, uint32_t w, uint32_t C, uint32_t P);
int set_row_band_override(uint32_t h, uint32_t w, uint32_t C, uint32_t RB);
// Threads per CTA of the column pass (256 or 512) and the row pass (128 or 256) for a frame shape; 0: default.
int set_cta_threads_override(uint32_t h, uint32_t w, uint32_t C, uint32_t st, uint32_t rt);
void cta_threads(uint32_t h, uint32_t w, uint32_t C, uint32_t *st, uint32_t *rt);
int set_encrypt_route(int route);   // FHD_ROUTE_TWO_PASS or FHD_ROUTE_SINGLE_PASS; -1 on a bad value

}  // namespace fhd
