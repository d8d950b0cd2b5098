/*
 * fhdcipher -- C ABI of a GB300 (sm_103a) implementation of the
 * diffusion-free bit-level video cipher of arXiv 2505.07158, "Real-Time
 * Bit-Level Encryption of Full High-Definition Video Without Diffusion".
 *
 * Per frame (Algorithm 1 of the paper): the frame digest H (XOR of the
 * SHA-256 digests of n sub-frames, Sec. II-A), the initial-condition
 * reconstruction from H and the stream's chaining state, 2n iterations of the
 * master Lorenz hyperchaotic system LHCS_m (Eq. (1)), 2n worker systems that
 * expand the shift distances D and XOR bytes B (Sec. II-B, Algorithm 2), and
 * one pass of bit-level horizontal + vertical circular shifts and XOR
 * (Sec. II-C, Algos 3-7); decryption runs the exact inverse.
 *
 * Conventions for every entry point:
 *  - Frames are H x W x C uint8, C-contiguous, channel fastest (HWC), with
 *    1 <= C <= 4, 1 <= H <= 12288, 1 <= W <= 16384.  Frame, digest, D and B pointers are
 *    DEVICE pointers owned by the caller; the library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued asynchronously; a return of FHD_OK means the
 *    arguments were accepted and the work enqueued, not that it finished.
 *  - Errors: 0 on success, a negative FHD_ERR_* code otherwise; nothing is
 *    enqueued when an argument check fails.  cipher_last_error() gives a
 *    message.  No call ever falls back to the CPU.
 *  - One handle is used from one host thread at a time.  It keeps scratch
 *    buffers per CUDA stream, so calls on different CUDA streams may run
 *    concurrently on the device; frames of one video stream must still reach
 *    the device in order (same CUDA stream, or the caller orders the streams
 *    with events).  A call may be captured into a CUDA graph once the same
 *    batch has run uncaptured on that CUDA stream (the scratch is then sized);
 *    stream open/close/export/import synchronise and must not be captured.
 */
#ifndef FHDCIPHER_H
#define FHDCIPHER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FHD_OK = 0,
    FHD_ERR_INVALID_ARG = -1, /* null pointer, zero or oversized dimension, bad parameter */
    FHD_ERR_OOM = -2,         /* device or pinned allocation failed */
    FHD_ERR_BAD_STREAM = -3,  /* unknown or closed stream id */
    FHD_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    FHD_ERR_CUDA = -6,        /* a CUDA runtime call failed */
    FHD_ERR_STATE = -7,       /* device status word reports a failed kernel check */
    FHD_ERR_TOO_LARGE = -8    /* request exceeds a documented maximum */
};

#define FHD_MAX_DIM 16384u    /* frame width limit: a band of whole rows lives in shared memory */
#define FHD_MAX_HEIGHT 12288u /* frame height limit: a full-height strip lives in shared memory */
#define FHD_MAX_WORKERS 1024u
#define FHD_STATE_BYTES 48u /* x, y, z, w, gamma (binary64) + frame counter (uint64) */

typedef struct fhd_cipher fhd_cipher;

/* Protocol parameters; both ends of a channel must use the same values
 * (the paper requires the same worker count n on sender and receiver,
 * Sec. V).  A zero field takes its default. */
typedef struct {
    uint32_t n_workers;  /* n: sub-frames per frame and worker pairs; default 32 (Tab. speedEvaluation) */
    double rk4_h;        /* step of the RK4 integration of Eq. (1); default 0.01 */
    uint32_t u_bound[4]; /* reconstruction upper bounds u_x, u_y, u_z, u_w; default 20, 20, 40, 20 */
    uint32_t digest_mode; /* how H is formed from the n sub-frame digests h_i: FHD_DIGEST_XOR (0, default) */
    uint32_t digest_transport; /* how H travels: FHD_TRANSPORT_PLAIN (0, default) or FHD_TRANSPORT_MASKED */
} fhd_params;

/* Digest modes.  FHD_DIGEST_XOR: H = h_1 xor ... xor h_n (Sec. II-A, Algorithm 1).  FHD_DIGEST_TREE, an
 * option of this library and not of the paper: H = SHA-256(h_1 || ... || h_n), the 32 n bytes of the
 * sub-frame digests concatenated in order, so that identical sub-frames do not cancel and their order
 * counts.  Same partition and sub-frame digests either way; both ends of a channel must use the same
 * mode (it decides the H the sender transmits and the receiver's integrity check). */
enum { FHD_DIGEST_XOR = 0, FHD_DIGEST_TREE = 1 };

/* Digest transport.  Sec. V sends the frames' hashes encrypted over the public channel but gives no
 * mechanism.  FHD_TRANSPORT_PLAIN: frames[i].digest holds H as computed.  FHD_TRANSPORT_MASKED, an option of
 * this library: encryption writes H xor M to frames[i].digest, with
 *   M = SHA-256("FHDMASK1" || LE64(x) || LE64(y) || LE64(z) || LE64(w) || LE64(gamma)),
 * the bit patterns of the stream's chaining state before the frame (the key's x0..w0 for the first
 * frame), so each frame has its own mask; the keystream still derives from H.  Decryption reads H xor M,
 * unmasks it with its own chaining state and leaves H in frames[i].digest (so cipher_verify_frames can
 * follow).  The masked digest is written by LHCS_m: encrypt_frames_split then records digests_done after
 * LHCS_m, not after the digest stage.  Both ends must use the same transport. */
enum { FHD_TRANSPORT_PLAIN = 0, FHD_TRANSPORT_MASKED = 1 };

/* One frame of a batch.  `digest` is written by encrypt_frames (the 32-byte
 * H the receiver needs, Sec. V) and read by decrypt_frames. */
typedef struct {
    uint32_t stream_id;
    uint32_t height, width, channels;
    const uint8_t *src; /* device, height*width*channels bytes */
    uint8_t *dst;       /* device, same size; must not overlap src */
    uint8_t *digest;    /* device, 32 bytes */
} fhd_frame;

/* Create a cipher from a 256-bit key.  The paper's key is the five doubles
 * x0, y0, z0, w0, gamma (Sec. IV-A); the 32 key bytes map to them as
 * k_m = little-endian uint64 of bytes [8m, 8m+8), v_m = (k_m >> 11) 2^-53 u_m,
 * gamma = -1.52 + 1.46 ((k0^k1^k2^k3) >> 11) 2^-53.  `params` may be NULL.
 * Selects the current CUDA device.  On success *out owns device memory. */
int cipher_init(const uint8_t key[32], const fhd_params *params, fhd_cipher **out);

/* Create a cipher from the paper's own key (x0, y0, z0, w0, gamma), Sec. II-A. */
int cipher_init_raw(double x0, double y0, double z0, double w0, double gamma,
                    const fhd_params *params, fhd_cipher **out);

/* Open a video stream whose chaining state starts at the cipher's key
 * (Algorithm 1: the first frame reconstructs from the user inputs). */
int cipher_open_stream(fhd_cipher *c, uint32_t *stream_id);

/* Open a stream with its own 256-bit key (same mapping as cipher_init). */
int cipher_open_stream_key(fhd_cipher *c, const uint8_t key[32], uint32_t *stream_id);

/* Close a stream; its id may be reused by a later open. */
int cipher_close_stream(fhd_cipher *c, uint32_t stream_id);

/* Encrypt `count` frames (Algorithm 1 per frame).  Frames of one stream are
 * processed in array order and each advances that stream's chaining state
 * (Sec. II-A: the next frame reconstructs from x_2n..w_2n of this one).
 * Frames of different streams and sizes may be mixed in one call; they run
 * in one batched pass.  count == 0 is a no-op. */
int encrypt_frames(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream);

/* Decrypt `count` frames: the inverse of encrypt_frames given each frame's
 * transmitted digest (read from frames[i].digest). */
int decrypt_frames(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream);

/* As encrypt_frames / decrypt_frames, with two CUDA events (cudaEvent_t
 * passed as void*) that order only the chaining step between calls: the
 * kernel that advances the streams' chaining state (LHCS_m) first waits on
 * the n_wait events in wait_events (may be NULL / 0), and `master_done` (may
 * be NULL) is recorded on `stream` right after it.  A caller can issue the
 * next frames of a stream on another CUDA stream, passing this call's
 * master_done as a wait event: the digests, keystreams and permutations of
 * consecutive frames then overlap while their chaining stays in order. */
int encrypt_frames_ex(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream,
                      void *const *wait_events, uint32_t n_wait, void *master_done);
int decrypt_frames_ex(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream,
                      void *const *wait_events, uint32_t n_wait, void *master_done);

/* Sender side with an early digest event: as encrypt_frames_ex, and
 * `digests_done` (may be NULL) is recorded on `stream` once every frame's
 * digest H (Algorithm 1: the XOR fold of the sub-frame digests) is in
 * frames[i].digest, before LHCS_m runs (after it with FHD_TRANSPORT_MASKED,
 * whose transmitted digest LHCS_m writes).  A receiver on the same device can
 * wait on it to start its own chaotic stage while the sender's keystream and
 * permutation are still running.  For more than 256 frames it is recorded
 * after the digests of the last group of 256.  `keystream_done` (may be
 * NULL) is recorded right after the last worker kernel (Sec. II-B), before
 * the permutation: later chaotic work gated on it does not share the FP64
 * pipes with this call's keystream, while the permutation may overlap it. */
int encrypt_frames_split(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream,
                         void *const *wait_events, uint32_t n_wait, void *digests_done, void *master_done,
                         void *keystream_done);

/* Receiver side with the ciphertext still in flight: as decrypt_frames_ex,
 * and the first kernel that reads frames[i].src (the inverse permutation of
 * Algorithm 2) also waits on the n_data events in data_events (may be NULL /
 * 0).  key_waits gate LHCS_m, which reads frames[i].digest; so a receiver can
 * run the chaotic stage (Sec. II-B: master and workers) of a batch as soon as
 * its digests are on the device, while the ciphertext is still being produced
 * or copied, and the permutation starts once data_events have fired.  Events
 * are cudaEvent_t passed as void*; master_done as in decrypt_frames_ex,
 * keystream_done as in encrypt_frames_split. */
int decrypt_frames_split(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream,
                         void *const *key_waits, uint32_t n_key_waits, void *const *data_events,
                         uint32_t n_data, void *master_done, void *keystream_done);

/* Every ordering hook of one call.  Events are cudaEvent_t passed as void*,
 * owned by the caller; a list may be NULL when its count is 0 (a nonzero count
 * with a NULL list is FHD_ERR_INVALID_ARG), NULL entries are skipped, and a
 * NULL output event is not recorded.
 *   key_waits      gate LHCS_m (Sec. II-A: the chaining step; it reads the
 *                  digests and the chaining state);
 *   worker_waits   gate the worker kernel (Sec. II-B, the 2n chaotic systems
 *                  that produce D and B).  A caller streaming batch after batch
 *                  can bound how many batches' workers share the FP64 pipes
 *                  (e.g. the workers of batch k wait for those of batch k - 2)
 *                  while the digest stage and LHCS_m of later batches still run
 *                  ahead of them;
 *   data_events    gate the first kernel that reads frames[i].src after the
 *                  digest stage (the permutation);
 *   digests_done   recorded once every digest H is in frames[i].digest, before
 *                  LHCS_m (after it with FHD_TRANSPORT_MASKED, whose transmitted
 *                  digest LHCS_m writes; encryption only: decryption reads the
 *                  digests);
 *   master_done    recorded right after LHCS_m;
 *   keystream_done recorded right after the last worker kernel, before the
 *                  permutation.
 * All hooks apply to the first group of 256 frames of the call, the output
 * events to the last; groups of one call run in order.  A pipeline that keeps
 * many CUDA streams busy (clips in flight, serving lanes, and with the SM
 * partition two internal streams per caller stream) should run with
 * CUDA_DEVICE_MAX_CONNECTIONS=32, set before CUDA starts: with the default 8
 * hardware queues, a stream held by an event wait stalls the streams that share
 * its queue. */
typedef struct {
    void *const *key_waits;
    uint32_t n_key_waits;
    void *const *worker_waits;
    uint32_t n_worker_waits;
    void *const *data_events;
    uint32_t n_data;
    void *digests_done;
    void *master_done;
    void *keystream_done;
} fhd_schedule;

/* encrypt_frames / decrypt_frames with the hooks of `sched` (NULL: none). */
int encrypt_frames_sched(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream,
                         const fhd_schedule *sched);
int decrypt_frames_sched(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream,
                         const fhd_schedule *sched);

/* Pre-allocate at least `bytes` of scratch for calls on CUDA stream `stream`
 * (synchronises that stream), so that later calls on it never allocate.
 * frame_scratch_bytes() gives the scratch one frame needs. */
int cipher_reserve(fhd_cipher *c, void *stream, uint64_t bytes);

/* Persistent batched launch (the paper runs one frame at a time; this is a
 * batching option of this library).  The whole of Algorithm 1 for `count`
 * frames (at most 64; frames of any size and stream, several frames of one
 * stream in call order) runs as ONE kernel launch with one CTA per SM that
 * pulls its tasks from device queues: the sub-frame digest pipelines (Sec.
 * II-A, largest frames first), LHCS_m of every stream (Algorithm 1), the
 * worker warps (Algorithm 2; one chain warp per SM sub-partition), and the
 * confusion + XOR passes (Sec. II-C, Algos 3-7) of each frame as soon as its
 * keystream exists.  Per-frame dependency counters order the tasks; every
 * wait is bounded (cipher_set_persistent_limits, default 2 s), after which
 * the launch ends with the batch unfinished and cipher_sync_status returns
 * FHD_ERR_TIMEOUT.  Results, chaining and digests are those of
 * encrypt_frames / decrypt_frames.  Asynchronous on `stream`; the handle's
 * scratch for `stream` is sized like encrypt_frames' (a first call outside
 * CUDA graph capture sizes it and the launch's counters, after which the call
 * can be captured and replayed).  Strip widths and row bands are those of the
 * other calls where they fit the launch's shared memory, smaller otherwise. */
int encrypt_frames_persistent(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream);
int decrypt_frames_persistent(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream);

/* Sender and receiver in one persistent launch: `sender` encrypts enc_frames
 * and `receiver` decrypts dec_frames, where dec_frames[k].src and .digest must
 * be enc_frames[k].dst and .digest (same shape), and two receiver frames
 * share a stream exactly when the two sender frames do.  The receiver's LHCS_m of a
 * frame waits only for the sender's LHCS_m of it (which has written the
 * transmitted digest), its inverse permutation for the frame's ciphertext, so
 * the two sides' chaotic stages overlap.  Both handles must share n_workers,
 * rk4_h, u_bound, digest mode and transport (FHD_ERR_INVALID_ARG otherwise);
 * a timeout is reported by both handles' cipher_sync_status. */
int cipher_round_trip_persistent(fhd_cipher *sender, fhd_cipher *receiver, uint32_t count,
                                 const fhd_frame *enc_frames, const fhd_frame *dec_frames, void *stream);

/* Wait limit of this handle's persistent launches (timeout_ns, 1 ms .. 60 s)
 * and a test hook: hold_frame >= 0 withholds that frame's digest, so that the
 * waits on it run out (-1: none). */
int cipher_set_persistent_limits(fhd_cipher *c, uint64_t timeout_ns, int hold_frame);

/* Timeline of this handle's last persistent launch (instrumentation; waits
 * for the handle's CUDA streams): for frame k < count (call order, at most
 * 64), ms[9k + 0] = when its digest was published, and for side s (0: this
 * handle's direction, 1: the receiver of a round trip) ms[9k + 1 + 4s ..
 * 9k + 4 + 4s] = when its LHCS_m iterates, its keystream (its last worker
 * warp, or its trajectory on the one-trajectory route), its last row band and
 * its last column strip were done, in milliseconds after the launch's start;
 * -1 where that never happened (e.g. no such side). */
int cipher_persistent_trace(fhd_cipher *c, uint32_t count, double *ms);
/* Device scratch one frame of this shape takes in a call (sub-frame digests,
 * LHCS_m iterates, D, B, the frame between the permutation passes and the
 * trajectory records), each part 16-byte aligned. */
uint64_t fhd_frame_scratch_bytes(uint32_t n_workers, uint32_t height, uint32_t width, uint32_t channels);

/* Receiver-side integrity check (the paper transmits the digests with the
 * frames, Sec. V): recompute H over frames[i].dst (the decrypted frames) with
 * the cipher's n and compare it with frames[i].digest; ok[i] (device, one
 * byte per frame) becomes 1 when they match and 0 otherwise.  A corrupted
 * ciphertext, digest or chaining state gives 0 with overwhelming probability.
 * Does not touch any stream's chaining state. */
int cipher_verify_frames(fhd_cipher *c, uint32_t count, const fhd_frame *frames, uint8_t *ok, void *stream);

/* Copy a stream's chaining state (FHD_STATE_BYTES bytes) to host memory
 * after synchronising the handle's last CUDA stream; for exact resume. */
int cipher_export_state(fhd_cipher *c, uint32_t stream_id, void *buf, size_t len);

/* Overwrite a stream's chaining state from FHD_STATE_BYTES bytes of host memory. */
int cipher_import_state(fhd_cipher *c, uint32_t stream_id, const void *buf, size_t len);

/* Synchronise `stream`, then read and clear the device status word.
 * Returns FHD_OK, FHD_ERR_STATE or FHD_ERR_TIMEOUT, or FHD_ERR_CUDA. */
int cipher_sync_status(fhd_cipher *c, void *stream);

/* Last error message of this handle (never NULL; valid until the next call). */
const char *cipher_last_error(const fhd_cipher *c);

/* Free the handle and its device memory (synchronises the device first). */
void cipher_destroy(fhd_cipher *c);

/* ---- The hot path's steps, one call each (device pointers, async). ---- */

/* Sec. II-A: digest[32] = XOR over i < n of SHA-256 of bytes
 * [floor(i*nbytes/n), floor((i+1)*nbytes/n)) of `data` (FIPS 180-4).
 * nbytes may be 0.  `count` independent buffers of equal size laid end to end
 * (data + k*nbytes -> digest + 32k) are hashed in one launch.  count * n above
 * 2^32 - 1 returns FHD_ERR_TOO_LARGE and enqueues nothing. */
int fhd_frame_digest(const uint8_t *data, uint64_t nbytes, uint32_t n, uint32_t count,
                     uint8_t *digest, void *stream);

/* As fhd_frame_digest with the FHD_DIGEST_TREE mode: digest[32] = SHA-256 of the n sub-frame digests
 * concatenated in order (not the paper's fold; see fhd_params.digest_mode). */
int fhd_frame_digest_tree(const uint8_t *data, uint64_t nbytes, uint32_t n, uint32_t count,
                          uint8_t *digest, void *stream);

/* fhd_frame_digest for callers that cannot allocate device memory (no
 * counterpart in the paper).  Some callers may not call cudaMalloc or any
 * allocating routine: a capture/encode loop on a real-time path, where an
 * allocator call can block or synchronise the whole device and stall work
 * already in flight, or a host framework that reserves all device memory up
 * front.  This entry point allocates nothing: the count * n sub-frame digests
 * live in a fixed device array of FHD_NOALLOC_MAX_SUBFRAMES x 32 bytes (2 MiB)
 * that every GPU loading the library holds until the process exits.
 * Same arguments and result as fhd_frame_digest.  count * n above
 * FHD_NOALLOC_MAX_SUBFRAMES returns FHD_ERR_TOO_LARGE and enqueues nothing.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device, with that device current); make
 * that first call before any stream capture.  The address is cached for the
 * life of the process: it assumes the device's primary context is never torn
 * down, so do not call this entry point again after cudaDeviceReset (the
 * reloaded module's array may sit elsewhere).  All calls share the one array:
 * calls that overlap on the GPU (e.g. on two CUDA streams without ordering)
 * race and may return wrong digests. */
#define FHD_NOALLOC_MAX_SUBFRAMES 65536u
int fhd_frame_digest_noalloc(const uint8_t *data, uint64_t nbytes, uint32_t n, uint32_t count,
                             uint8_t *digest, void *stream);

/* Sec. II-A and Algorithm 1: reconstruct x, y, z, w from state[0..3] and the
 * 32-byte digest H, iterate LHCS_m 2n times with gamma = state[4]; write the
 * iterates to IR (2n x 4 binary64, row t = state after step t+1) and the last
 * iterate back into state[0..3].  `state` (5 doubles), `H` and `IR` are
 * device pointers. */
int fhd_master(double *state, const uint8_t *H, const fhd_params *params, double *IR, void *stream);

/* Sec. II-B and Algorithm 2: from IR (2n x 4 binary64, device), run the n
 * worker pairs and fill D (C*(h+w) uint16: D[c*h+i] row shifts, then
 * D[C*h+c*w+j] pixel-column shifts) and B (h*w*C bytes, frame order). */
int fhd_keystream(const double *IR, double gamma, const fhd_params *params, uint32_t height,
                  uint32_t width, uint32_t channels, uint16_t *D, uint8_t *B, void *stream);

/* The same D and B by the one-trajectory route (fhd_set_keystream_route), for
 * an IR that holds LHCS_m's 2n iterates as fhd_master writes them (row t the
 * state after step t+1 of one trajectory of Eq. (1) with this gamma and step):
 * the route reads IR[0] .. IR[2n-1] as that trajectory and continues it from
 * IR[2n-1].  For such an IR the result equals fhd_keystream's; for iterates
 * of no single trajectory it does not (use fhd_keystream).  Takes
 * 24 ceil((48 (n-1) + 2 ceil(C (h+w)/n) + ceil(h w C/n)) / 24) + 64 bytes of
 * scratch from cudaMallocAsync on `stream` for the call. */
int fhd_keystream_trajectory(const double *IR, double gamma, const fhd_params *params, uint32_t height,
                             uint32_t width, uint32_t channels, uint16_t *D, uint8_t *B, void *stream);

/* Sec. II-C, Algos 3-7 fused: dst = XOR(B, vertical shift(horizontal bit
 * shift(src))) with the distances in D, one frame, device pointers. */
int fhd_permute_encrypt(const uint8_t *src, uint8_t *dst, uint32_t height, uint32_t width,
                        uint32_t channels, const uint16_t *D, const uint8_t *B, void *stream);

/* Exact inverse of fhd_permute_encrypt. */
int fhd_permute_decrypt(const uint8_t *src, uint8_t *dst, uint32_t height, uint32_t width,
                        uint32_t channels, const uint16_t *D, const uint8_t *B, void *stream);

/* Strip width (pixels) the permutation kernels use for this shape, and the
 * override hook of the autotuner: 0 restores the built-in choice. */
uint32_t fhd_strip_width(uint32_t height, uint32_t width, uint32_t channels);
int fhd_set_strip_width(uint32_t height, uint32_t width, uint32_t channels, uint32_t P);

/* Rows per CTA of the row pass for this shape, and its autotuner override
 * (1..64 rows; 0 restores the built-in choice, bands of about 32 KB of shared
 * memory).  An override whose band does not fit shared memory is ignored. */
uint32_t fhd_row_band(uint32_t height, uint32_t width, uint32_t channels);
int fhd_set_row_band(uint32_t height, uint32_t width, uint32_t channels, uint32_t RB);


/* Threads per CTA of the permutation passes for frames of one shape (autotuner
 * hook): the column pass 256 or 512 (default 512, two CTAs per SM; 256 runs four
 * per SM), the row pass 128 or 256 (default 256, six CTAs per SM; 128 runs
 * twelve); 0 keeps the default.  A batch takes the choice of its largest frame's
 * shape.  Results are the same for every value.  FHD_ERR_INVALID_ARG for another
 * value or a bad shape, FHD_ERR_TOO_LARGE when the override table (64 shapes) is
 * full.  fhd_cta_threads reports the choice in effect. */
int fhd_set_cta_threads(uint32_t height, uint32_t width, uint32_t channels, uint32_t strip_threads,
                        uint32_t row_threads);
int fhd_cta_threads(uint32_t height, uint32_t width, uint32_t channels, uint32_t *strip_threads,
                    uint32_t *row_threads);
/* Route of the encryption's confusion + XOR (Sec. II-C), bit-identical either
 * way, process-wide.  FHD_ROUTE_TWO_PASS (default): a row pass (row
 * rotations, whole rows staged in shared memory) writes the row-rotated frame
 * to scratch, then a column pass (full-height strips in shared memory)
 * rotates its columns and XORs with B.  FHD_ROUTE_SINGLE_PASS: one gather
 * pass -- each CTA builds a full-height strip of the row-rotated frame from the
 * source rows at their offsets, rotates its columns in shared memory and
 * writes it XORed with B, so the row-rotated frame never reaches memory (one
 * frame read, B read and one frame written) -- for batches of interleaved RGB
 * frames with width % 16 == 0, strip widths 16, 32 or 64 and 16-byte aligned
 * buffers, the two passes otherwise.  Decryption always runs its two passes.
 * Returns FHD_ERR_INVALID_ARG for another value. */
enum { FHD_ROUTE_TWO_PASS = 0, FHD_ROUTE_SINGLE_PASS = 1 };
int fhd_set_encrypt_route(int route);

/* Route of the keystream (Sec. II-B, Algorithm 2: D and B from the iterates
 * IR), bit-identical either way, process-wide; taken by encrypt_frames and
 * decrypt_frames and their variants, where IR is always LHCS_m's (the
 * persistent launches always run the worker pairs; fhd_keystream, which takes
 * any IR, too).
 * FHD_KS_ROUTE_TRAJECTORY (default): worker pair i starts from IR[2i] and
 * IR[2i+1] and iterates the same map with the same step as LHCS_m, so both of
 * its systems are the frame's LHCS_m trajectory continued, and worker i's
 * byte stream is worker 0's from 48 i bytes on.  The route computes that one
 * trajectory per frame -- about N/(24 n) + 2n states, each once, instead of
 * 2n chains of about N/(24 n) steps -- into 24-byte records (the XOR of the
 * stream bytes of consecutive states), then copies each worker's window of
 * the records into its slices of D and B.  Its time per frame is the
 * trajectory's sequential latency, the same as one worker chain's.
 * FHD_KS_ROUTE_PAIRS: the n worker pairs as 2n chains (the warp layout of
 * cipher_set_layout).  Returns the previous route, or FHD_ERR_INVALID_ARG for
 * another value. */
enum { FHD_KS_ROUTE_PAIRS = 0, FHD_KS_ROUTE_TRAJECTORY = 1 };
int fhd_set_keystream_route(int route);

/* ---- Instrumentation (not part of the cipher). ---- */

/* SM partition (CUDA green contexts, on by default where the device and
 * driver support them).  The chaining kernel LHCS_m (Algorithm 1) is one warp
 * on a strictly sequential chain; beside the worker kernels it would share an
 * SM's binary64 pipes with them.  With the partition on, each call forks from
 * its CUDA stream to two internal streams, LHCS_m on a small partition of
 * SMs (8 on GB300) and every other kernel of the call on the rest, and joins
 * back, so results and ordering on the caller's stream are unchanged; calls
 * on a stream that is being captured into a CUDA graph stay on that stream.
 * cipher_set_partition(c, 0) turns it off for this handle; enabling fails
 * with FHD_ERR_CUDA (and leaves it off) where partitioning is unavailable.
 * cipher_set_partition(c, 2) splits three ways: LHCS_m, the digest stage
 * (sub-frame SHA-256 and fold, Algorithm 1) on a second small partition, and
 * the rest; other modes are FHD_ERR_INVALID_ARG.  cipher_get_partition reports
 * the SM counts of the LHCS_m partition and of the rest (0, 0 when off). */
int cipher_set_partition(fhd_cipher *c, int enable);
int cipher_get_partition(fhd_cipher *c, uint32_t *chain_sms, uint32_t *bulk_sms);

/* Warp layout of the worker kernel (Sec. II-B), bit-identical results either
 * way.  FHD_LAYOUT_LATENCY (default): six chains per warp, one variable per
 * lane and two lanes holding constants; the shortest RK4 step (~2.0k cycles
 * on GB300), for a batch that has the device to itself.
 * FHD_LAYOUT_THROUGHPUT: eight chains per warp (four worker pairs) with
 * selects instead of constant lanes; a longer step (~2.4k cycles) but 27 %
 * fewer binary64 instructions per frame, for when several batches' workers
 * share the FP64 pipes (clips in flight, many concurrent streams). */
enum { FHD_LAYOUT_LATENCY = 0, FHD_LAYOUT_THROUGHPUT = 1 };
int cipher_set_layout(fhd_cipher *c, int layout);

/* Worker warps per CTA of the worker kernel (1 -- the default --, 2, 4 or 8):
 * the warps of one CTA are consecutive worker groups of a frame, spread over
 * the SM's four sub-partitions (binary64 pipes) together.  Results are the
 * same for every value; FHD_ERR_INVALID_ARG for another value. */
int cipher_set_worker_cta(fhd_cipher *c, uint32_t warps);

/* Worker warps of the eight-chain layout (FHD_LAYOUT_THROUGHPUT), per 8
 * consecutive warps, that run their RK4 steps (Sec. II-B, Algorithm 2) on the
 * integer pipes instead of the binary64 pipe: every multiply and add done in
 * integer arithmetic, rounded to nearest even exactly as IEEE 754 binary64
 * prescribes, with the binary64 instruction for the operands that path does
 * not cover (a step with such an operand is done again with binary64
 * instructions).  The two kinds of pipe work side by side on a GB300
 * sub-partition, but an integer-pipe step takes ~3,300 warp instructions and
 * about four times as long as a binary64 one, and a worker launch lasts as long
 * as its slowest warp: with the clip pipeline every mix measured slower than 0.
 * 0 (the default) to 8; results are bit-identical for every value;
 * FHD_ERR_INVALID_ARG above 8. */
int cipher_set_int_mix(fhd_cipher *c, uint32_t per8);

/* Dynamic shared memory each CTA of the worker kernel requests (0, the
 * default, to 232448 bytes).  The kernel does not use it: it caps how many
 * worker CTAs an SM holds at once (a placement control).  Results are the
 * same for every value; FHD_ERR_INVALID_ARG above 232448. */
int cipher_set_worker_smem(fhd_cipher *c, uint32_t bytes);


/* ---- Frame statistics of the paper's evaluation (Sec. III and IV-B) ----
 * Batched over `count` frames stored contiguously in device memory as
 * [count][height][width][channels] uint8, reported per frame and channel
 * (index f * channels + c).  All output pointers are device pointers owned by
 * the caller; calls are asynchronous on `stream`; argument errors return a
 * negative FHD_ERR_* code and enqueue nothing.  Counts are exact integers and
 * only each statistic's final formula rounds (binary64).  Random sample
 * positions (pairs, blocks) are inputs: the caller draws them. */

/* Histogram statistics, Sec. III-A and III-C: per frame and channel the 256-bin
 * histogram z (optional `hist`, uint32 count*channels*256, may be NULL) and
 * stats[3 * (f * channels + c) + {0, 1, 2}] = histogram variance (Eq. 4),
 * chi^2 (Eq. 5), information entropy in bits (Eq. 10).  Uses a stream-ordered
 * scratch of count*channels*256*8 bytes. */
int fhd_stats_histogram(const uint8_t *frames, uint32_t count, uint32_t height, uint32_t width, uint32_t channels,
                        uint32_t *hist, double *stats, void *stream);

/* NPCR and UACI between frames a[f] and b[f] (Sec. IV-B, Eqs. 14-15), in
 * percent: out[2 * (f * channels + c) + {0, 1}].  `counts` (optional, uint64
 * count*channels*2, may be NULL) receives the exact number of changed pixels
 * and the sum of |a - b| per frame and channel. */
int fhd_stats_npcr_uaci(const uint8_t *a, const uint8_t *b, uint32_t count, uint32_t height, uint32_t width,
                        uint32_t channels, uint64_t *counts, double *out, void *stream);

/* Correlation coefficient of adjacent pixel pairs (Sec. III-B, Eqs. 6-9) in
 * the horizontal (d = 0), vertical (1) and diagonal (2) directions:
 * pairs[2 * ((f * 3 + d) * npairs + k) + {0, 1}] = (row, column) of pixel x
 * of pair k; y is its right, lower or lower-right neighbour, which must lie
 * inside the frame (1 <= npairs <= 2^22).  r[3 * (f * channels + c) + d];
 * `sums` (optional, int64 count*channels*3*5, may be NULL) receives the exact
 * sums of x, y, x^2, y^2, xy.  A pair outside the frame is skipped and sets
 * bit 0 of *status (device uint32, optional). */
int fhd_stats_correlation(const uint8_t *frames, uint32_t count, uint32_t height, uint32_t width, uint32_t channels,
                          const uint32_t *pairs, uint32_t npairs, int64_t *sums, double *r, unsigned *status,
                          void *stream);

/* Local Shannon entropy (Sec. III-C, Eq. 11): the mean over k blocks of
 * block x block pixels of their information entropy, per frame and channel:
 * out[f * channels + c].  blocks[2 * (f * k + q) + {0, 1}] = (row, column) of
 * block q's top-left pixel (the paper draws 30 non-overlapping 44 x 44
 * blocks at random).  A block outside the frame sets bit 0 of *status.
 * Uses a stream-ordered scratch of count*k*channels doubles. */
int fhd_stats_local_entropy(const uint8_t *frames, uint32_t count, uint32_t height, uint32_t width,
                            uint32_t channels, const uint32_t *blocks, uint32_t k, uint32_t block, double *out,
                            unsigned *status, void *stream);

/* Kernel kinds reported by cipher_profile_read, in this order. */
enum { FHD_K_SHA = 0, FHD_K_MASTER = 1, FHD_K_KEYSTREAM = 2, FHD_K_ENCRYPT = 3, FHD_K_DECRYPT = 4, FHD_K_COUNT = 5 };

/* Start (enable != 0) or stop recording a CUDA event pair on the launch
 * stream around every kernel this handle launches. */
int cipher_profile(fhd_cipher *c, int enable);

/* Wait for the recorded events, add up per kernel kind the elapsed
 * milliseconds and launch counts since the last read into ms[FHD_K_COUNT]
 * and launches[FHD_K_COUNT], and forget them. */
int cipher_profile_read(fhd_cipher *c, double *ms, uint32_t *launches);

/* The launches recorded since the last cipher_profile_read, one span each,
 * without clearing them: kinds[i] (FHD_K_*), start_ms[i] and end_ms[i] in
 * milliseconds after `origin` (a cudaEvent_t passed as void*, recorded with
 * timing enabled before those launches).  Fills at most `cap` entries and
 * sets *count to the number of recorded launches (which may exceed cap).
 * Synchronises on the launches' events.  With several CUDA streams in
 * flight the spans overlap; their union is the time a kind of kernel kept
 * the device busy. */
int cipher_profile_spans(fhd_cipher *c, void *origin, uint32_t cap, int32_t *kinds, double *start_ms,
                         double *end_ms, uint32_t *count);

/* Binary64 pipe probe (measurement only; the paper has no counterpart): the
 * peak rate against which the worker kernel's roofline (Sec. II-B) is quoted.
 * Launches one CTA per SM with 4 * warps_per_subpartition warps (1..8), every
 * lane running eight independent binary64 fused multiply-add chains of `iters`
 * steps (1..2^24), asynchronously on `stream`; the caller times it with CUDA
 * events.  *lane_ops (host) receives the binary64 lane-operations it executes
 * (SMs x threads x iters x 8).  `sink` is a device buffer of at least one
 * double per SM that the kernel may write.  Bad arguments return
 * FHD_ERR_INVALID_ARG and enqueue nothing. */
int fhd_fp64_probe(uint32_t warps_per_subpartition, uint32_t iters, double *sink, uint64_t *lane_ops, void *stream);

/* Check of the integer-pipe binary64 multiply and add that cipher_set_int_mix
 * uses, against the binary64 instructions, on `pairs` (1 .. 2^40) operand
 * pairs from a counter-based generator seeded by `seed` (any bit patterns, the
 * chaotic range, near cancellation, the alignment boundary of the sum, few
 * significand bits for exact products and ties, zeros and subnormals).
 * counts (host, 4 entries) receives: mismatched products, mismatched sums
 * (bit for bit; the target is 0 and 0), and the products and sums that the
 * integer fast path took.  Synchronises `stream`.  FHD_ERR_INVALID_ARG for a
 * null counts or pairs out of range; FHD_ERR_OOM; FHD_ERR_CUDA. */
int fhd_binary64_check(uint64_t pairs, uint64_t seed, uint64_t *counts, void *stream);

/* Number of kernels this library has launched in this process. */
uint64_t fhd_launch_count(void);

/* Library version string. */
const char *fhd_version(void);

/* ---- Checked build (range checks of every computed index) ----
 * The library can be compiled with -DFHD_BOUNDS_CHECK (libfhdcipher_checked.so beside the default
 * library).  In that build each global or shared-memory access of a kernel whose index is computed from
 * the frame geometry, the keystream, the launch descriptor or a task queue is first compared with the
 * extent of its buffer; an access that fails is counted and skipped (a skipped load reads 0, a skipped
 * store writes nothing), nothing traps, and the kernel runs to its end.  Results of a call in which a
 * check failed are void.  cipher_sync_status of a checked build also returns FHD_ERR_STATE when a check
 * has failed since the last report.  Identical results and no failed check on valid input are what the
 * checked build's tests assert. */

/* Build options of the loaded library: FHD_BUILD_BOUNDS_CHECK when it is the checked build. */
#define FHD_BUILD_BOUNDS_CHECK 1u
uint32_t fhd_build_flags(void);

/* Synchronise the device, then read and clear the bounds records of every kernel of the library:
 * *count = accesses that failed their range check since the last report; of the first of them, *site (a
 * code that fhd_bounds_site_name describes), *index and *limit (the checked index and the extent it had
 * to stay below, in elements of the buffer).  Any out pointer may be NULL.  In the default build every
 * output is 0 and nothing is synchronised.  Returns FHD_OK or FHD_ERR_CUDA. */
int fhd_bounds_report(uint32_t *count, uint32_t *site, uint64_t *index, uint64_t *limit);

/* Description of a bounds-check site ("column pass: frame store", ...); "unknown site" otherwise. */
const char *fhd_bounds_site_name(uint32_t site);

/* Checked build: run the encryption's permutation kernels (row pass, column pass) on a 16 x 64 x 3 frame
 * whose descriptor declares one row fewer than its buffers hold, so that the checks of the last row's
 * accesses fail and those accesses are skipped.  Every buffer is allocated at its full size, so no access
 * leaves its allocation either way.  The bounds records are cleared first; *count and *site (either may
 * be NULL) are fhd_bounds_report's afterwards.  Runs on `stream` and synchronises it.  Returns
 * FHD_ERR_STATE in the default build, FHD_ERR_OOM or FHD_ERR_CUDA on failure. */
int fhd_bounds_selftest(uint32_t *count, uint32_t *site, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FHDCIPHER_H */
