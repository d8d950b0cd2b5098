// Host side of the C ABI declared in include/fhdcipher.h: argument checks,
// per-stream chaining state, scratch management and the four launches of a
// batch (K1 sub-frame SHA-256, K2a master LHCS, K2b worker LHCS pairs,
// K3/K4 fused permutation).  Every step of the cipher runs in the kernels;
// the host only validates, lays out descriptors and enqueues.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>   // driver-API types only: its entry points are fetched at run time

#include "common.cuh"

using fhd::Batch;
using fhd::FrameDesc;
using fhd::StreamState;

struct fhd_cipher {
    int device = 0;
    uint32_t n = 32;
    double h = 0.01;
    uint32_t u[4] = {20, 20, 40, 20};
    double key_ic[5] = {0, 0, 0, 0, 0};
    std::vector<StreamState> mirror;   // host copy of gamma (and initial state)
    std::vector<uint8_t> open;
    StreamState *d_states = nullptr;
    size_t cap_states = 0;
    unsigned *d_status = nullptr;
    // Scratch (sub-frame digests, LHCS_m iterates, D, B) per CUDA stream, so
    // that calls on different CUDA streams can run concurrently.
    // With the SM partition on, a call on `stream` forks to two internal
    // streams: `chain` in the small partition (LHCS_m) and `bulk` in the rest
    // (digests, workers, permutation), and joins back; ev = fork, digests,
    // master, join.
    // With the three-way partition (mode 2) the digest stage runs on `digest3` in a partition of its own,
    // LHCS_m on `chain3` and the rest on `bulk3`; ev[4] orders LHCS_m after the bulk stream's work so far.
    struct Scratch {
        cudaStream_t stream;
        uint8_t *ptr;
        size_t cap;
        cudaStream_t chain = nullptr, bulk = nullptr;
        cudaStream_t chain3 = nullptr, digest3 = nullptr, bulk3 = nullptr;
        cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    };
    std::vector<Scratch> scratch;
    int partition = 0;   // 0 off, 1 LHCS_m on its own SMs, 2 LHCS_m and the digest stage each on their own
    int layout = FHD_LAYOUT_LATENCY;
    uint32_t worker_cta = 1;   // worker warps per CTA of the keystream kernel
    uint32_t int_mix = 0;      // eight-chain worker warps per 8 on the integer pipes
    uint32_t worker_smem = 0;  // dynamic shared memory per worker CTA (caps worker CTAs per SM)
    uint32_t digest_mode = FHD_DIGEST_XOR;
    uint32_t transport = FHD_TRANSPORT_PLAIN;
    cudaStream_t last_stream = nullptr;
    // Persistent launches: the dependency counters of the launch (device), its wait limit and test hook.
    fhd::PCounters *d_pcnt = nullptr;
    unsigned long long p_timeout_ns = 2000000000ull;
    int p_hold = -1;
    std::string err;
    bool prof = false;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
};

namespace {

thread_local std::string g_err;   // last error of the handle-less entry points
std::atomic<uint64_t> g_launches{0};

}  // namespace

namespace fhd {
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace fhd

namespace {

cudaEvent_t take_event(fhd_cipher *c) {
    if (!c->pool.empty()) { cudaEvent_t e = c->pool.back(); c->pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch one kernel family, counting it and (when profiling) bracketing it
// with events on the launch stream.
template <class F>
cudaError_t timed(fhd_cipher *c, int kind, cudaStream_t s, F &&launch) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (c && c->prof) { a = take_event(c); b = take_event(c); cudaEventRecord(a, s); }
    cudaError_t e = launch();
    if (c && c->prof) { cudaEventRecord(b, s); c->recs.push_back({kind, a, b}); }
    return e;
}

int fail(fhd_cipher *c, int code, const std::string &msg) {
    if (c) c->err = msg; else g_err = msg;
    return code;
}

int cuda_fail(fhd_cipher *c, cudaError_t e, const char *what) {
    return fail(c, FHD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool resolve_params(const fhd_params *p, uint32_t &n, double &h, uint32_t u[4], std::string &why) {
    n = 32;
    h = 0.01;
    const uint32_t du[4] = {20, 20, 40, 20};
    for (int m = 0; m < 4; ++m) u[m] = du[m];
    if (!p) return true;
    if (p->n_workers) n = p->n_workers;
    if (p->rk4_h != 0.0) h = p->rk4_h;
    for (int m = 0; m < 4; ++m)
        if (p->u_bound[m]) u[m] = p->u_bound[m];
    if (n > FHD_MAX_WORKERS) { why = "n_workers exceeds FHD_MAX_WORKERS"; return false; }
    if (!(h > 0.0) || !(h < 1.0)) { why = "rk4_h must be in (0, 1)"; return false; }
    for (int m = 0; m < 4; ++m)
        if (u[m] > 65536u) { why = "u_bound entries must be <= 65536"; return false; }
    return true;
}

// 256-bit key -> x0, y0, z0, w0, gamma (the mapping documented in the header).
// Built with -ffp-contract=off: each product and sum is rounded on its own.
void key_to_ic(const uint8_t key[32], const uint32_t u[4], double ic[5]) {
    uint64_t k[4];
    for (int m = 0; m < 4; ++m) {
        uint64_t v = 0;
        for (int i = 7; i >= 0; --i) v = (v << 8) | key[8 * m + i];
        k[m] = v;
    }
    for (int m = 0; m < 4; ++m) {
        volatile double unit = (double)(k[m] >> 11) * 0x1p-53;
        ic[m] = unit * (double)u[m];
    }
    volatile double g = (double)((k[0] ^ k[1] ^ k[2] ^ k[3]) >> 11) * 0x1p-53;
    volatile double prod = 1.46 * g;
    ic[4] = -1.52 + prod;
}

uint64_t align16(uint64_t x) { return (x + 15) & ~15ull; }

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone;
}

// Wait for every CUDA stream this handle has used.
cudaError_t sync_all(fhd_cipher *c) {
    cudaError_t e = cudaSuccess;
    for (auto &sc : c->scratch) {
        cudaError_t e2 = cudaStreamSynchronize(sc.stream);
        if (e == cudaSuccess) e = e2;
    }
    if (c->last_stream) {
        cudaError_t e2 = cudaStreamSynchronize(c->last_stream);
        if (e == cudaSuccess) e = e2;
    }
    return e;
}


std::mutex g_prep_mu;
bool g_prepared[64] = {};

cudaError_t prepare_device() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_prep_mu);
    if (dev >= 0 && dev < 64 && g_prepared[dev]) return cudaSuccess;
    e = fhd::permute_prepare();
    if (e == cudaSuccess && dev >= 0 && dev < 64) g_prepared[dev] = true;
    return e;
}

// ---- SM partition (CUDA green contexts).  The chaining kernel (LHCS_m) is a
// single warp on a strictly sequential chain; beside the worker kernels it
// would share an SM sub-partition's FP64 pipe with them.  A small partition
// of kChainSms SMs runs only LHCS_m, the rest runs everything else, so the
// next batch's LHCS_m can overlap this batch's workers at full speed.
constexpr unsigned kChainSms = 8;   // the minimum partition on sm_90 and later

struct DriverApi {
    CUresult (*deviceGet)(CUdevice *, int) = nullptr;
    CUresult (*getDevResource)(CUdevice, CUdevResource *, CUdevResourceType) = nullptr;
    CUresult (*smSplit)(CUdevResource *, unsigned *, const CUdevResource *, CUdevResource *, unsigned, unsigned) = nullptr;
    CUresult (*genDesc)(CUdevResourceDesc *, CUdevResource *, unsigned) = nullptr;
    CUresult (*greenCreate)(CUgreenCtx *, CUdevResourceDesc, CUdevice, unsigned) = nullptr;
    CUresult (*greenStream)(CUstream *, CUgreenCtx, unsigned, int) = nullptr;
    CUresult (*streamDestroy)(CUstream) = nullptr;
};

struct DevicePartition {
    bool tried = false, ok = false;
    CUgreenCtx chain = nullptr, bulk = nullptr;
    unsigned chain_sms = 0, bulk_sms = 0;
    std::string why;   // the step that failed, when !ok
    // The three-way split (cipher_set_partition(c, 2)): LHCS_m, the digest stage, and the rest.
    bool tried3 = false, ok3 = false;
    CUgreenCtx chain3 = nullptr, digest3 = nullptr, bulk3 = nullptr;
    unsigned chain3_sms = 0, digest3_sms = 0, bulk3_sms = 0;
};

std::mutex g_part_mu;
DriverApi g_drv;
bool g_drv_tried = false, g_drv_ok = false;
DevicePartition g_part[64];

std::string g_drv_why;

bool load_driver_api() {
    auto get = [](const char *name, void **fn) {
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        cudaError_t e = cudaGetDriverEntryPointByVersion(name, fn, CUDA_VERSION, cudaEnableDefault, &q);
        if (e == cudaSuccess && q == cudaDriverEntryPointSuccess && *fn != nullptr) return true;
        g_drv_why = std::string("driver entry point ") + name + ": " + cudaGetErrorString(e) + ", query " +
                    std::to_string((int)q);
        return false;
    };
    return get("cuDeviceGet", (void **)&g_drv.deviceGet) &&
           get("cuDeviceGetDevResource", (void **)&g_drv.getDevResource) &&
           get("cuDevSmResourceSplitByCount", (void **)&g_drv.smSplit) &&
           get("cuDevResourceGenerateDesc", (void **)&g_drv.genDesc) &&
           get("cuGreenCtxCreate", (void **)&g_drv.greenCreate) &&
           get("cuGreenCtxStreamCreate", (void **)&g_drv.greenStream) &&
           get("cuStreamDestroy", (void **)&g_drv.streamDestroy);
}

// The partition of device `dev`, created on first use; nullptr when the
// device or driver cannot partition (then calls stay on the caller's stream).
const DevicePartition *device_partition(int dev) {
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_part_mu);
    DevicePartition &p = g_part[dev];
    if (!p.tried) {
        p.tried = true;
        if (!g_drv_tried) {
            g_drv_tried = true;
            g_drv_ok = load_driver_api();
        }
        CUdevice cd;
        CUdevResource all{}, part{}, rest{};
        CUdevResourceDesc da = nullptr, db = nullptr;
        unsigned nb = 1;
        CUresult r = CUDA_SUCCESS;
        auto step = [&](CUresult rr, const char *what) {
            r = rr;
            if (rr != CUDA_SUCCESS) p.why = std::string(what) + " failed with CUresult " + std::to_string((int)rr);
            return rr == CUDA_SUCCESS;
        };
        if (!g_drv_ok) {
            p.why = g_drv_why;
        } else if (step(g_drv.deviceGet(&cd, dev), "cuDeviceGet") &&
                   step(g_drv.getDevResource(cd, &all, CU_DEV_RESOURCE_TYPE_SM), "cuDeviceGetDevResource")) {
            if (all.sm.smCount < 4 * kChainSms) {
                p.why = "too few SMs to partition";
            } else if (step(g_drv.smSplit(&part, &nb, &all, &rest, 0, kChainSms), "cuDevSmResourceSplitByCount") &&
                       step(g_drv.genDesc(&da, &part, 1), "cuDevResourceGenerateDesc") &&
                       step(g_drv.genDesc(&db, &rest, 1), "cuDevResourceGenerateDesc") &&
                       step(g_drv.greenCreate(&p.chain, da, cd, CU_GREEN_CTX_DEFAULT_STREAM), "cuGreenCtxCreate") &&
                       step(g_drv.greenCreate(&p.bulk, db, cd, CU_GREEN_CTX_DEFAULT_STREAM), "cuGreenCtxCreate")) {
                p.ok = true;
                p.chain_sms = part.sm.smCount;
                p.bulk_sms = rest.sm.smCount;
            }
        }
        (void)r;
    }
    return p.ok ? &p : nullptr;
}

// The three-way partition of device `dev` (kChainSms for LHCS_m, kChainSms for the digest stage, the rest),
// created on first use; nullptr where the device or driver cannot partition.
const DevicePartition *device_partition3(int dev) {
    if (!device_partition(dev)) return nullptr;
    std::lock_guard<std::mutex> lk(g_part_mu);
    DevicePartition &p = g_part[dev];
    if (!p.tried3) {
        p.tried3 = true;
        // One split into two groups of kChainSms and the remainder (a remainder cannot be split again).
        CUdevice cd;
        CUdevResource all{}, g2[2] = {}, r2{};
        CUdevResourceDesc da = nullptr, dd = nullptr, db = nullptr;
        unsigned n2 = 2;
        auto ok = [&](CUresult rr, const char *what) {
            if (rr != CUDA_SUCCESS) p.why = std::string(what) + " failed with CUresult " + std::to_string((int)rr);
            return rr == CUDA_SUCCESS;
        };
        CUdevResource &a = g2[0], &d = g2[1];
        if (ok(g_drv.deviceGet(&cd, dev), "cuDeviceGet") &&
            ok(g_drv.getDevResource(cd, &all, CU_DEV_RESOURCE_TYPE_SM), "cuDeviceGetDevResource") &&
            ok(g_drv.smSplit(g2, &n2, &all, &r2, 0, kChainSms), "cuDevSmResourceSplitByCount") &&
            ok(n2 == 2 ? CUDA_SUCCESS : CUDA_ERROR_INVALID_VALUE, "two SM groups") &&
            ok(g_drv.genDesc(&da, &a, 1), "cuDevResourceGenerateDesc") &&
            ok(g_drv.genDesc(&dd, &d, 1), "cuDevResourceGenerateDesc") &&
            ok(g_drv.genDesc(&db, &r2, 1), "cuDevResourceGenerateDesc") &&
            ok(g_drv.greenCreate(&p.chain3, da, cd, CU_GREEN_CTX_DEFAULT_STREAM), "cuGreenCtxCreate") &&
            ok(g_drv.greenCreate(&p.digest3, dd, cd, CU_GREEN_CTX_DEFAULT_STREAM), "cuGreenCtxCreate") &&
            ok(g_drv.greenCreate(&p.bulk3, db, cd, CU_GREEN_CTX_DEFAULT_STREAM), "cuGreenCtxCreate")) {
            p.ok3 = true;
            p.chain3_sms = a.sm.smCount;
            p.digest3_sms = d.sm.smCount;
            p.bulk3_sms = r2.sm.smCount;
        }
    }
    return p.ok3 ? &p : nullptr;
}

// The internal streams and events of caller stream `sc` for the handle's partition mode (created on first
// use).
cudaError_t partition_streams(fhd_cipher *c, fhd_cipher::Scratch &sc) {
    if (!sc.ev[0]) {
        for (auto &e : sc.ev) {
            cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
            if (r != cudaSuccess) return r;
        }
    }
    if (c->partition == 2) {
        if (sc.chain3) return cudaSuccess;
        const DevicePartition *p = device_partition3(c->device);
        if (!p) return cudaErrorNotSupported;
        CUstream s3[3] = {nullptr, nullptr, nullptr};
        CUgreenCtx g3[3] = {p->chain3, p->digest3, p->bulk3};
        for (int k = 0; k < 3; ++k)
            if (g_drv.greenStream(&s3[k], g3[k], CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS) {
                for (int j = 0; j < k; ++j) g_drv.streamDestroy(s3[j]);
                return cudaErrorNotSupported;
            }
        sc.chain3 = (cudaStream_t)s3[0];
        sc.digest3 = (cudaStream_t)s3[1];
        sc.bulk3 = (cudaStream_t)s3[2];
        return cudaSuccess;
    }
    if (sc.chain) return cudaSuccess;
    const DevicePartition *p = device_partition(c->device);
    if (!p) return cudaErrorNotSupported;
    CUstream a = nullptr, b = nullptr;
    if (g_drv.greenStream(&a, p->chain, CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS) return cudaErrorNotSupported;
    if (g_drv.greenStream(&b, p->bulk, CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS) {
        g_drv.streamDestroy(a);
        return cudaErrorNotSupported;
    }
    sc.chain = (cudaStream_t)a;
    sc.bulk = (cudaStream_t)b;
    return cudaSuccess;
}

fhd_cipher::Scratch *scratch_of(fhd_cipher *c, cudaStream_t s) {
    for (auto &sc : c->scratch)
        if (sc.stream == s) return &sc;
    return nullptr;
}

bool check_dims(uint32_t h, uint32_t w, uint32_t C, std::string &why) {
    if (h == 0 || w == 0 || C == 0) { why = "frame dimensions must be non-zero"; return false; }
    if (C > 4) { why = "channels must be 1..4"; return false; }
    if (h > FHD_MAX_HEIGHT || w > FHD_MAX_DIM) { why = "frame exceeds FHD_MAX_HEIGHT rows or FHD_MAX_DIM columns"; return false; }
    if (fhd::strip_width(h, w, C) == 0) { why = "frame too tall for the shared-memory strip"; return false; }
    if (fhd::row_smem_bytes(w, C, 1) > 232448) { why = "frame rows too wide for the shared-memory row band"; return false; }
    return true;
}

int init_common(const double ic[5], uint32_t n, double h, const uint32_t u[4], fhd_cipher **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    e = prepare_device();
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("prepare: ") + cudaGetErrorString(e));
    fhd_cipher *c = new fhd_cipher();
    c->device = dev;
    c->partition = device_partition(dev) != nullptr;
    c->n = n;
    c->h = h;
    for (int m = 0; m < 4; ++m) c->u[m] = u[m];
    for (int m = 0; m < 5; ++m) c->key_ic[m] = ic[m];
    e = cudaMalloc(&c->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return fail(nullptr, FHD_ERR_OOM, std::string("cudaMalloc status: ") + cudaGetErrorString(e));
    }
    *out = c;
    return FHD_OK;
}

int open_with_ic(fhd_cipher *c, const double ic[5], uint32_t *id) {
    if (!c || !id) return fail(c, FHD_ERR_INVALID_ARG, "null argument");
    uint32_t slot = 0;
    while (slot < c->open.size() && c->open[slot]) ++slot;
    if (slot >= c->cap_states) {
        size_t cap = c->cap_states ? 2 * c->cap_states : 64;
        while (cap <= slot) cap *= 2;
        StreamState *d = nullptr;
        cudaError_t e = cudaMalloc(&d, cap * sizeof(StreamState));
        if (e != cudaSuccess) return fail(c, FHD_ERR_OOM, std::string("cudaMalloc states: ") + cudaGetErrorString(e));
        if (c->d_states) {
            sync_all(c);
            e = cudaMemcpy(d, c->d_states, c->cap_states * sizeof(StreamState), cudaMemcpyDeviceToDevice);
            cudaFree(c->d_states);
            if (e != cudaSuccess) { cudaFree(d); c->d_states = nullptr; c->cap_states = 0;
                return cuda_fail(c, e, "copy states"); }
        }
        c->d_states = d;
        c->cap_states = cap;
    }
    if (slot >= c->open.size()) {
        c->open.resize(slot + 1, 0);
        c->mirror.resize(slot + 1);
    }
    StreamState st{};
    for (int m = 0; m < 4; ++m) st.v[m] = ic[m];
    st.gamma = ic[4];
    st.frames = 0;
    sync_all(c);
    cudaError_t e = cudaMemcpy(c->d_states + slot, &st, sizeof st, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload state");
    c->mirror[slot] = st;
    c->open[slot] = 1;
    *id = slot;
    return FHD_OK;
}

// Scratch of at least `need` bytes for CUDA stream s.  Growing it waits for
// the stream's earlier work, so it is refused while the stream is being
// captured into a CUDA graph (make one uncaptured call of the same batch first).
int ensure_scratch(fhd_cipher *c, cudaStream_t s, size_t need, uint8_t **out) {
    fhd_cipher::Scratch *slot = nullptr;
    for (auto &sc : c->scratch)
        if (sc.stream == s) slot = &sc;
    if (slot && need <= slot->cap) { *out = slot->ptr; return FHD_OK; }
    if (capturing(s))
        return fail(c, FHD_ERR_STATE, "scratch too small during CUDA graph capture: run the batch once uncaptured first");
    if (!slot) {
        c->scratch.push_back({});
        slot = &c->scratch.back();
        slot->stream = s;
    }
    cudaStreamSynchronize(s);
    if (slot->chain) {   // work of the current call may still be on the internal streams
        cudaStreamSynchronize(slot->chain);
        cudaStreamSynchronize(slot->bulk);
    }
    cudaFree(slot->ptr);
    slot->ptr = nullptr;
    slot->cap = 0;
    size_t cap = need + need / 8;
    cudaError_t e = cudaMalloc(&slot->ptr, cap);
    if (e != cudaSuccess) {
        slot->ptr = nullptr;
        return fail(c, FHD_ERR_OOM, std::string("cudaMalloc scratch: ") + cudaGetErrorString(e));
    }
    slot->cap = cap;
    *out = slot->ptr;
    return FHD_OK;
}

// Per-frame scratch: n sub-frame digests, 2n LHCS_m iterates, D, B, the
// frame between the two permutation passes, and the trajectory records.
uint64_t frame_scratch(uint32_t n, uint32_t h, uint32_t w, uint32_t C) {
    const uint64_t LD = (uint64_t)C * (h + w), N = (uint64_t)h * w * C;
    return align16(32ull * n) + align16(64ull * n) + align16(2 * LD) + 2 * align16(N) +
           align16(fhd::traj_bytes(LD, N, n));
}

int run_frames(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream, bool encrypt,
               const fhd_schedule *sched = nullptr) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    static const fhd_schedule kNoHooks{};
    const fhd_schedule &hk = sched ? *sched : kNoHooks;
    if ((hk.n_key_waits && !hk.key_waits) || (hk.n_worker_waits && !hk.worker_waits) || (hk.n_data && !hk.data_events))
        return fail(c, FHD_ERR_INVALID_ARG, "null event list with a nonzero count");
    if (count == 0) return FHD_OK;
    if (!frames) return fail(c, FHD_ERR_INVALID_ARG, "null frames");
    const cudaEvent_t digests_done = (cudaEvent_t)hk.digests_done, master_done = (cudaEvent_t)hk.master_done,
                      keystream_done = (cudaEvent_t)hk.keystream_done;
    cudaStream_t s = (cudaStream_t)stream;
    for (uint32_t k = 0; k < count; ++k) {
        const fhd_frame &f = frames[k];
        std::string why;
        if (!f.src || !f.dst || !f.digest) return fail(c, FHD_ERR_INVALID_ARG, "frame " + std::to_string(k) + ": null pointer");
        if (!check_dims(f.height, f.width, f.channels, why)) return fail(c, FHD_ERR_INVALID_ARG, "frame " + std::to_string(k) + ": " + why);
        if (f.stream_id >= c->open.size() || !c->open[f.stream_id])
            return fail(c, FHD_ERR_BAD_STREAM, "frame " + std::to_string(k) + ": stream not open");
        uint64_t N = (uint64_t)f.height * f.width * f.channels;
        const uint8_t *s0 = f.src, *d0 = f.dst;
        if (s0 < d0 + N && d0 < s0 + N) return fail(c, FHD_ERR_INVALID_ARG, "frame " + std::to_string(k) + ": src and dst overlap");
    }
    cudaError_t e = prepare_device();
    if (e != cudaSuccess) return cuda_fail(c, e, "prepare");
    static thread_local Batch b;   // ~12 KB: kept off the stack
    bool part = false;
    cudaStream_t sc = s, sb = s, sd = s;   // LHCS_m, the rest, the digest stage
    cudaEvent_t *ev = nullptr;
    for (uint32_t base = 0; base < count; base += fhd::kMaxBatch) {
        uint32_t m = count - base < (uint32_t)fhd::kMaxBatch ? count - base : (uint32_t)fhd::kMaxBatch;
        std::memset(&b, 0, sizeof b);
        b.count = m;
        b.n = c->n;
        b.digest_mode = c->digest_mode;
        b.digest_masked = c->transport == FHD_TRANSPORT_MASKED;
        b.encrypt = encrypt;
        b.int_mix = c->layout == FHD_LAYOUT_THROUGHPUT ? c->int_mix : 0;
        b.hstep = c->h;
        b.hhalf = c->h / 2.0;
        b.hsixth = c->h / 6.0;
        for (int q = 0; q < 4; ++q) b.u[q] = c->u[q];
        uint64_t need = 0;
        for (uint32_t k = 0; k < m; ++k) {
            const fhd_frame &f = frames[base + k];
            need += frame_scratch(c->n, f.height, f.width, f.channels);
        }
        uint8_t *p = nullptr;
        int rc = ensure_scratch(c, s, need, &p);
        if (rc != FHD_OK) return rc;
        if (base == 0) {
            // Streams of this call: with the SM partition (and outside graph capture), LHCS_m runs on
            // `sc` (small partition) and everything else on `sb` (the rest), forked from and joined
            // back to the caller's stream; otherwise everything runs on the caller's stream.
            fhd_cipher::Scratch *slot = scratch_of(c, s);
            part = c->partition && slot && !capturing(s) && partition_streams(c, *slot) == cudaSuccess;
            if (part) {
                const bool three = c->partition == 2;
                sc = three ? slot->chain3 : slot->chain;
                sb = three ? slot->bulk3 : slot->bulk;
                sd = three ? slot->digest3 : sb;
                ev = slot->ev;
                if ((e = cudaEventRecord(ev[0], s)) != cudaSuccess || (e = cudaStreamWaitEvent(sb, ev[0], 0)) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(sc, ev[0], 0)) != cudaSuccess ||
                    (three && (e = cudaStreamWaitEvent(sd, ev[0], 0)) != cudaSuccess))
                    return cuda_fail(c, e, "fork");
            }
        }
        uint32_t ctas = 0, rctas = 0;
        for (uint32_t k = 0; k < m; ++k) {
            const fhd_frame &f = frames[base + k];
            FrameDesc &d = b.f[k];
            d.src = f.src;
            d.dst = f.dst;
            d.digest = f.digest;
            d.h = f.height;
            d.w = f.width;
            d.C = f.channels;
            d.N = (uint64_t)f.height * f.width * f.channels;
            d.slot = f.stream_id;
            d.gamma = c->mirror[f.stream_id].gamma;
            d.part = p; p += align16(32ull * c->n);
            d.IR = reinterpret_cast<double *>(p); p += align16(64ull * c->n);
            d.D = reinterpret_cast<uint16_t *>(p); p += align16(2ull * d.C * (d.h + d.w));
            d.B = p; p += align16(d.N);
            d.G = p; p += align16(d.N);
            d.T = p; p += align16(fhd::traj_bytes((uint64_t)d.C * (d.h + d.w), d.N, c->n));
            d.P = fhd::strip_width(d.h, d.w, d.C);
            d.cta0 = ctas;
            ctas += fhd::permute_strips(d.w, d.P);
            d.RB = fhd::row_band(d.h, d.w, d.C);
            d.rcta0 = rctas;
            rctas += (d.h + d.RB - 1) / d.RB;
        }
        b.perm_ctas = ctas;
        b.row_ctas = rctas;
        // Group frames by stream (stable): each master CTA walks one stream in order.
        std::vector<uint32_t> seen;
        uint32_t pos = 0;
        for (uint32_t k = 0; k < m; ++k) {
            uint32_t sid = b.f[k].slot;
            bool dup = false;
            for (uint32_t x : seen) if (x == sid) { dup = true; break; }
            if (dup) continue;
            seen.push_back(sid);
            b.group_begin[b.groups++] = (uint16_t)pos;
            for (uint32_t k2 = k; k2 < m; ++k2)
                if (b.f[k2].slot == sid) b.order[pos++] = (uint16_t)k2;
        }
        b.group_begin[b.groups] = (uint16_t)pos;
        if (encrypt) {
            if ((e = timed(c, FHD_K_SHA, sd, [&] {
                     cudaError_t r = fhd::launch_sha_subframes(b, sd);
                     if (r != cudaSuccess) return r;
                     return b.digest_mode == FHD_DIGEST_TREE ? fhd::launch_tree_batch(b, sd)
                                                             : fhd::launch_fold_batch(b, sd);
                 })) != cudaSuccess)
                return cuda_fail(c, e, "sha launch");
            if (digests_done && !b.digest_masked && base + m >= count &&
                (e = cudaEventRecord(digests_done, sd)) != cudaSuccess)
                return cuda_fail(c, e, "record digest event");
        }
        // LHCS_m of this group of frames after the bulk stream's work so far: this group's digests,
        // and the previous group's workers, which read the iterates this LHCS_m overwrites.
        if (part && ((e = cudaEventRecord(ev[1], sb)) != cudaSuccess || (e = cudaStreamWaitEvent(sc, ev[1], 0)) != cudaSuccess))
            return cuda_fail(c, e, "bulk to chain stream");
        if (part && sd != sb &&
            ((e = cudaEventRecord(ev[4], sd)) != cudaSuccess || (e = cudaStreamWaitEvent(sc, ev[4], 0)) != cudaSuccess))
            return cuda_fail(c, e, "digest to chain stream");
        if (base == 0)
            for (uint32_t k = 0; k < hk.n_key_waits; ++k)
                if (hk.key_waits[k] && (e = cudaStreamWaitEvent(sc, (cudaEvent_t)hk.key_waits[k], 0)) != cudaSuccess)
                    return cuda_fail(c, e, "wait event");
        if ((e = timed(c, FHD_K_MASTER, sc, [&] { return fhd::launch_master(b, c->d_states, c->d_status, sc); })) != cudaSuccess)
            return cuda_fail(c, e, "master launch");
        if (master_done && base + m >= count && (e = cudaEventRecord(master_done, sc)) != cudaSuccess)
            return cuda_fail(c, e, "record master event");
        // With the masked transport the transmitted digests (H xor M) are written by LHCS_m.
        if (encrypt && digests_done && b.digest_masked && base + m >= count &&
            (e = cudaEventRecord(digests_done, sc)) != cudaSuccess)
            return cuda_fail(c, e, "record digest event");
        if (part && ((e = cudaEventRecord(ev[2], sc)) != cudaSuccess || (e = cudaStreamWaitEvent(sb, ev[2], 0)) != cudaSuccess))
            return cuda_fail(c, e, "master to bulk stream");
        if (base == 0)   // caller's gate of the workers (e.g. how many batches' workers share the FP64 pipes)
            for (uint32_t k = 0; k < hk.n_worker_waits; ++k)
                if (hk.worker_waits[k] && (e = cudaStreamWaitEvent(sb, (cudaEvent_t)hk.worker_waits[k], 0)) != cudaSuccess)
                    return cuda_fail(c, e, "wait worker event");
        if ((e = timed(c, FHD_K_KEYSTREAM, sb, [&] {
                 return fhd::keystream_route() == FHD_KS_ROUTE_TRAJECTORY
                            ? fhd::launch_trajectory_keystream(b, sb)
                            : fhd::launch_keystream(b, sb, c->layout == FHD_LAYOUT_THROUGHPUT, c->worker_cta,
                                                    c->worker_smem);
             })) != cudaSuccess)
            return cuda_fail(c, e, "keystream launch");
        if (keystream_done && base + m >= count && (e = cudaEventRecord(keystream_done, sb)) != cudaSuccess)
            return cuda_fail(c, e, "record keystream event");
        if (base == 0)   // the first reader of frames[].src after the digest stage
            for (uint32_t k = 0; k < hk.n_data; ++k)
                if (hk.data_events[k] && (e = cudaStreamWaitEvent(sb, (cudaEvent_t)hk.data_events[k], 0)) != cudaSuccess)
                    return cuda_fail(c, e, "wait data event");
        if ((e = timed(c, encrypt ? FHD_K_ENCRYPT : FHD_K_DECRYPT, sb, [&] { return fhd::launch_permute(b, encrypt, sb); })) != cudaSuccess)
            return cuda_fail(c, e, "permute launch");
    }
    if (part && ((e = cudaEventRecord(ev[3], sb)) != cudaSuccess || (e = cudaStreamWaitEvent(s, ev[3], 0)) != cudaSuccess))
        return cuda_fail(c, e, "join");
    c->last_stream = s;
    return FHD_OK;
}

// Checks shared by the batched entry points: pointers, dimensions, open streams, no src/dst overlap.
int check_frames(fhd_cipher *c, uint32_t count, const fhd_frame *frames) {
    for (uint32_t k = 0; k < count; ++k) {
        const fhd_frame &f = frames[k];
        std::string why;
        if (!f.src || !f.dst || !f.digest) return fail(c, FHD_ERR_INVALID_ARG, "frame " + std::to_string(k) + ": null pointer");
        if (!check_dims(f.height, f.width, f.channels, why)) return fail(c, FHD_ERR_INVALID_ARG, "frame " + std::to_string(k) + ": " + why);
        if (f.stream_id >= c->open.size() || !c->open[f.stream_id])
            return fail(c, FHD_ERR_BAD_STREAM, "frame " + std::to_string(k) + ": stream not open");
        const uint64_t N = (uint64_t)f.height * f.width * f.channels;
        if (f.src < f.dst + N && f.dst < f.src + N) return fail(c, FHD_ERR_INVALID_ARG, "frame " + std::to_string(k) + ": src and dst overlap");
    }
    return FHD_OK;
}

// One side of a persistent launch: descriptors (scratch of this handle on stream s), stream groups, and
// the strip widths and row bands that fit the launch's permutation shared memory.
int persistent_side(fhd_cipher *c, uint32_t count, const fhd_frame *frames, bool encrypt, cudaStream_t s,
                    fhd::PSide &S, size_t &mem_smem) {
    const size_t lim = fhd::persistent_mem_smem_limit();
    std::memset(&S, 0, sizeof S);
    S.count = count;
    S.n = c->n;
    S.digest_mode = c->digest_mode;
    S.digest_masked = c->transport == FHD_TRANSPORT_MASKED;
    S.encrypt = encrypt;
    S.hstep = c->h;
    S.hhalf = c->h / 2.0;
    S.hsixth = c->h / 6.0;
    for (int q = 0; q < 4; ++q) S.u[q] = c->u[q];
    S.states = c->d_states;
    S.status = c->d_status;
    uint64_t need = 0;
    for (uint32_t k = 0; k < count; ++k)
        need += frame_scratch(c->n, frames[k].height, frames[k].width, frames[k].channels);
    uint8_t *p = nullptr;
    int rc = ensure_scratch(c, s, need, &p);
    if (rc != FHD_OK) return rc;
    for (uint32_t k = 0; k < count; ++k) {
        const fhd_frame &f = frames[k];
        FrameDesc &d = S.f[k];
        d.src = f.src;
        d.dst = f.dst;
        d.digest = f.digest;
        d.h = f.height;
        d.w = f.width;
        d.C = f.channels;
        d.N = (uint64_t)f.height * f.width * f.channels;
        d.slot = f.stream_id;
        d.gamma = c->mirror[f.stream_id].gamma;
        d.part = p; p += align16(32ull * c->n);
        d.IR = reinterpret_cast<double *>(p); p += align16(64ull * c->n);
        d.D = reinterpret_cast<uint16_t *>(p); p += align16(2ull * d.C * (d.h + d.w));
        d.B = p; p += align16(d.N);
        d.G = p; p += align16(d.N);
        d.T = p; p += align16(fhd::traj_bytes((uint64_t)d.C * (d.h + d.w), d.N, c->n));
        S.emits[k] = fhd::keystream_route() == FHD_KS_ROUTE_TRAJECTORY
                         ? (uint32_t)((d.N + fhd::kEmitTaskBytes - 1) / fhd::kEmitTaskBytes) : 0u;
        // at most 64 pixels: the persistent column pass (352 threads) covers a strip row (<= 256 bytes) per pass
        uint32_t P = std::min(fhd::strip_width(d.h, d.w, d.C), 64u);
        while (P > 1 && fhd::strip_smem_bytes(d.h, P, d.C) > lim) P /= 2;
        if (fhd::strip_smem_bytes(d.h, P, d.C) > lim)
            return fail(c, FHD_ERR_TOO_LARGE, "frame " + std::to_string(k) + ": too tall for a persistent launch");
        d.P = P;
        const size_t pitch = ((size_t)d.w * d.C + 15) & ~(size_t)15;
        uint32_t RB = (uint32_t)(lim / (2 * pitch + 4 * d.C));
        RB = RB > 16 ? 16 : RB;
        if (RB < 1) return fail(c, FHD_ERR_TOO_LARGE, "frame " + std::to_string(k) + ": too wide for a persistent launch");
        d.RB = RB;
        S.strips[k] = fhd::permute_strips(d.w, P);
        S.bands[k] = (d.h + RB - 1) / RB;
        const size_t a = fhd::strip_smem_bytes(d.h, P, d.C), r = fhd::row_smem_bytes(d.w, d.C, RB);
        mem_smem = std::max(mem_smem, std::max(a, r));
    }
    std::vector<uint32_t> seen;
    uint32_t pos = 0;
    for (uint32_t k = 0; k < count; ++k) {
        const uint32_t sid = S.f[k].slot;
        bool dup = false;
        for (uint32_t x : seen) if (x == sid) { dup = true; break; }
        if (dup) continue;
        seen.push_back(sid);
        S.group_begin[S.groups++] = (uint16_t)pos;
        for (uint32_t k2 = k; k2 < count; ++k2)
            if (S.f[k2].slot == sid) S.order[pos++] = (uint16_t)k2;
    }
    S.group_begin[S.groups] = (uint16_t)pos;
    return FHD_OK;
}

// A persistent launch of one direction (c1 == nullptr) or of a round trip: c0 encrypts frames0 and c1
// decrypts frames1, frame k of frames1 being the ciphertext of frame k of frames0.
int run_persistent(fhd_cipher *c0, fhd_cipher *c1, uint32_t count, const fhd_frame *f0, const fhd_frame *f1,
                   bool encrypt0, void *stream) {
    if (!c0 || (f1 && !c1)) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    if (count == 0) return FHD_OK;
    if (!f0 || (c1 && !f1)) return fail(c0, FHD_ERR_INVALID_ARG, "null frames");
    if (count > (uint32_t)fhd::kPMax) return fail(c0, FHD_ERR_TOO_LARGE, "more than 64 frames in a persistent launch");
    int rc = check_frames(c0, count, f0);
    if (rc == FHD_OK && c1) rc = check_frames(c1, count, f1);
    if (rc != FHD_OK) return rc;
    if (c1) {
        if (c0->n != c1->n || c0->h != c1->h || std::memcmp(c0->u, c1->u, sizeof c0->u) ||
            c0->digest_mode != c1->digest_mode || c0->transport != c1->transport)
            return fail(c0, FHD_ERR_INVALID_ARG, "sender and receiver protocol parameters differ");
        for (uint32_t k = 0; k < count; ++k) {
            if (f1[k].src != f0[k].dst || f1[k].digest != f0[k].digest || f1[k].height != f0[k].height ||
                f1[k].width != f0[k].width || f1[k].channels != f0[k].channels)
                return fail(c0, FHD_ERR_INVALID_ARG, "frame " + std::to_string(k) +
                                                       ": the receiver's frame is not the sender's ciphertext");
            // the receiver's streams mirror the sender's: frames k and k2 share a stream on one side iff on both
            for (uint32_t k2 = 0; k2 < k; ++k2)
                if ((f0[k].stream_id == f0[k2].stream_id) != (f1[k].stream_id == f1[k2].stream_id))
                    return fail(c0, FHD_ERR_INVALID_ARG, "frame " + std::to_string(k) +
                                                           ": the receiver's streams do not mirror the sender's");
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = prepare_device();
    if (e != cudaSuccess) return cuda_fail(c0, e, "prepare");
    if (!c0->d_pcnt) {
        if (capturing(s))
            return fail(c0, FHD_ERR_STATE, "persistent launch during CUDA graph capture: run the batch once uncaptured first");
        e = cudaMalloc(&c0->d_pcnt, sizeof(fhd::PCounters));
        if (e != cudaSuccess) { c0->d_pcnt = nullptr; return fail(c0, FHD_ERR_OOM, "cudaMalloc persistent counters"); }
    }
    static thread_local fhd::PLaunch L;
    std::memset(&L, 0, sizeof L);
    size_t mem_smem = 0;
    rc = persistent_side(c0, count, f0, encrypt0, s, L.s[0], mem_smem);
    if (rc == FHD_OK && c1) rc = persistent_side(c1, count, f1, false, s, L.s[1], mem_smem);
    if (rc != FHD_OK) return rc;
    L.sides = c1 ? 2 : 1;
    L.traj = fhd::keystream_route() == FHD_KS_ROUTE_TRAJECTORY;
    L.wpf = L.traj ? 1u : (c0->n + 2) / 3;
    L.sha_units = encrypt0 ? (uint32_t)(((uint64_t)count * c0->n + 31) / 32) : 0;

    std::vector<uint32_t> idx(count);
    for (uint32_t k = 0; k < count; ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) { return L.s[0].f[a].N > L.s[0].f[b].N; });
    for (uint32_t k = 0; k < count; ++k) {
        L.prio[k] = idx[k];
        L.mprio[k] = idx[count - 1 - k];
    }
    // chain queue: the LHCS_m tasks of all stream groups (in the order of each group's earliest frame in
    // mprio order), then per frame in mprio order its worker warps: every task after those it waits for
    {
        std::vector<uint32_t> rank(count);
        for (uint32_t r = 0; r < count; ++r) rank[L.mprio[r]] = r;
        for (uint32_t k = 0; k < count; ++k) L.chain_masters[k] = 0;
        for (uint32_t g = 0; g < L.s[0].groups; ++g) {
            uint32_t best = L.s[0].order[L.s[0].group_begin[g]];
            for (uint32_t q = L.s[0].group_begin[g]; q < L.s[0].group_begin[g + 1]; ++q)
                if (rank[L.s[0].order[q]] < rank[best]) best = L.s[0].order[q];
            L.chain_masters[best] = (uint16_t)L.sides;
            L.chain_group[best] = (uint16_t)g;
        }
        L.chain_begin[0] = 0;
        for (uint32_t r = 0; r < count; ++r) L.chain_begin[r + 1] = L.chain_begin[r] + L.chain_masters[L.mprio[r]];
        L.chain_masters_total = L.chain_begin[count];
        L.chain_tasks = L.chain_masters_total + L.sides * L.wpf * count;
    }
    L.memb_begin[0] = 0;
    for (uint32_t r = 0; r < count; ++r) {
        const uint32_t f = L.mprio[r];
        uint32_t blk = L.s[0].emits[f] + L.s[0].strips[f] + L.s[0].bands[f];
        if (c1) blk += L.s[1].emits[f] + L.s[1].strips[f] + L.s[1].bands[f];
        L.memb_begin[r + 1] = L.memb_begin[r] + blk;
    }
    L.mem_tasks = L.memb_begin[count];
    L.timeout_ns = c0->p_timeout_ns;
    // a digest CTA's pipeline may hash several tasks in turn: allow ~4 us per 64-byte block of all the
    // digest work (far above its speed) beyond the dependency limit
    {
        int sms = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c0->device);
        uint64_t blocks = 0;
        if (encrypt0)
            for (uint32_t k = 0; k < count; ++k) blocks += L.s[0].f[k].N / 64 + 2ull * c0->n;
        const uint64_t ctas = std::max<uint64_t>(1, std::min<uint64_t>(L.sha_units, (uint64_t)std::max(sms, 1)));
        L.digest_wait_ns = L.timeout_ns + 4000ull * blocks / ctas;
    }
    L.hold_frame = c0->p_hold;
    L.cnt = c0->d_pcnt;
    if ((e = cudaMemsetAsync(c0->d_pcnt, 0, sizeof(fhd::PCounters), s)) != cudaSuccess)
        return cuda_fail(c0, e, "reset persistent counters");
    if ((e = fhd::launch_persistent(L, mem_smem, s)) != cudaSuccess) return cuda_fail(c0, e, "persistent launch");
    c0->last_stream = s;
    if (c1) c1->last_stream = s;
    return FHD_OK;
}

#ifdef FHD_BOUNDS_CHECK
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// The bounds records of every translation unit with kernels, read and cleared (the caller has synchronised).
cudaError_t take_all_bounds(fhd::BoundsRecord &r) {
    r = fhd::BoundsRecord{};
    cudaError_t (*const takers[])(fhd::BoundsRecord *) = {fhd::take_bounds_sha, fhd::take_bounds_chaos,
                                                          fhd::take_bounds_permute, fhd::take_bounds_persist,
                                                          fhd::take_bounds_stats};
    for (auto t : takers) {
        cudaError_t e = t(&r);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

std::string bounds_message(const fhd::BoundsRecord &r) {
    return std::to_string(r.count) + " range check(s) failed; first: " + fhd::bounds_site_name(r.site) +
           ", index " + std::to_string(r.index) + " of " + std::to_string(r.limit);
}

}  // namespace

namespace fhd {
const char *bounds_site_name(unsigned site) {
    switch (site) {
        case kSiteShaMessage: return "digest: sub-frame message outside its frame";
        case kSiteShaBlock: return "digest: message block past the message";
        case kSiteShaDigest: return "digest: frame index past the batch";
        case kSiteMasterIR: return "LHCS_m: iterate past 2n x 4";
        case kSiteMasterFrame: return "LHCS_m: frame index past the batch";
        case kSiteWorkerIR: return "worker: initial value past the iterates";
        case kSiteWorkerD: return "worker: shift-distance byte past C (h + w) entries";
        case kSiteWorkerB: return "worker: XOR byte past the frame";
        case kSiteTrajIR: return "trajectory: iterate past 2n x 4";
        case kSiteTrajRecord: return "trajectory: record past the frame's records";
        case kSiteEmitLoad: return "emission: record byte past the frame's records";
        case kSiteEmitStore: return "emission: D or B byte past its buffer";
        case kSiteRowLoad: return "row pass: frame load";
        case kSiteRowShift: return "row pass: row shift load";
        case kSiteRowSmem: return "row pass: shared-memory band or shift table";
        case kSiteRowStore: return "row pass: frame store";
        case kSiteStripShift: return "column pass: column shift load";
        case kSiteStripLoad: return "column pass: frame or keystream load";
        case kSiteStripSmem: return "column pass: shared-memory strip";
        case kSiteStripStore: return "column pass: frame store";
        case kSiteGatherShift: return "single pass: shift distance or rotation table";
        case kSiteGatherLoad: return "single pass: frame load";
        case kSiteGatherSmem: return "single pass: staging buffer or strip";
        case kSiteGatherStore: return "single pass: keystream load or ciphertext store";
        case kSitePersistTask: return "persistent launch: task outside the launch";
        case kSiteStats: return "statistics: frame load past the batch";
        default: return "unknown site";
    }
}
}  // namespace fhd

extern "C" {

uint32_t fhd_build_flags(void) { return kChecked ? FHD_BUILD_BOUNDS_CHECK : 0u; }

const char *fhd_bounds_site_name(uint32_t site) { return fhd::bounds_site_name(site); }

int fhd_bounds_report(uint32_t *count, uint32_t *site, uint64_t *index, uint64_t *limit) {
    fhd::BoundsRecord r{};
    if (kChecked) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = take_all_bounds(r);
        if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("bounds report: ") + cudaGetErrorString(e));
    }
    if (count) *count = r.count;
    if (site) *site = r.site;
    if (index) *index = r.index;
    if (limit) *limit = r.limit;
    return FHD_OK;
}

int fhd_bounds_selftest(uint32_t *count, uint32_t *site, void *stream) {
    if (!kChecked) return fail(nullptr, FHD_ERR_STATE, "not a bounds-checked build");
    constexpr uint32_t h = 16, w = 64, C = 3;
    constexpr uint64_t N = (uint64_t)h * w * C;
    cudaStream_t s = (cudaStream_t)stream;
    fhd::BoundsRecord r{};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = take_all_bounds(r);   // start from clear records
    if (e == cudaSuccess) e = prepare_device();
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("selftest: ") + cudaGetErrorString(e));
    uint8_t *buf = nullptr;   // F, E, B, G (N bytes each) and D (C (h + w) 16-bit entries), all full size
    const size_t bytes = 4 * N + 2ull * C * (h + w);
    if ((e = cudaMalloc(&buf, bytes)) != cudaSuccess) return fail(nullptr, FHD_ERR_OOM, "selftest buffers");
    static thread_local Batch b;
    std::memset(&b, 0, sizeof b);
    b.count = 1;
    FrameDesc &d = b.f[0];
    d.src = buf;
    d.dst = buf + N;
    d.B = buf + 2 * N;
    d.G = buf + 3 * N;
    d.D = reinterpret_cast<uint16_t *>(buf + 4 * N);
    d.h = h;
    d.w = w;
    d.C = C;
    d.N = N - (uint64_t)w * C;   // the descriptor's extent: one row short of the buffers
    d.P = fhd::strip_width(h, w, C);
    b.perm_ctas = fhd::permute_strips(w, d.P);
    d.RB = fhd::row_band(h, w, C);
    b.row_ctas = (h + d.RB - 1) / d.RB;
    e = cudaMemsetAsync(buf, 0x5a, bytes, s);
    if (e == cudaSuccess) e = fhd::launch_permute(b, true, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = take_all_bounds(r);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("selftest: ") + cudaGetErrorString(e));
    if (count) *count = r.count;
    if (site) *site = r.site;
    return FHD_OK;
}

const char *fhd_version(void) { return "fhdcipher 0.1 (sm_103a)"; }

// The digest mode and transport of `params` (the paper's fold, sent as computed, when params is NULL).
bool resolve_digest_mode(const fhd_params *p, uint32_t &mode, uint32_t &transport, std::string &why) {
    mode = p ? p->digest_mode : (uint32_t)FHD_DIGEST_XOR;
    transport = p ? p->digest_transport : (uint32_t)FHD_TRANSPORT_PLAIN;
    if (mode != FHD_DIGEST_XOR && mode != FHD_DIGEST_TREE) { why = "unknown digest_mode"; return false; }
    if (transport != FHD_TRANSPORT_PLAIN && transport != FHD_TRANSPORT_MASKED) {
        why = "unknown digest_transport";
        return false;
    }
    return true;
}

int cipher_init(const uint8_t key[32], const fhd_params *params, fhd_cipher **out) {
    if (!key || !out) return fail(nullptr, FHD_ERR_INVALID_ARG, "null argument");
    uint32_t n, u[4], mode, transport;
    double h;
    std::string why;
    if (!resolve_params(params, n, h, u, why) || !resolve_digest_mode(params, mode, transport, why))
        return fail(nullptr, FHD_ERR_INVALID_ARG, why);
    double ic[5];
    key_to_ic(key, u, ic);
    int rc = init_common(ic, n, h, u, out);
    if (rc == FHD_OK) {
        (*out)->digest_mode = mode;
        (*out)->transport = transport;
    }
    return rc;
}

int cipher_init_raw(double x0, double y0, double z0, double w0, double gamma, const fhd_params *params,
                    fhd_cipher **out) {
    if (!out) return fail(nullptr, FHD_ERR_INVALID_ARG, "null argument");
    uint32_t n, u[4], mode, transport;
    double h;
    std::string why;
    if (!resolve_params(params, n, h, u, why) || !resolve_digest_mode(params, mode, transport, why))
        return fail(nullptr, FHD_ERR_INVALID_ARG, why);
    const double ic[5] = {x0, y0, z0, w0, gamma};
    int rc = init_common(ic, n, h, u, out);
    if (rc == FHD_OK) {
        (*out)->digest_mode = mode;
        (*out)->transport = transport;
    }
    return rc;
}

int cipher_open_stream(fhd_cipher *c, uint32_t *stream_id) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    return open_with_ic(c, c->key_ic, stream_id);
}

int cipher_open_stream_key(fhd_cipher *c, const uint8_t key[32], uint32_t *stream_id) {
    if (!c || !key) return fail(c, FHD_ERR_INVALID_ARG, "null argument");
    double ic[5];
    key_to_ic(key, c->u, ic);
    return open_with_ic(c, ic, stream_id);
}

int cipher_close_stream(fhd_cipher *c, uint32_t stream_id) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    if (stream_id >= c->open.size() || !c->open[stream_id]) return fail(c, FHD_ERR_BAD_STREAM, "stream not open");
    c->open[stream_id] = 0;
    return FHD_OK;
}

int encrypt_frames(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream) {
    return run_frames(c, count, frames, stream, true);
}

int decrypt_frames(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream) {
    return run_frames(c, count, frames, stream, false);
}

int encrypt_frames_ex(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream,
                      void *const *wait_events, uint32_t n_wait, void *master_done) {
    fhd_schedule hk{};
    hk.key_waits = wait_events;
    hk.n_key_waits = n_wait;
    hk.master_done = master_done;
    return run_frames(c, count, frames, stream, true, &hk);
}

int decrypt_frames_ex(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream,
                      void *const *wait_events, uint32_t n_wait, void *master_done) {
    fhd_schedule hk{};
    hk.key_waits = wait_events;
    hk.n_key_waits = n_wait;
    hk.master_done = master_done;
    return run_frames(c, count, frames, stream, false, &hk);
}

int encrypt_frames_split(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream,
                         void *const *wait_events, uint32_t n_wait, void *digests_done, void *master_done,
                         void *keystream_done) {
    fhd_schedule hk{};
    hk.key_waits = wait_events;
    hk.n_key_waits = n_wait;
    hk.digests_done = digests_done;
    hk.master_done = master_done;
    hk.keystream_done = keystream_done;
    return run_frames(c, count, frames, stream, true, &hk);
}

int decrypt_frames_split(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream,
                         void *const *key_waits, uint32_t n_key_waits, void *const *data_events,
                         uint32_t n_data, void *master_done, void *keystream_done) {
    fhd_schedule hk{};
    hk.key_waits = key_waits;
    hk.n_key_waits = n_key_waits;
    hk.data_events = data_events;
    hk.n_data = n_data;
    hk.master_done = master_done;
    hk.keystream_done = keystream_done;
    return run_frames(c, count, frames, stream, false, &hk);
}

int encrypt_frames_sched(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream,
                         const fhd_schedule *sched) {
    return run_frames(c, count, frames, stream, true, sched);
}

int decrypt_frames_sched(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream,
                         const fhd_schedule *sched) {
    return run_frames(c, count, frames, stream, false, sched);
}

int cipher_verify_frames(fhd_cipher *c, uint32_t count, const fhd_frame *frames, uint8_t *ok, void *stream) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    if (count == 0) return FHD_OK;
    if (!frames || !ok) return fail(c, FHD_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    for (uint32_t k = 0; k < count; ++k) {
        const fhd_frame &f = frames[k];
        std::string why;
        if (!f.dst || !f.digest) return fail(c, FHD_ERR_INVALID_ARG, "frame " + std::to_string(k) + ": null pointer");
        if (!check_dims(f.height, f.width, f.channels, why)) return fail(c, FHD_ERR_INVALID_ARG, why);
    }
    static thread_local Batch b;
    for (uint32_t base = 0; base < count; base += fhd::kMaxBatch) {
        const uint32_t m = count - base < (uint32_t)fhd::kMaxBatch ? count - base : (uint32_t)fhd::kMaxBatch;
        std::memset(&b, 0, sizeof b);
        b.count = m;
        b.n = c->n;
        b.digest_mode = c->digest_mode;
        uint8_t *p = nullptr;
        int rc = ensure_scratch(c, s, (uint64_t)m * 32ull * c->n, &p);
        if (rc != FHD_OK) return rc;
        for (uint32_t k = 0; k < m; ++k) {
            const fhd_frame &f = frames[base + k];
            FrameDesc &d = b.f[k];
            d.dst = f.dst;
            d.digest = f.digest;
            d.h = f.height;
            d.w = f.width;
            d.C = f.channels;
            d.N = (uint64_t)f.height * f.width * f.channels;
            d.part = p + 32ull * c->n * k;
            d.slot = base + k;   // index into ok[]
        }
        cudaError_t e = timed(c, FHD_K_SHA, s, [&] { return fhd::launch_verify(b, ok, s); });
        if (e != cudaSuccess) return cuda_fail(c, e, "verify launch");
    }
    c->last_stream = s;
    return FHD_OK;
}

int cipher_reserve(fhd_cipher *c, void *stream, uint64_t bytes) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    uint8_t *p = nullptr;
    return ensure_scratch(c, (cudaStream_t)stream, bytes, &p);
}

uint64_t fhd_frame_scratch_bytes(uint32_t n_workers, uint32_t height, uint32_t width, uint32_t channels) {
    return frame_scratch(n_workers ? n_workers : 32, height, width, channels);
}

int cipher_export_state(fhd_cipher *c, uint32_t stream_id, void *buf, size_t len) {
    if (!c || !buf) return fail(c, FHD_ERR_INVALID_ARG, "null argument");
    if (len < FHD_STATE_BYTES) return fail(c, FHD_ERR_INVALID_ARG, "buffer shorter than FHD_STATE_BYTES");
    if (stream_id >= c->open.size() || !c->open[stream_id]) return fail(c, FHD_ERR_BAD_STREAM, "stream not open");
    cudaError_t e = sync_all(c);
    if (e == cudaSuccess) e = cudaMemcpy(buf, c->d_states + stream_id, FHD_STATE_BYTES, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "export state");
    return FHD_OK;
}

int cipher_import_state(fhd_cipher *c, uint32_t stream_id, const void *buf, size_t len) {
    if (!c || !buf) return fail(c, FHD_ERR_INVALID_ARG, "null argument");
    if (len < FHD_STATE_BYTES) return fail(c, FHD_ERR_INVALID_ARG, "buffer shorter than FHD_STATE_BYTES");
    if (stream_id >= c->open.size() || !c->open[stream_id]) return fail(c, FHD_ERR_BAD_STREAM, "stream not open");
    StreamState st;
    std::memcpy(&st, buf, sizeof st);
    cudaError_t e = sync_all(c);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_states + stream_id, &st, sizeof st, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "import state");
    c->mirror[stream_id] = st;
    return FHD_OK;
}

int encrypt_frames_persistent(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream) {
    return run_persistent(c, nullptr, count, frames, nullptr, true, stream);
}

int decrypt_frames_persistent(fhd_cipher *c, uint32_t count, const fhd_frame *frames, void *stream) {
    return run_persistent(c, nullptr, count, frames, nullptr, false, stream);
}

int cipher_round_trip_persistent(fhd_cipher *sender, fhd_cipher *receiver, uint32_t count,
                                 const fhd_frame *enc_frames, const fhd_frame *dec_frames, void *stream) {
    if (!sender || !receiver) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    return run_persistent(sender, receiver, count, enc_frames, dec_frames, true, stream);
}

int cipher_persistent_trace(fhd_cipher *c, uint32_t count, double *ms) {
    if (!c || (!ms && count)) return fail(c, FHD_ERR_INVALID_ARG, "null argument");
    if (count > (uint32_t)fhd::kPMax) return fail(c, FHD_ERR_TOO_LARGE, "more than 64 frames");
    if (!c->d_pcnt) return fail(c, FHD_ERR_STATE, "no persistent launch yet");
    cudaError_t e = sync_all(c);
    fhd::PCounters h;
    if (e == cudaSuccess) e = cudaMemcpy(&h, c->d_pcnt, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read persistent counters");
    auto rel = [&](unsigned long long t) { return t ? (double)(long long)(t - h.t0) * 1e-6 : -1.0; };
    for (uint32_t k = 0; k < count; ++k) {
        double *o = ms + 9 * k;
        o[0] = rel(h.t_digest[k]);
        for (int s = 0; s < 2; ++s) {
            o[1 + 4 * s] = rel(h.t_master[s][k]);
            o[2 + 4 * s] = rel(h.t_ks[s][k]);
            o[3 + 4 * s] = rel(h.t_rows[s][k]);
            o[4 + 4 * s] = rel(h.t_strips[s][k]);
        }
    }
    return FHD_OK;
}

int cipher_set_persistent_limits(fhd_cipher *c, uint64_t timeout_ns, int hold_frame) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    if (timeout_ns < 1000000ull || timeout_ns > 60000000000ull)
        return fail(c, FHD_ERR_INVALID_ARG, "timeout_ns must be 1 ms .. 60 s");
    if (hold_frame < -1 || hold_frame >= fhd::kPMax) return fail(c, FHD_ERR_INVALID_ARG, "hold_frame must be -1 .. 63");
    c->p_timeout_ns = timeout_ns;
    c->p_hold = hold_frame;
    return FHD_OK;
}

int cipher_sync_status(fhd_cipher *c, void *stream) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    unsigned st = 0;
    e = cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof st);
    if (e != cudaSuccess) return cuda_fail(c, e, "read status");
    if (st & fhd::kStatusTimeout) return fail(c, FHD_ERR_TIMEOUT, "a bounded device wait timed out");
    if (st) return fail(c, FHD_ERR_STATE, "device status word " + std::to_string(st));
    if (kChecked) {
        fhd::BoundsRecord r{};
        if ((e = cudaDeviceSynchronize()) == cudaSuccess) e = take_all_bounds(r);
        if (e != cudaSuccess) return cuda_fail(c, e, "read bounds records");
        if (r.count) return fail(c, FHD_ERR_STATE, bounds_message(r));
    }
    return FHD_OK;
}

const char *cipher_last_error(const fhd_cipher *c) { return c ? c->err.c_str() : g_err.c_str(); }

int cipher_profile(fhd_cipher *c, int enable) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    c->prof = enable != 0;
    return FHD_OK;
}

int cipher_profile_read(fhd_cipher *c, double *ms, uint32_t *launches) {
    if (!c || !ms || !launches) return fail(c, FHD_ERR_INVALID_ARG, "null argument");
    for (int k = 0; k < FHD_K_COUNT; ++k) { ms[k] = 0.0; launches[k] = 0; }
    int rc = FHD_OK;
    for (auto &r : c->recs) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) rc = cuda_fail(c, e, "profile events");
        ms[r.kind] += t;
        launches[r.kind] += 1;
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->recs.clear();
    return rc;
}

int cipher_profile_spans(fhd_cipher *c, void *origin, uint32_t cap, int32_t *kinds, double *start_ms,
                         double *end_ms, uint32_t *count) {
    if (!c || !origin || !count || (cap && (!kinds || !start_ms || !end_ms)))
        return fail(c, FHD_ERR_INVALID_ARG, "null argument");
    *count = (uint32_t)c->recs.size();
    uint32_t i = 0;
    for (auto &r : c->recs) {
        if (i >= cap) break;
        float a = 0.f, b = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, (cudaEvent_t)origin, r.a);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, (cudaEvent_t)origin, r.b);
        if (e != cudaSuccess) return cuda_fail(c, e, "profile spans");
        kinds[i] = r.kind;
        start_ms[i] = a;
        end_ms[i] = b;
        ++i;
    }
    return FHD_OK;
}

uint64_t fhd_launch_count(void) { return g_launches.load(); }

int fhd_set_keystream_route(int route) {
    const int old = fhd::set_keystream_route(route);
    if (old < 0) return fail(nullptr, FHD_ERR_INVALID_ARG, "route must be FHD_KS_ROUTE_PAIRS or FHD_KS_ROUTE_TRAJECTORY");
    return old;
}

int fhd_set_encrypt_route(int route) {
    if (fhd::set_encrypt_route(route) != 0) return fail(nullptr, FHD_ERR_INVALID_ARG, "route must be FHD_ROUTE_TWO_PASS or FHD_ROUTE_SINGLE_PASS");
    return FHD_OK;
}

int fhd_fp64_probe(uint32_t warps_per_subpartition, uint32_t iters, double *sink, uint64_t *lane_ops, void *stream) {
    if (!sink || !lane_ops) return fail(nullptr, FHD_ERR_INVALID_ARG, "null argument");
    if (warps_per_subpartition < 1 || warps_per_subpartition > 8)
        return fail(nullptr, FHD_ERR_INVALID_ARG, "warps_per_subpartition must be 1..8");
    if (iters < 1 || iters > (1u << 24)) return fail(nullptr, FHD_ERR_INVALID_ARG, "iters must be 1..2^24");
    cudaError_t e = fhd::launch_fp64_probe(warps_per_subpartition, iters, sink, lane_ops, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("probe launch: ") + cudaGetErrorString(e));
    return FHD_OK;
}

int fhd_binary64_check(uint64_t pairs, uint64_t seed, uint64_t *counts, void *stream) {
    if (!counts) return fail(nullptr, FHD_ERR_INVALID_ARG, "null counts");
    if (pairs < 1 || pairs > (1ull << 40)) return fail(nullptr, FHD_ERR_INVALID_ARG, "pairs must be 1..2^40");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *d = nullptr;
    cudaError_t e = cudaMallocAsync(&d, 4 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    unsigned long long h[4] = {0, 0, 0, 0};
    e = cudaMemsetAsync(d, 0, sizeof h, s);
    if (e == cudaSuccess) e = fhd::launch_binary64_check(pairs, seed, d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d, s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("binary64 check: ") + cudaGetErrorString(e));
    for (int k = 0; k < 4; ++k) counts[k] = h[k];
    return FHD_OK;
}

int cipher_set_partition(fhd_cipher *c, int enable) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    if (enable < 0 || enable > 2) return fail(c, FHD_ERR_INVALID_ARG, "partition mode must be 0, 1 or 2");
    if (!enable) { c->partition = 0; return FHD_OK; }
    if (!(enable == 2 ? device_partition3(c->device) : device_partition(c->device))) {
        c->partition = 0;
        std::string why;
        {
            std::lock_guard<std::mutex> lk(g_part_mu);
            why = c->device >= 0 && c->device < 64 ? g_part[c->device].why : "device index";
        }
        return fail(c, FHD_ERR_CUDA, "the device or driver cannot partition its SMs (green contexts): " + why);
    }
    c->partition = enable;
    return FHD_OK;
}

static int stats_args(const void *frames, uint32_t count, uint32_t h, uint32_t w, uint32_t C, const void *out) {
    if (!frames || !out) return fail(nullptr, FHD_ERR_INVALID_ARG, "null argument");
    if (count == 0) return fail(nullptr, FHD_ERR_INVALID_ARG, "count must be positive");
    if (h == 0 || w == 0 || C == 0 || C > 4 || h > FHD_MAX_HEIGHT || w > FHD_MAX_DIM)
        return fail(nullptr, FHD_ERR_INVALID_ARG, "frame dimensions out of range");
    return FHD_OK;
}

int fhd_stats_histogram(const uint8_t *frames, uint32_t count, uint32_t height, uint32_t width, uint32_t channels,
                        uint32_t *hist, double *stats, void *stream) {
    int rc = stats_args(frames, count, height, width, channels, stats);
    if (rc != FHD_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *h64 = nullptr;
    const uint64_t items = (uint64_t)count * channels;
    cudaError_t e = cudaMallocAsync(&h64, items * 256 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    e = fhd::launch_stats_histogram(frames, count, (uint64_t)height * width * channels, channels, h64, hist, stats, s);
    cudaFreeAsync(h64, s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("histogram launch: ") + cudaGetErrorString(e));
    return FHD_OK;
}

int fhd_stats_npcr_uaci(const uint8_t *a, const uint8_t *b, uint32_t count, uint32_t height, uint32_t width,
                        uint32_t channels, uint64_t *counts, double *out, void *stream) {
    int rc = stats_args(a, count, height, width, channels, out);
    if (rc != FHD_OK) return rc;
    if (!b) return fail(nullptr, FHD_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(counts);
    const uint64_t items = (uint64_t)count * channels;
    cudaError_t e = cudaSuccess;
    if (!acc) e = cudaMallocAsync(&acc, items * 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    e = fhd::launch_stats_npcr(a, b, count, (uint64_t)height * width * channels, channels, (uint64_t)height * width,
                               acc, out, s);
    if (!counts) cudaFreeAsync(acc, s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("npcr launch: ") + cudaGetErrorString(e));
    return FHD_OK;
}

int fhd_stats_correlation(const uint8_t *frames, uint32_t count, uint32_t height, uint32_t width, uint32_t channels,
                          const uint32_t *pairs, uint32_t npairs, int64_t *sums, double *r, unsigned *status,
                          void *stream) {
    int rc = stats_args(frames, count, height, width, channels, r);
    if (rc != FHD_OK) return rc;
    if (!pairs || npairs == 0 || npairs > (1u << 22))
        return fail(nullptr, FHD_ERR_INVALID_ARG, "pairs must be non-null and 1 <= npairs <= 2^22");
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t items = (uint64_t)count * channels;
    long long *sm = reinterpret_cast<long long *>(sums);
    unsigned *st = status;
    cudaError_t e = cudaSuccess;
    if (!sm) e = cudaMallocAsync(&sm, items * 3 * 5 * sizeof(long long), s);
    if (e == cudaSuccess && !st) e = cudaMallocAsync(&st, sizeof(unsigned), s);
    if (e == cudaSuccess && !status) e = cudaMemsetAsync(st, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_OOM, std::string("scratch: ") + cudaGetErrorString(e));
    e = fhd::launch_stats_correlation(frames, count, height, width, channels, pairs, npairs, sm, r, st, s);
    if (!sums) cudaFreeAsync(sm, s);
    if (!status) cudaFreeAsync(st, s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("correlation launch: ") + cudaGetErrorString(e));
    return FHD_OK;
}

int fhd_stats_local_entropy(const uint8_t *frames, uint32_t count, uint32_t height, uint32_t width,
                            uint32_t channels, const uint32_t *blocks, uint32_t k, uint32_t block, double *out,
                            unsigned *status, void *stream) {
    int rc = stats_args(frames, count, height, width, channels, out);
    if (rc != FHD_OK) return rc;
    if (!blocks || k == 0 || block == 0 || block > height || block > width)
        return fail(nullptr, FHD_ERR_INVALID_ARG, "blocks must be non-null, k >= 1 and 1 <= block <= min(height, width)");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *st = status;
    double *ent = nullptr;
    cudaError_t e = cudaMallocAsync(&ent, (uint64_t)count * k * channels * sizeof(double), s);
    if (e == cudaSuccess && !st) e = cudaMallocAsync(&st, sizeof(unsigned), s);
    if (e == cudaSuccess && !status) e = cudaMemsetAsync(st, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_OOM, std::string("scratch: ") + cudaGetErrorString(e));
    e = fhd::launch_stats_local_entropy(frames, count, height, width, channels, blocks, k, block, ent, out, st, s);
    cudaFreeAsync(ent, s);
    if (!status) cudaFreeAsync(st, s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("local entropy launch: ") + cudaGetErrorString(e));
    return FHD_OK;
}

int cipher_set_worker_smem(fhd_cipher *c, uint32_t bytes) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    if (bytes > 232448) return fail(c, FHD_ERR_INVALID_ARG, "bytes must be at most 232448");
    c->worker_smem = bytes;
    return FHD_OK;
}

int cipher_set_int_mix(fhd_cipher *c, uint32_t per8) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    if (per8 > 8) return fail(c, FHD_ERR_INVALID_ARG, "per8 must be 0..8");
    c->int_mix = per8;
    return FHD_OK;
}

int cipher_set_worker_cta(fhd_cipher *c, uint32_t warps) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    if (warps != 1 && warps != 2 && warps != 4 && warps != 8) return fail(c, FHD_ERR_INVALID_ARG, "warps must be 1, 2, 4 or 8");
    c->worker_cta = warps;
    return FHD_OK;
}

int cipher_set_layout(fhd_cipher *c, int layout) {
    if (!c) return fail(nullptr, FHD_ERR_INVALID_ARG, "null cipher");
    if (layout != FHD_LAYOUT_LATENCY && layout != FHD_LAYOUT_THROUGHPUT)
        return fail(c, FHD_ERR_INVALID_ARG, "unknown worker layout");
    c->layout = layout;
    return FHD_OK;
}

int cipher_get_partition(fhd_cipher *c, uint32_t *chain_sms, uint32_t *bulk_sms) {
    if (!c || !chain_sms || !bulk_sms) return fail(c, FHD_ERR_INVALID_ARG, "null argument");
    if (c->partition == 2) {
        const DevicePartition *p = device_partition3(c->device);
        *chain_sms = p ? p->chain3_sms : 0;
        *bulk_sms = p ? p->bulk3_sms : 0;
        return FHD_OK;
    }
    const DevicePartition *p = c->partition ? device_partition(c->device) : nullptr;
    *chain_sms = p ? p->chain_sms : 0;
    *bulk_sms = p ? p->bulk_sms : 0;
    return FHD_OK;
}

void cipher_destroy(fhd_cipher *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    for (auto &r : c->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->pool) cudaEventDestroy(e);
    for (auto &sc : c->scratch) {
        cudaFree(sc.ptr);
        for (auto e : sc.ev)
            if (e) cudaEventDestroy(e);
        if (sc.chain) g_drv.streamDestroy((CUstream)sc.chain);
        if (sc.bulk) g_drv.streamDestroy((CUstream)sc.bulk);
        if (sc.chain3) g_drv.streamDestroy((CUstream)sc.chain3);
        if (sc.digest3) g_drv.streamDestroy((CUstream)sc.digest3);
        if (sc.bulk3) g_drv.streamDestroy((CUstream)sc.bulk3);
    }
    cudaFree(c->d_states);
    cudaFree(c->d_status);
    cudaFree(c->d_pcnt);
    delete c;
}

int fhd_frame_digest(const uint8_t *data, uint64_t nbytes, uint32_t n, uint32_t count, uint8_t *digest,
                     void *stream) {
    if ((!data && nbytes) || !digest) return fail(nullptr, FHD_ERR_INVALID_ARG, "null argument");
    if (n == 0 || n > FHD_MAX_WORKERS) return fail(nullptr, FHD_ERR_INVALID_ARG, "n must be 1..FHD_MAX_WORKERS");
    if (count == 0) return FHD_OK;
    if ((uint64_t)count * n > UINT32_MAX)   // the hash kernel numbers the count * n messages with 32 bits
        return fail(nullptr, FHD_ERR_TOO_LARGE, "count * n exceeds 2^32 - 1 sub-frames");
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *part = nullptr;
    cudaError_t e = cudaMallocAsync(&part, 32ull * n * count, s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    e = timed(nullptr, FHD_K_SHA, s, [&] { return fhd::launch_sha_plain(data, nbytes, n, count, part, s); });
    if (e == cudaSuccess) e = timed(nullptr, FHD_K_SHA, s, [&] { return fhd::launch_fold(part, n, count, digest, s); });
    cudaFreeAsync(part, s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("digest launch: ") + cudaGetErrorString(e));
    return FHD_OK;
}

int fhd_frame_digest_tree(const uint8_t *data, uint64_t nbytes, uint32_t n, uint32_t count, uint8_t *digest,
                          void *stream) {
    if ((!data && nbytes) || !digest) return fail(nullptr, FHD_ERR_INVALID_ARG, "null argument");
    if (n == 0 || n > FHD_MAX_WORKERS) return fail(nullptr, FHD_ERR_INVALID_ARG, "n must be 1..FHD_MAX_WORKERS");
    if (count == 0) return FHD_OK;
    if ((uint64_t)count * n > UINT32_MAX)   // the hash kernel numbers the count * n messages with 32 bits
        return fail(nullptr, FHD_ERR_TOO_LARGE, "count * n exceeds 2^32 - 1 sub-frames");
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *part = nullptr;
    cudaError_t e = cudaMallocAsync(&part, 32ull * n * count, s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    e = timed(nullptr, FHD_K_SHA, s, [&] { return fhd::launch_sha_plain(data, nbytes, n, count, part, s); });
    if (e == cudaSuccess) e = timed(nullptr, FHD_K_SHA, s, [&] { return fhd::launch_tree(part, n, count, digest, s); });
    cudaFreeAsync(part, s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("digest launch: ") + cudaGetErrorString(e));
    return FHD_OK;
}

// fhd_frame_digest without any allocation: the sub-frame digests go to a
// fixed device array instead of memory from cudaMallocAsync.  For callers
// that may not allocate device memory -- e.g. a capture/encode loop on a
// real-time path, where an allocator call can block or synchronise the device
// and stall the work already in flight, or a host framework that reserves all
// device memory up front.  Limits and sharing rules are in the header.
int fhd_frame_digest_noalloc(const uint8_t *data, uint64_t nbytes, uint32_t n, uint32_t count, uint8_t *digest,
                             void *stream) {
    if ((!data && nbytes) || !digest) return fail(nullptr, FHD_ERR_INVALID_ARG, "null argument");
    if (n == 0 || n > FHD_MAX_WORKERS) return fail(nullptr, FHD_ERR_INVALID_ARG, "n must be 1..FHD_MAX_WORKERS");
    if (count == 0) return FHD_OK;
    if ((uint64_t)count * n > fhd::noalloc_max_digests())
        return fail(nullptr, FHD_ERR_TOO_LARGE,
                    "count * n exceeds FHD_NOALLOC_MAX_SUBFRAMES (the fixed sub-frame digest array)");
    uint8_t *part = nullptr;
    cudaError_t e = fhd::noalloc_scratch(&part);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    // Every digest slot the fold reads is written by the hash kernel of this
    // same call, so nothing left by an earlier call needs clearing.
    e = timed(nullptr, FHD_K_SHA, s, [&] { return fhd::launch_sha_plain(data, nbytes, n, count, part, s); });
    if (e == cudaSuccess) e = timed(nullptr, FHD_K_SHA, s, [&] { return fhd::launch_fold(part, n, count, digest, s); });
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("digest launch: ") + cudaGetErrorString(e));
    return FHD_OK;
}

int fhd_master(double *state, const uint8_t *H, const fhd_params *params, double *IR, void *stream) {
    if (!state || !H || !IR) return fail(nullptr, FHD_ERR_INVALID_ARG, "null argument");
    uint32_t n, u[4];
    double h;
    std::string why;
    if (!resolve_params(params, n, h, u, why)) return fail(nullptr, FHD_ERR_INVALID_ARG, why);
    cudaError_t e = timed(nullptr, FHD_K_MASTER, (cudaStream_t)stream,
                          [&] { return fhd::launch_master_raw(state, H, n, h, u, IR, nullptr, (cudaStream_t)stream); });
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("master launch: ") + cudaGetErrorString(e));
    return FHD_OK;
}

static int keystream_one(const double *IR, double gamma, const fhd_params *params, uint32_t height, uint32_t width,
                         uint32_t channels, uint16_t *D, uint8_t *B, void *stream, bool trajectory) {
    if (!IR || !D || !B) return fail(nullptr, FHD_ERR_INVALID_ARG, "null argument");
    uint32_t n, u[4];
    double h;
    std::string why;
    if (!resolve_params(params, n, h, u, why)) return fail(nullptr, FHD_ERR_INVALID_ARG, why);
    if (!check_dims(height, width, channels, why)) return fail(nullptr, FHD_ERR_INVALID_ARG, why);
    static thread_local Batch b;
    std::memset(&b, 0, sizeof b);
    b.count = 1;
    b.n = n;
    b.hstep = h;
    b.hhalf = h / 2.0;
    b.hsixth = h / 6.0;
    FrameDesc &d = b.f[0];
    d.IR = const_cast<double *>(IR);
    d.D = D;
    d.B = B;
    d.gamma = gamma;
    d.h = height;
    d.w = width;
    d.C = channels;
    d.N = (uint64_t)height * width * channels;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (trajectory) {
        e = cudaMallocAsync(&d.T, fhd::traj_bytes((uint64_t)channels * (height + width), d.N, n), s);
        if (e != cudaSuccess) return fail(nullptr, FHD_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        e = timed(nullptr, FHD_K_KEYSTREAM, s, [&] { return fhd::launch_trajectory_keystream(b, s); });
        cudaFreeAsync(d.T, s);
    } else {
        e = timed(nullptr, FHD_K_KEYSTREAM, s, [&] { return fhd::launch_keystream(b, s); });
    }
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("keystream launch: ") + cudaGetErrorString(e));
    return FHD_OK;
}

int fhd_keystream(const double *IR, double gamma, const fhd_params *params, uint32_t height, uint32_t width,
                  uint32_t channels, uint16_t *D, uint8_t *B, void *stream) {
    return keystream_one(IR, gamma, params, height, width, channels, D, B, stream, false);
}

int fhd_keystream_trajectory(const double *IR, double gamma, const fhd_params *params, uint32_t height,
                             uint32_t width, uint32_t channels, uint16_t *D, uint8_t *B, void *stream) {
    return keystream_one(IR, gamma, params, height, width, channels, D, B, stream, true);
}

static int permute_one(const uint8_t *src, uint8_t *dst, uint32_t height, uint32_t width, uint32_t channels,
                       const uint16_t *D, const uint8_t *B, void *stream, bool encrypt) {
    if (!src || !dst || !D || !B) return fail(nullptr, FHD_ERR_INVALID_ARG, "null argument");
    std::string why;
    if (!check_dims(height, width, channels, why)) return fail(nullptr, FHD_ERR_INVALID_ARG, why);
    uint64_t N = (uint64_t)height * width * channels;
    if (src < dst + N && dst < src + N) return fail(nullptr, FHD_ERR_INVALID_ARG, "src and dst overlap");
    cudaError_t e = prepare_device();
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("prepare: ") + cudaGetErrorString(e));
    static thread_local Batch b;
    std::memset(&b, 0, sizeof b);
    b.count = 1;
    FrameDesc &d = b.f[0];
    d.src = src;
    d.dst = dst;
    d.D = const_cast<uint16_t *>(D);
    d.B = const_cast<uint8_t *>(B);
    d.h = height;
    d.w = width;
    d.C = channels;
    d.N = N;
    d.P = fhd::strip_width(height, width, channels);
    d.cta0 = 0;
    b.perm_ctas = fhd::permute_strips(width, d.P);
    d.RB = fhd::row_band(height, width, channels);
    d.rcta0 = 0;
    b.row_ctas = (height + d.RB - 1) / d.RB;
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMallocAsync(&d.G, N, s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    e = timed(nullptr, encrypt ? FHD_K_ENCRYPT : FHD_K_DECRYPT, s, [&] { return fhd::launch_permute(b, encrypt, s); });
    cudaFreeAsync(d.G, s);
    if (e != cudaSuccess) return fail(nullptr, FHD_ERR_CUDA, std::string("permute launch: ") + cudaGetErrorString(e));
    return FHD_OK;
}

int fhd_permute_encrypt(const uint8_t *src, uint8_t *dst, uint32_t height, uint32_t width, uint32_t channels,
                        const uint16_t *D, const uint8_t *B, void *stream) {
    return permute_one(src, dst, height, width, channels, D, B, stream, true);
}

int fhd_permute_decrypt(const uint8_t *src, uint8_t *dst, uint32_t height, uint32_t width, uint32_t channels,
                        const uint16_t *D, const uint8_t *B, void *stream) {
    return permute_one(src, dst, height, width, channels, D, B, stream, false);
}

uint32_t fhd_row_band(uint32_t height, uint32_t width, uint32_t channels) {
    if (!height || !width || !channels || channels > 4) return 0;
    return fhd::row_band(height, width, channels);
}

int fhd_set_cta_threads(uint32_t height, uint32_t width, uint32_t channels, uint32_t strip_threads,
                        uint32_t row_threads) {
    if (!height || !width || !channels || channels > 4 || (strip_threads && strip_threads != 256 && strip_threads != 512) ||
        (row_threads && row_threads != 128 && row_threads != 256))
        return fail(nullptr, FHD_ERR_INVALID_ARG, "bad CTA threads override");
    return fhd::set_cta_threads_override(height, width, channels, strip_threads, row_threads) == 0
               ? FHD_OK
               : fail(nullptr, FHD_ERR_TOO_LARGE, "override table full");
}

int fhd_cta_threads(uint32_t height, uint32_t width, uint32_t channels, uint32_t *strip_threads, uint32_t *row_threads) {
    if (!strip_threads || !row_threads) return fail(nullptr, FHD_ERR_INVALID_ARG, "null argument");
    if (!height || !width || !channels || channels > 4) return fail(nullptr, FHD_ERR_INVALID_ARG, "bad frame shape");
    fhd::cta_threads(height, width, channels, strip_threads, row_threads);
    return FHD_OK;
}

int fhd_set_row_band(uint32_t height, uint32_t width, uint32_t channels, uint32_t RB) {
    if (!height || !width || !channels || channels > 4 || RB > 64)
        return fail(nullptr, FHD_ERR_INVALID_ARG, "bad row band override");
    return fhd::set_row_band_override(height, width, channels, RB) == 0 ? FHD_OK
                                                                          : fail(nullptr, FHD_ERR_TOO_LARGE, "override table full");
}

uint32_t fhd_strip_width(uint32_t height, uint32_t width, uint32_t channels) {
    if (!height || !width || !channels || channels > 4) return 0;
    return fhd::strip_width(height, width, channels);
}

int fhd_set_strip_width(uint32_t height, uint32_t width, uint32_t channels, uint32_t P) {
    if (!height || !width || !channels || channels > 4 || P > 4096)
        return fail(nullptr, FHD_ERR_INVALID_ARG, "bad strip override");
    return fhd::set_strip_override(height, width, channels, P) == 0 ? FHD_OK
                                                                     : fail(nullptr, FHD_ERR_TOO_LARGE, "override table full");
}

}  // extern "C"
