// fhp_api.cu -- the extern "C" boundary declared in include/fhp.h.
//
// Owns lattice handles (geometry, device buffers, step counter, stream),
// validates arguments, turns CUDA errors into status codes and messages, and
// sequences the kernels of fhp_step.cu, fhp_pack.cu and fhp_coarse.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/fhp.h"
#include "fhp_debug.cuh"
#include "fhp_internal.h"

struct fhp_lattice {
    fhp::Geometry g;
    uint64_t seed = 0;
    double p = 0.0;
    fhp::ForcingTable ft{};
    bool force = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    bool owns_memory = false;
    uint8_t* base = nullptr;
    size_t bytes = 0;
    uint32_t* buf[2] = {nullptr, nullptr};
    uint32_t* solid = nullptr;
    unsigned int* flags = nullptr;  // device words: [0] any solid node, [1] kernel wait gave up
    uint8_t* staging = nullptr;
    size_t staging_bytes = 0;
    unsigned int* tile_done = nullptr;  // multi-step kernel: per-tile counters (H words)
    int cur = 0;
    int64_t t = 0;
    bool has_solid = false;
    int k_block = 1;
    int block_kernel = 0;          // temporal-block kernel: 0 automatic, 1 row wavefronts, 2 tiles
    int step_kernel = fhp::kStepAuto;
    int64_t launches = 0;
    std::string err;
};

namespace {

constexpr int64_t kMaxTime = (int64_t)1 << 48;
thread_local std::string g_create_error;

// Autotuned step configurations, per device and lattice shape.
struct TuneKey {
    int device, W, H;
    bool solid, force;
    int rules;
    bool operator==(const TuneKey& o) const {
        return device == o.device && W == o.W && H == o.H && solid == o.solid && force == o.force &&
               rules == o.rules;
    }
};
struct TuneChoice {
    int kernel;   // fhp::StepKernel other than kStepAuto
    int k;        // temporal block
    int bk;       // temporal-block kernel (0 automatic, 1 row wavefronts, 2 tiles)
};
std::mutex g_tune_mutex;
std::vector<std::pair<TuneKey, TuneChoice>> g_tuned;

bool tuned_choice(const TuneKey& key, TuneChoice* out) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (const auto& kv : g_tuned)
        if (kv.first == key) {
            *out = kv.second;
            return true;
        }
    return false;
}

void record_tuned(const TuneKey& key, const TuneChoice& c) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (auto& kv : g_tuned)
        if (kv.first == key) {
            kv.second = c;
            return;
        }
    g_tuned.emplace_back(key, c);
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int fail(fhp_lattice* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_create_error = buf;
    return code;
}

int cuda_fail(fhp_lattice* h, cudaError_t e, const char* what) {
    return fail(h, FHP_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool valid_size(int32_t W, int32_t H) {
    return W >= 32 && W % 32 == 0 && H >= 2 && H % 2 == 0 && (int64_t)W * H <= ((int64_t)1 << 40);
}

// Debug builds put a canary block of kCanaryBytes (filled with kCanaryByte)
// after every region of a lattice's device memory; fhp_debug_canaries checks
// them.  Release builds have none.
constexpr size_t kCanaryBytes = fhp::kDebugBuild ? 256 : 0;
constexpr unsigned char kCanaryByte = 0xA5;
constexpr int kRegions = 6;

struct Layout {
    size_t plane_bytes, state_bytes, state1_off, solid_off, flags_off, counters_off, staging_off, staging_bytes,
        total;
    size_t canary_off[kRegions];   // one canary after each region (debug builds)
};

Layout layout(int32_t W, int32_t H) {
    const fhp::Geometry g = fhp::make_geometry(W, H);
    Layout L;
    L.plane_bytes = round_up(g.plane_words * sizeof(uint32_t), 256);
    L.state_bytes = 7 * L.plane_bytes;
    L.canary_off[0] = L.state_bytes;
    L.state1_off = L.state_bytes + kCanaryBytes;
    L.canary_off[1] = L.state1_off + L.state_bytes;
    L.solid_off = L.canary_off[1] + kCanaryBytes;
    L.canary_off[2] = L.solid_off + L.plane_bytes;
    L.flags_off = L.canary_off[2] + kCanaryBytes;
    L.canary_off[3] = L.flags_off + 256;
    L.counters_off = L.canary_off[3] + kCanaryBytes;  // one word per row covers any tiling
    L.canary_off[4] = L.counters_off + round_up((size_t)H * sizeof(unsigned int), 256);
    L.staging_off = L.canary_off[4] + kCanaryBytes;
    // W*H bytes, and at least the resident kernel's exchange rows for two
    // ghost rows per side (2 parities x 2 sides x 9 row planes of Pq words for
    // each of up to min(H/4, 256) strips).
    const size_t ghost_exchange = (size_t)144 * (H / 4 < 256 ? H / 4 : 256) * g.Pq;
    L.staging_bytes = round_up((size_t)W * H > ghost_exchange ? (size_t)W * H : ghost_exchange, 256);
    L.canary_off[5] = L.staging_off + L.staging_bytes;
    L.total = L.canary_off[5] + kCanaryBytes;
    return L;
}

// Makes the lattice's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else if (prev == dev) prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Kernel and temporal block fhp_step uses: the lattice's own settings, or,
// while they are automatic (kernel 0, k = 1), the configuration autotuned
// for this shape if there is one, else the shared-memory resident kernel
// (exchanging every second step where the strips allow it) for lattices it
// holds whose multi-step ring would give fewer than two tiles per SM
// (launch-bound sizes, where it measured fastest: 1163 vs 957 GSUPS on
// 4096 x 1024, 1979 vs 1573 on 4096 x 2048).
void effective_settings(const fhp_lattice* h, int* kernel, int* k_block, int* bk = nullptr) {
    *kernel = h->step_kernel;
    *k_block = h->k_block;
    if (bk) *bk = h->block_kernel;
    if (h->step_kernel != fhp::kStepAuto || h->k_block != 1) return;
    TuneChoice c;
    if (tuned_choice(TuneKey{h->device, h->g.W, h->g.H, h->has_solid, h->force, h->g.rules}, &c)) {
        *kernel = c.kernel;
        *k_block = c.k;
        if (bk) *bk = c.bk;
        return;
    }
    const int resolved = fhp::resolved_step_kernel(h->g, h->has_solid, fhp::kStepAuto);
    const int tiles = fhp::run_tiles(h->g, h->has_solid);
    int dev_sms = 0;
    if (resolved == fhp::kStepRun && cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, h->device) ==
                                         cudaSuccess &&
        tiles < 2 * dev_sms && fhp::resident_supported(h->g, h->has_solid, h->staging_bytes)) {
        *kernel = fhp::kStepResident;
        *k_block = fhp::resident_supported(h->g, h->has_solid, h->staging_bytes, 2) ? 2 : 1;
    }
}

// Steps between exchanges of the resident kernel for these settings (2 when
// asked for and supported, else 1), or 0 if the resident kernel does not run.
int resident_interval(const fhp_lattice* h, int kernel, int k_block) {
    if (kernel != fhp::kStepResident) return 0;
    if (k_block == 2 && fhp::resident_supported(h->g, h->has_solid, h->staging_bytes, 2)) return 2;
    return fhp::resident_supported(h->g, h->has_solid, h->staging_bytes, 1) ? 1 : 0;
}

// Kernel of a temporally blocked pass of k steps for the requested kind
// (0 automatic, 1 row wavefronts, 2 tiles): 1 or 2, the other one where the
// requested kernel does not support the lattice, 0 if neither does (k = 1).
// Automatic takes the 2-D tiles where they apply: on GB300 they measured
// faster than the row wavefronts on every lattice tried (16384 x 4096,
// k = 2: 1815 against 1175 GSUPS), whose per-row hand-offs between warps
// leave most warps waiting.
int blocked_kind(const fhp_lattice* h, int k, int bk) {
    if (k <= 1) return 0;
    const bool wave = fhp::wave_supported(h->g, k), tiles = fhp::block_supported(h->g, k);
    if (bk == 1) return wave ? 1 : (tiles ? 2 : 0);
    return tiles ? 2 : (wave ? 1 : 0);
}

int check_block(fhp_lattice* h, int32_t B) {
    if (B < 32 || B % 32 != 0 || h->g.W % B != 0 || h->g.H % B != 0)
        return fail(h, FHP_EINVAL, "coarse-grain block %d must be a multiple of 32 dividing W=%d and H=%d",
                    B, h->g.W, h->g.H);
    return FHP_OK;
}

// Device-side error word: a bounded wait in a kernel gave up.  Reads it after
// the stream has drained, clears it, and reports FHP_ETIMEOUT if it was set.
int check_device_error(fhp_lattice* h) {
    unsigned int word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, h->flags + 1, sizeof word, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reading the device error word");
    if (word) {
        cudaMemsetAsync(h->flags + 1, 0, sizeof word, h->stream);
        cudaStreamSynchronize(h->stream);
        if (word & fhp::kErrBounds)
            return fail(h, FHP_EDEBUG, "a debug-build index check failed (site %u); the access was skipped",
                        (word >> 8) & 0xFFu);
        return fail(h, FHP_ETIMEOUT, "a step kernel gave up waiting for its input copies; the state is unreliable");
    }
    return FHP_OK;
}

int read_solid_flag(fhp_lattice* h) {
    unsigned int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, h->flags, sizeof flag, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reading the solid flag");
    h->has_solid = flag != 0;
    return check_device_error(h);
}

}  // namespace

void fhp::set_thread_error(const char* message) { g_create_error = message; }

fhp::ForcingTable fhp::forcing_table(double p) {
    const unsigned long long one = 1ULL << 32;
    unsigned long long P;
    const double scaled = std::ldexp(p, 32);   // exact: a power-of-two scaling
    if (!(scaled > 0.0)) {
        P = 0;
    } else if (scaled >= std::ldexp(1.0, 32)) {
        P = one;
    } else {
        // scaled < 2^32: its integer part fits, and scaled - floor(scaled) is exact.
        const unsigned long long ip = (unsigned long long)scaled;   // truncation = floor for scaled > 0
        const double frac = scaled - (double)ip;
        P = ip + ((frac > 0.5 || (frac == 0.5 && (ip & 1ull))) ? 1ull : 0ull);
    }
    fhp::ForcingTable ft;
    unsigned long long S = one;
    ft.p_plus_1 = P + 1;
    ft.q[0] = 0;
    for (int g = 1; g <= 32; ++g) {
        S = (unsigned long long)(((unsigned __int128)S * (one - P)) >> 32);
        ft.q[g] = one - S;
    }
    return ft;
}

extern "C" {

size_t fhp_required_bytes(int32_t width, int32_t height) {
    if (!valid_size(width, height)) return 0;
    return layout(width, height).total;
}

int fhp_create(fhp_lattice** out, const fhp_params* params) {
    if (!out) return fail(nullptr, FHP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params) return fail(nullptr, FHP_EINVAL, "params is NULL");
    const int32_t W = params->width, H = params->height;
    if (!valid_size(W, H))
        return fail(nullptr, FHP_EINVAL, "invalid lattice %d x %d: W must be a positive multiple of 32, H even >= 2",
                    W, H);
    if (!(params->forcing_p >= 0.0 && params->forcing_p <= 1.0))
        return fail(nullptr, FHP_EINVAL, "forcing probability %g outside [0, 1]", params->forcing_p);
    fhp_lattice* h = new (std::nothrow) fhp_lattice();
    if (!h) return fail(nullptr, FHP_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail(nullptr, FHP_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    }
    h->g = fhp::make_geometry(W, H);
    h->seed = params->seed;
    h->p = params->forcing_p;
    h->ft = fhp::forcing_table(h->p);
    h->force = h->ft.q[32] != 0;
    h->stream = (cudaStream_t)params->stream;
    const Layout L = layout(W, H);
    if (params->device_memory) {
        if (params->device_memory_bytes < L.total || ((uintptr_t)params->device_memory & 255u)) {
            delete h;
            return fail(nullptr, FHP_ENOMEM, "device_memory must be 256-byte aligned and hold %zu bytes (got %zu)",
                        L.total, params->device_memory_bytes);
        }
        h->base = (uint8_t*)params->device_memory;
        h->owns_memory = false;
    } else {
        e = cudaMalloc((void**)&h->base, L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return fail(nullptr, FHP_ENOMEM, "cudaMalloc(%zu): %s", L.total, cudaGetErrorString(e));
        }
        h->owns_memory = true;
    }
    h->bytes = L.total;
    h->buf[0] = (uint32_t*)h->base;
    h->buf[1] = (uint32_t*)(h->base + L.state1_off);
    h->solid = (uint32_t*)(h->base + L.solid_off);
    h->flags = (unsigned int*)(h->base + L.flags_off);
    h->tile_done = (unsigned int*)(h->base + L.counters_off);
    h->staging = h->base + L.staging_off;
    h->staging_bytes = L.staging_bytes;
    // Empty fluid lattice: zero both buffers and the solid plane.
    e = cudaMemsetAsync(h->base, 0, L.staging_off, h->stream);
    for (int r = 0; r < kRegions && kCanaryBytes && e == cudaSuccess; ++r)
        e = cudaMemsetAsync(h->base + L.canary_off[r], kCanaryByte, kCanaryBytes, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        if (h->owns_memory) cudaFree(h->base);
        delete h;
        return fail(nullptr, FHP_ECUDA, "initialising device memory: %s", cudaGetErrorString(e));
    }
    *out = h;
    return FHP_OK;
}

void fhp_destroy(fhp_lattice* h) {
    if (!h) return;
    DeviceGuard dg(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->owns_memory && h->base) cudaFree(h->base);
    delete h;
}

const char* fhp_last_error(const fhp_lattice* h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

int fhp_set_state(fhp_lattice* h, const uint8_t* host_bytes) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (!host_bytes) return fail(h, FHP_EINVAL, "host_bytes is NULL");
    DeviceGuard dg(h->device);
    const size_t n = (size_t)h->g.W * h->g.H;
    cudaError_t e = cudaMemcpyAsync(h->staging, host_bytes, n, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "copying the state to the device");
    return fhp_set_state_device(h, h->staging);
}

int fhp_set_state_device(fhp_lattice* h, const uint8_t* device_bytes) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (!device_bytes) return fail(h, FHP_EINVAL, "device_bytes is NULL");
    DeviceGuard dg(h->device);
    cudaError_t e = cudaMemsetAsync(h->flags, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess) e = fhp::launch_pack(h->g, device_bytes, h->buf[h->cur], h->solid, h->flags, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "packing the state");
    ++h->launches;
    return read_solid_flag(h);
}

int fhp_get_state(fhp_lattice* h, uint8_t* host_bytes) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (!host_bytes) return fail(h, FHP_EINVAL, "host_bytes is NULL");
    DeviceGuard dg(h->device);
    int rc = fhp_get_state_device(h, h->staging);
    if (rc != FHP_OK) return rc;
    const size_t n = (size_t)h->g.W * h->g.H;
    cudaError_t e = cudaMemcpyAsync(host_bytes, h->staging, n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "copying the state to the host");
    return check_device_error(h);
}

int fhp_get_state_device(fhp_lattice* h, uint8_t* device_bytes) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (!device_bytes) return fail(h, FHP_EINVAL, "device_bytes is NULL");
    DeviceGuard dg(h->device);
    cudaError_t e = fhp::launch_unpack(h->g, h->buf[h->cur], h->solid, device_bytes, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "unpacking the state");
    ++h->launches;
    return FHP_OK;
}

int fhp_load_obstacles(fhp_lattice* h, const uint8_t* host_mask) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (!host_mask) return fail(h, FHP_EINVAL, "host_mask is NULL");
    DeviceGuard dg(h->device);
    const size_t n = (size_t)h->g.W * h->g.H;
    cudaError_t e = cudaMemcpyAsync(h->staging, host_mask, n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->flags, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess)
        e = fhp::launch_load_obstacles(h->g, h->staging, h->buf[h->cur], h->solid, h->flags, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "loading obstacles");
    ++h->launches;
    return read_solid_flag(h);
}

namespace {
// Validates and copies shapes; returns false (with the lattice's message) if invalid.
bool shape_list(const fhp_shape* shapes, int32_t count, fhp::ShapeList* out, bool* any) {
    if (count < 0 || count > FHP_MAX_SHAPES || (count > 0 && !shapes)) return false;
    out->n = count;
    *any = false;
    for (int i = 0; i < count; ++i) {
        const fhp_shape& s = shapes[i];
        if (s.kind != FHP_SHAPE_DISC && s.kind != FHP_SHAPE_ROWS) return false;
        if (s.kind == FHP_SHAPE_DISC && s.c < 0) return false;
        out->s[i] = fhp::Shape{s.kind, s.a, s.b, s.c};
    }
    return true;
}
}  // namespace

int fhp_load_obstacle_shapes(fhp_lattice* h, const fhp_shape* shapes, int32_t count) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    fhp::ShapeList list{};
    bool any;
    if (!shape_list(shapes, count, &list, &any))
        return fail(h, FHP_EINVAL, "invalid shape list (count %d, at most %d, kinds DISC or ROWS)", count,
                    FHP_MAX_SHAPES);
    DeviceGuard dg(h->device);
    cudaError_t e = cudaMemsetAsync(h->flags, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess)
        e = fhp::launch_obstacle_shapes(h->g, list, h->buf[h->cur], h->solid, h->flags, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "generating obstacles");
    ++h->launches;
    return read_solid_flag(h);
}

int fhp_init_random(fhp_lattice* h, double density) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (!(density >= 0.0 && density <= 1.0)) return fail(h, FHP_EINVAL, "density %g outside [0, 1]", density);
    DeviceGuard dg(h->device);
    cudaError_t e = fhp::launch_init_random(h->g, h->buf[h->cur], h->solid, h->has_solid, h->seed, density,
                                            h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "launching the init kernel");
    ++h->launches;
    return FHP_OK;
}

namespace {
// NVTX range for the duration of an API call (visible in Nsight tools; a
// no-op without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

int fhp_step(fhp_lattice* h, int64_t n) {
    NvtxRange nvtx("fhp_step");
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (n < 0) return fail(h, FHP_EINVAL, "negative step count %lld", (long long)n);
    if (n > kMaxTime - h->t) return fail(h, FHP_EINVAL, "step counter would pass 2^48");
    DeviceGuard dg(h->device);
    const fhp::Key2 key{(uint32_t)h->seed, (uint32_t)(h->seed >> 32)};
    int kernel = h->step_kernel, k_block = h->k_block, bk = h->block_kernel;
    effective_settings(h, &kernel, &k_block, &bk);
    const int gh = resident_interval(h, kernel, k_block);
    if (gh > 0) {
        // The lattice stays in shared memory for launches of up to 2^24 steps
        // (exchange rows in the byte-staging area, step counters in the tile
        // counters).
        int64_t left = n;
        while (left > 0) {
            const int chunk = (int)(left < (1 << 24) ? left : (1 << 24));
            cudaError_t e = fhp::launch_resident(h->g, h->buf[h->cur], h->buf[h->cur ^ 1], h->solid, h->has_solid,
                                                 h->force, h->ft, key, (uint64_t)h->t, chunk, gh,
                                                 reinterpret_cast<uint32_t*>(h->staging), h->tile_done, h->stream,
                                                 h->flags + 1);
            if (e != cudaSuccess) return cuda_fail(h, e, "launching the resident kernel");
            ++h->launches;
            h->cur ^= (chunk & 1);
            h->t += chunk;
            left -= chunk;
        }
        return FHP_OK;
    }
    if (kernel == fhp::kStepResident) kernel = fhp::kStepAuto;  // not supported for this lattice
    const int blocked = blocked_kind(h, k_block, bk);
    if (blocked != 0) {
        const bool wave = blocked == 1;
        // Temporal blocking: passes of k steps (row wavefronts where the rows
        // fit shared memory, else 2-D tiles); the remainder one step at a time.
        const int k = k_block;
        while (n >= k) {
            cudaError_t e = wave ? fhp::launch_wave(h->g, h->buf[h->cur], h->buf[h->cur ^ 1], h->solid,
                                                    h->has_solid, h->force, h->ft, key, (uint64_t)h->t, k,
                                                    h->stream, h->flags + 1)
                                 : fhp::launch_block(h->g, h->buf[h->cur], h->buf[h->cur ^ 1], h->solid,
                                                     h->has_solid, h->force, h->ft, key, (uint64_t)h->t, k,
                                                     h->stream, h->flags + 1);
            if (e != cudaSuccess) return cuda_fail(h, e, "launching the temporally blocked kernel");
            ++h->launches;
            h->cur ^= 1;
            h->t += k;
            n -= k;
        }
    }
    if (n >= 2 && fhp::resolved_step_kernel(h->g, h->has_solid, kernel) == fhp::kStepRun) {
        // All n steps in cooperative launches of up to 2^24 steps each.
        int64_t left = n;
        while (left > 0) {
            const int chunk = (int)(left < (1 << 24) ? left : (1 << 24));
            cudaError_t e = fhp::launch_run(h->g, h->buf[h->cur], h->buf[h->cur ^ 1], h->solid, h->has_solid,
                                            h->force, h->ft, key, (uint64_t)h->t, chunk, h->tile_done,
                                            h->stream, h->flags + 1);
            if (e != cudaSuccess) return cuda_fail(h, e, "launching the multi-step kernel");
            ++h->launches;
            h->cur ^= (chunk & 1);
            h->t += chunk;
            left -= chunk;
        }
        return FHP_OK;
    }
    for (int64_t i = 0; i < n; ++i) {
        cudaError_t e = fhp::launch_step(h->g, h->buf[h->cur], h->buf[h->cur ^ 1], h->solid, h->has_solid,
                                         h->force, h->ft, key, (uint64_t)h->t, h->stream, h->flags + 1,
                                         kernel);
        if (e != cudaSuccess) return cuda_fail(h, e, "launching the step kernel");
        ++h->launches;
        h->cur ^= 1;
        ++h->t;
    }
    return FHP_OK;
}

int fhp_coarse_grain(fhp_lattice* h, int32_t block, int32_t* counts, float* rho, float* ux, float* uy) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    int rc = check_block(h, block);
    if (rc != FHP_OK) return rc;
    DeviceGuard dg(h->device);
    const size_t cells = (size_t)(h->g.W / block) * (h->g.H / block);
    int32_t* d_counts = (int32_t*)h->staging;
    float* d_rho = (float*)(h->staging + round_up(cells * 9 * sizeof(int32_t), 256));
    float* d_ux = (float*)((uint8_t*)d_rho + round_up(cells * sizeof(float), 256));
    float* d_uy = (float*)((uint8_t*)d_ux + round_up(cells * sizeof(float), 256));
    rc = fhp_coarse_grain_device(h, block, d_counts, d_rho, d_ux, d_uy);
    if (rc != FHP_OK) return rc;
    cudaError_t e = cudaSuccess;
    if (counts && e == cudaSuccess)
        e = cudaMemcpyAsync(counts, d_counts, cells * 9 * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    if (rho && e == cudaSuccess)
        e = cudaMemcpyAsync(rho, d_rho, cells * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (ux && e == cudaSuccess)
        e = cudaMemcpyAsync(ux, d_ux, cells * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (uy && e == cudaSuccess)
        e = cudaMemcpyAsync(uy, d_uy, cells * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "copying coarse-grained fields to the host");
    return check_device_error(h);
}

int fhp_coarse_grain_device(fhp_lattice* h, int32_t block, int32_t* counts, float* rho, float* ux, float* uy) {
    NvtxRange nvtx("fhp_coarse_grain");
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    int rc = check_block(h, block);
    if (rc != FHP_OK) return rc;
    if (!counts || !rho || !ux || !uy) return fail(h, FHP_EINVAL, "device outputs must not be NULL");
    DeviceGuard dg(h->device);
    cudaError_t e = fhp::launch_coarse_grain(h->g, h->buf[h->cur], h->solid, h->has_solid, block, counts, rho,
                                             ux, uy, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "launching the coarse-grain kernel");
    ++h->launches;
    return FHP_OK;
}

int64_t fhp_get_time(const fhp_lattice* h) { return h ? h->t : -1; }

int fhp_set_time(fhp_lattice* h, int64_t t) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (t < 0 || t >= kMaxTime) return fail(h, FHP_EINVAL, "step counter %lld outside [0, 2^48)", (long long)t);
    h->t = t;
    return FHP_OK;
}

int fhp_set_forcing(fhp_lattice* h, double p) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (!(p >= 0.0 && p <= 1.0)) return fail(h, FHP_EINVAL, "forcing probability %g outside [0, 1]", p);
    h->p = p;
    h->ft = fhp::forcing_table(p);
    h->force = h->ft.q[32] != 0;
    return FHP_OK;
}

int fhp_set_temporal_block(fhp_lattice* h, int32_t k) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (k != 1 && k != 2 && k != 3 && k != 4 && k != 8)
        return fail(h, FHP_EINVAL, "temporal block %d not in {1, 2, 3, 4, 8}", k);
    h->k_block = k;
    return FHP_OK;
}

int fhp_set_step_kernel(fhp_lattice* h, int32_t kind) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (kind < 0 || kind > 4) return fail(h, FHP_EINVAL, "step kernel %d not in {0, 1, 2, 3, 4}", kind);
    h->step_kernel = kind;
    return FHP_OK;
}

int fhp_get_step_kernel(const fhp_lattice* h) {
    if (!h) return -1;
    DeviceGuard dg(h->device);
    int kernel, k_block;
    effective_settings(h, &kernel, &k_block);
    if (kernel == fhp::kStepResident)
        return fhp::resident_supported(h->g, h->has_solid, h->staging_bytes)
                   ? fhp::kStepResident
                   : fhp::resolved_step_kernel(h->g, h->has_solid, fhp::kStepAuto);
    return fhp::resolved_step_kernel(h->g, h->has_solid, kernel);
}

int fhp_set_rules(fhp_lattice* h, int32_t rules) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (rules != FHP_RULES_FHP_I && rules != FHP_RULES_FHP_II && rules != FHP_RULES_FHP_III)
        return fail(h, FHP_EINVAL, "rule set %d is not FHP_RULES_FHP_I (1), _II (2) or _III (3)", rules);
    h->g.rules = rules;
    return FHP_OK;
}

int fhp_get_rules(const fhp_lattice* h) { return h ? h->g.rules : -1; }

int fhp_set_row_offset(fhp_lattice* h, int32_t row_base) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (row_base % 2) return fail(h, FHP_EINVAL, "row offset %d must be even", row_base);
    h->g.row_base = row_base;
    return FHP_OK;
}

int32_t fhp_row_pitch_words(const fhp_lattice* h) { return h ? h->g.Pq : -1; }

namespace {
// Rows [y0, y0 + n) of the 7 state planes to or from a packed device buffer
// [plane][row][word] of 7 * n * Pq words.
int copy_rows(fhp_lattice* h, int32_t y0, int32_t n, uint32_t* packed, bool to_lattice) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (!packed || y0 < 0 || n < 0 || (int64_t)y0 + n > h->g.H)
        return fail(h, FHP_EINVAL, "rows [%d, %d) outside the lattice's %d rows or NULL buffer", y0, y0 + n, h->g.H);
    if (n == 0) return FHP_OK;
    DeviceGuard dg(h->device);
    const size_t row_words = (size_t)h->g.Pq;
    for (int p = 0; p < 7; ++p) {
        uint32_t* plane = h->buf[h->cur] + (size_t)p * h->g.plane_words + (size_t)y0 * row_words;
        uint32_t* buf = packed + (size_t)p * n * row_words;
        cudaError_t e = to_lattice ? cudaMemcpyAsync(plane, buf, n * row_words * 4, cudaMemcpyDeviceToDevice, h->stream)
                                   : cudaMemcpyAsync(buf, plane, n * row_words * 4, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "copying rows");
    }
    return FHP_OK;
}
}  // namespace

int fhp_get_rows_device(fhp_lattice* h, int32_t y0, int32_t n, uint32_t* device_words) {
    return copy_rows(h, y0, n, device_words, false);
}

int fhp_set_rows_device(fhp_lattice* h, int32_t y0, int32_t n, const uint32_t* device_words) {
    return copy_rows(h, y0, n, const_cast<uint32_t*>(device_words), true);
}

int fhp_get_temporal_block(const fhp_lattice* h) {
    if (!h) return -1;
    int kernel, k_block, bk;
    effective_settings(h, &kernel, &k_block, &bk);
    const int gh = resident_interval(h, kernel, k_block);
    if (gh > 0) return gh;
    return blocked_kind(h, k_block, bk) != 0 ? k_block : 1;
}

int fhp_set_temporal_block_kernel(fhp_lattice* h, int32_t kind) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (kind < 0 || kind > 2) return fail(h, FHP_EINVAL, "temporal-block kernel %d not in {0, 1, 2}", kind);
    h->block_kernel = kind;
    return FHP_OK;
}

int fhp_get_temporal_block_kernel(const fhp_lattice* h) {
    if (!h) return -1;
    int kernel, k_block, bk;
    effective_settings(h, &kernel, &k_block, &bk);
    if (resident_interval(h, kernel, k_block) > 0) return 0;
    return blocked_kind(h, k_block, bk);
}

int fhp_autotune(fhp_lattice* h, int32_t trial_steps, int32_t* out_kernel, int32_t* out_temporal_block) {
    NvtxRange nvtx("fhp_autotune");
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    if (trial_steps < 8 || trial_steps > 4096 || trial_steps % 8)
        return fail(h, FHP_EINVAL, "trial_steps %d must be a multiple of 8 in [8, 4096]", trial_steps);
    DeviceGuard dg(h->device);
    int rc = fhp_synchronize(h);
    if (rc != FHP_OK) return rc;
    // The trials start from a saved copy of the state, restored afterwards.
    const size_t state_bytes = (size_t)7 * h->g.plane_words * sizeof(uint32_t);
    uint32_t* saved = nullptr;
    cudaError_t e = cudaMalloc((void**)&saved, state_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, FHP_ENOMEM, "autotune: no room for a copy of the state (%zu bytes)", state_bytes);
    }
    const int cur0 = h->cur;
    const int64_t t0 = h->t;
    const int kernel0 = h->step_kernel, k0 = h->k_block, bk0 = h->block_kernel;
    e = cudaMemcpyAsync(saved, h->buf[cur0], state_bytes, cudaMemcpyDeviceToDevice, h->stream);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    std::vector<TuneChoice> cands;
    cands.push_back({fhp::kStepDirect, 1, 0});
    if (fhp::resolved_step_kernel(h->g, h->has_solid, fhp::kStepRing) != fhp::kStepDirect) {
        cands.push_back({fhp::kStepRing, 1, 0});
        cands.push_back({fhp::kStepRun, 1, 0});
    }
    if (fhp::resident_supported(h->g, h->has_solid, h->staging_bytes, 1))
        cands.push_back({fhp::kStepResident, 1, 0});
    if (fhp::resident_supported(h->g, h->has_solid, h->staging_bytes, 2))
        cands.push_back({fhp::kStepResident, 2, 0});
    // Temporal blocks (trial_steps mod k steps run one at a time): row
    // wavefronts and 2-D tiles, where each supports the lattice.
    for (int k : {2, 3, 4})
        if (fhp::wave_supported(h->g, k)) cands.push_back({fhp::kStepDirect, k, 1});
    for (int k : {2, 4, 8})
        if (fhp::block_supported(h->g, k)) cands.push_back({fhp::kStepDirect, k, 2});
    TuneChoice best{fhp::kStepDirect, 1, 0};
    float best_ms = -1.0f;
    for (size_t i = 0; e == cudaSuccess && i < cands.size(); ++i) {
        h->step_kernel = cands[i].kernel;
        h->k_block = cands[i].k;
        h->block_kernel = cands[i].bk;
        // One untimed trial (first-use set-up), then the timed one.
        rc = fhp_step(h, trial_steps);
        if (rc == FHP_OK) rc = fhp_synchronize(h);
        if (rc == FHP_OK) {
            e = cudaEventRecord(ev[0], h->stream);
            if (e == cudaSuccess) rc = fhp_step(h, trial_steps);
            if (e == cudaSuccess && rc == FHP_OK) e = cudaEventRecord(ev[1], h->stream);
            if (e == cudaSuccess && rc == FHP_OK) rc = fhp_synchronize(h);
            float ms = 0.0f;
            if (e == cudaSuccess && rc == FHP_OK) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (e == cudaSuccess && rc == FHP_OK && (best_ms < 0.0f || ms < best_ms)) {
                best_ms = ms;
                best = cands[i];
            }
        }
        if (rc != FHP_OK || e != cudaSuccess) {
            // A candidate that cannot launch is skipped; a failure the device
            // reported (a wait that gave up, a sticky CUDA error) ends the tuning.
            if (rc == FHP_ETIMEOUT) break;
            cudaGetLastError();
            const cudaError_t se = cudaStreamSynchronize(h->stream);
            if (se != cudaSuccess) {
                e = se;
                break;
            }
            e = cudaSuccess;
            rc = FHP_OK;
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->buf[cur0], saved, state_bytes, cudaMemcpyDeviceToDevice, h->stream);
        h->cur = cur0;
        h->t = t0;
    }
    if (e == cudaSuccess && rc == FHP_OK) e = cudaStreamSynchronize(h->stream);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    cudaFree(saved);
    h->cur = cur0;
    h->t = t0;
    if (rc != FHP_OK || e != cudaSuccess || best_ms < 0.0f) {
        h->step_kernel = kernel0;
        h->k_block = k0;
        h->block_kernel = bk0;
        if (rc != FHP_OK) return rc;
        if (e != cudaSuccess) return cuda_fail(h, e, "autotuning");
        return fail(h, FHP_ECUDA, "autotune: no step configuration ran");
    }
    // Keep the lattice automatic; the choice applies to every lattice of this
    // shape (and obstacle / forcing flags) on this device.
    h->step_kernel = fhp::kStepAuto;
    h->k_block = 1;
    h->block_kernel = 0;
    record_tuned(TuneKey{h->device, h->g.W, h->g.H, h->has_solid, h->force, h->g.rules}, best);
    if (out_kernel) *out_kernel = best.kernel;
    if (out_temporal_block) *out_temporal_block = best.k;
    return FHP_OK;
}

int fhp_synchronize(fhp_lattice* h) {
    if (!h) return fail(nullptr, FHP_EINVAL, "lattice is NULL");
    DeviceGuard dg(h->device);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "synchronizing");
    return check_device_error(h);
}

int64_t fhp_kernel_launches(const fhp_lattice* h) { return h ? h->launches : -1; }

int fhp_debug_build(void) { return fhp::kDebugBuild ? 1 : 0; }

int fhp_debug_canaries(fhp_lattice* h, int32_t* checked, int32_t* corrupted) {
    if (!h || !checked || !corrupted) return fail(h, FHP_EINVAL, "NULL argument");
    *checked = 0;
    *corrupted = 0;
    if (!kCanaryBytes) return FHP_OK;
    DeviceGuard dg(h->device);
    const Layout L = layout(h->g.W, h->g.H);
    std::vector<unsigned char> buf(kCanaryBytes);
    for (int r = 0; r < kRegions; ++r) {
        cudaError_t e = cudaMemcpyAsync(buf.data(), h->base + L.canary_off[r], kCanaryBytes, cudaMemcpyDeviceToHost,
                                        h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "reading a canary");
        ++*checked;
        for (unsigned char c : buf)
            if (c != kCanaryByte) {
                ++*corrupted;
                break;
            }
    }
    return FHP_OK;
}

int fhp_philox4x32_10_device(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, void* stream) {
    if (!ctr || !key || !out || n < 0) return fail(nullptr, FHP_EINVAL, "invalid Philox arguments");
    if (n == 0) return FHP_OK;
    cudaError_t e = fhp::launch_philox(ctr, key, out, n, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(nullptr, FHP_ECUDA, "Philox kernel: %s", cudaGetErrorString(e));
    return FHP_OK;
}

}  // extern "C"
