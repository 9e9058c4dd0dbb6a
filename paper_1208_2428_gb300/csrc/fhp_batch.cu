// fhp_batch.cu -- many independent FHP lattices advanced by shared launches.
//
// A batch owns one device arena.  Member lattices (any sizes, seeds, forcing
// probabilities, obstacle maps) are carved out of it and may join or leave
// between calls.  fhp_batch_step(n) advances every member by
// min(n, its step budget) steps; each step is ONE launch of fhp_batch_kernel
// over a tile list that spans all members, and the per-step launches are
// replayed from a captured CUDA graph.
//
// fhp_batch_kernel is the warp-specialised ring of the single-lattice path
// (producer warp streaming row tiles into a 3-stage shared-memory ring with
// cp.async.bulk, 8 consumer warps computing), except that every tile may
// belong to a different lattice: the producer copies that lattice's
// descriptor (geometry, buffers, generator key, step, forcing table) into a
// per-stage header in shared memory, and the consumers run the same per-quad
// code against it.  Members whose budget is used up are skipped.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/fhp.h"
#include "fhp_arena.h"
#include "fhp_debug.cuh"
#include "fhp_device.cuh"
#include "fhp_internal.h"
#include "fhp_quad.cuh"

namespace fhp {
namespace {

constexpr int kBConsumerWarps = 8;
constexpr int kBThreads = (kBConsumerWarps + 1) * 32;       // + producer warp
constexpr int kBRunThreads = (kBConsumerWarps + 2) * 32;    // + producer and publisher warps
constexpr int kBStages = 3;
constexpr int kBStageBudget = 32 * 1024;

// Device descriptor of one member lattice.
struct BatchLattice {
    StepArgs a;               // geometry, solid plane, key, forcing table, err
    TileArgs ta;              // rows per tile (ntiles unused)
    uint32_t* buf[2];
    unsigned long long t0;    // step counter at the start of the current call
    int cur;                  // buffer holding S_{t0}
    int steps;                // steps in the current call (0: idle)
    int force;
    int tile_base;            // index of the lattice's tile 0 in the tile list
};

struct BatchTile {
    int lattice;
    int tile;                 // row tile index within the lattice
};

// Written by the producer warp for every staged tile.
struct __align__(16) StageHeader {
    StepArgs a;               // with src/dst/t of this step
    TileArgs ta;
    int tile;
    int active;
    int force;
    int pad;
};

constexpr int kHeaderBytes = (int)((sizeof(StageHeader) + 127) / 128 * 128);
constexpr int kDescWords = (int)(sizeof(StepArgs) / 4);
constexpr int kDescRegs = (kDescWords + 31) / 32;
static_assert(sizeof(StepArgs) % 4 == 0, "StepArgs is copied as 32-bit words");
constexpr int kBPrefixBytes = 128 + kBStages * kHeaderBytes;  // barriers, then headers

// Producer-side copy of one lattice's descriptor: word w of its StepArgs in
// register w / 32 of lane w mod 32, the per-call fields in lane 0.
struct DescCache {
    int lat = -1;
    uint32_t dw[kDescRegs];
    int steps = 0, cur = 0, force = 0, tile_base = 0;
    unsigned long long t0 = 0;
    uint32_t* buf0 = nullptr;
    uint32_t* buf1 = nullptr;
    TileArgs ta{};
};

__device__ __forceinline__ void load_desc(DescCache& c, const BatchLattice* __restrict__ lats, int lat, int lane) {
    const BatchLattice* L = lats + lat;
    const uint32_t* srcw = reinterpret_cast<const uint32_t*>(&L->a);
#pragma unroll
    for (int j = 0; j < kDescRegs; ++j) {
        const int w = lane + 32 * j;
        c.dw[j] = w < kDescWords ? srcw[w] : 0u;
    }
    if (lane == 0) {
        c.steps = L->steps;
        c.cur = L->cur;
        c.force = L->force;
        c.tile_base = L->tile_base;
        c.t0 = L->t0;
        c.buf0 = L->buf[0];
        c.buf1 = L->buf[1];
        c.ta = L->ta;
    }
    c.lat = lat;
}

// All lanes write the descriptor words into the stage header, then lane 0
// fills in the fields of step s and tile `tile`.
__device__ __forceinline__ void write_header(StageHeader* h, const DescCache& c, int s, int tile, unsigned int* err,
                                             int lane) {
    uint32_t* dstw = reinterpret_cast<uint32_t*>(&h->a);
#pragma unroll
    for (int j = 0; j < kDescRegs; ++j) {
        const int w = lane + 32 * j;
        if (w < kDescWords) dstw[w] = c.dw[j];
    }
    __syncwarp();
    if (lane == 0) {
        const int par = (c.cur + s) & 1;
        const unsigned long long t = c.t0 + (unsigned long long)s;
        h->a.src = par ? c.buf1 : c.buf0;
        h->a.dst = par ? c.buf0 : c.buf1;
        h->a.t_lo = (uint32_t)t;
        h->a.t_hi = (uint32_t)(t >> 32);
        h->a.err = err;
        h->ta = c.ta;
        h->tile = tile;
        h->active = s < c.steps && dbg_ok(tile >= 0 && tile < c.ta.ntiles, err, kSiteBatchTile) &&
                    dbg_ok(8LL * c.ta.R * h->a.Pq * 4 <= kBStageBudget, err, kSiteStageFit);
        h->force = c.force;
    }
}

template <bool FORCE>
__device__ __forceinline__ void batch_compute(const StageHeader& h, const uint32_t* stage) {
    const StepVar v{h.a.dst, h.a.t_lo, h.a.t_hi};
    compute_tile<true, FORCE, true>(h.a, v, h.ta, h.tile, stage, (int)threadIdx.x, kBConsumerWarps * 32);
}

__global__ void __launch_bounds__(kBThreads, 2)
    fhp_batch_kernel(const BatchLattice* __restrict__ lats, const BatchTile* __restrict__ tiles,
                     const int* __restrict__ step_base, int step_offset, unsigned int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + kBStages;
    StageHeader* headers = reinterpret_cast<StageHeader*>(smem_raw + 128);
    uint32_t* stages = reinterpret_cast<uint32_t*>(smem_raw + kBPrefixBytes);
    const int stage_words = kBStageBudget / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // step_base[0]: steps of the current call already done by earlier graph
    // replays; step_base[1]: number of tiles.  Both live in device memory so
    // that a captured graph stays valid when members join or leave.
    const int ntiles = step_base[1];
    // Each CTA takes a contiguous run of the tile list, so consecutive tiles
    // mostly belong to the same lattice and its descriptor is loaded once.
    const int first = (int)(((long long)blockIdx.x * ntiles) / gridDim.x);
    const int count = (int)(((long long)(blockIdx.x + 1) * ntiles) / gridDim.x) - first;
    const int s = step_base[0] + step_offset;  // step index within the current call

    if (threadIdx.x == 0) {
        for (int k = 0; k < kBStages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kBConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kBConsumerWarps) {
        // The producer keeps the current lattice's descriptor in registers
        // and reloads it only when the tile list moves on to another
        // lattice; tile records are fetched 32 at a time.
        bool ok = true;
        int i = 0;
        DescCache c;
        BatchTile rec{0, 0};
        for (; i < count; ++i) {
            const int st = i % kBStages;
            if ((i & 31) == 0 && i + lane < count) rec = tiles[first + i + lane];
            const int bt_lat = __shfl_sync(0xFFFFFFFFu, rec.lattice, i & 31);
            const int bt_tile = __shfl_sync(0xFFFFFFFFu, rec.tile, i & 31);
            if (bt_lat != c.lat) load_desc(c, lats, bt_lat, lane);
            int waited = 1;
            if (lane == 0 && i >= kBStages)
                waited = mbar_wait_bounded(&empty[st], (uint32_t)(((i / kBStages) - 1) & 1)) ? 1 : 0;
            if (!__shfl_sync(0xFFFFFFFFu, waited, 0)) {
                ok = false;
                break;
            }
            __syncwarp();  // order lane 0's acquire of "empty" before the lanes rewrite the header
            StageHeader* h = headers + st;
            write_header(h, c, s, bt_tile, err, lane);
            if (lane == 0) {
                if (h->active) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue_tile<true>(h->a, h->ta, h->a.src, bt_tile, stages + (size_t)st * stage_words, &full[st]);
                } else {
                    mbar_arrive_expect_tx(&full[st], 0u);  // nothing to stage: release the stage at once
                }
            }
            __syncwarp();
        }
        if (lane == 0) {
            if (!ok && err) atomicOr(err, 1u);
            for (int k = (i > kBStages ? i - kBStages : 0); k < i; ++k)
                (void)mbar_wait_bounded(&full[k % kBStages], (uint32_t)((k / kBStages) & 1));
        }
        return;
    }

    for (int i = 0; i < count; ++i) {
        const int st = i % kBStages;
        if (!mbar_wait_bounded(&full[st], (uint32_t)((i / kBStages) & 1))) {
            if (lane == 0 && err) atomicOr(err, 1u);
            return;
        }
        const StageHeader& h = headers[st];
        if (h.active) {
            if (h.force) batch_compute<true>(h, stages + (size_t)st * stage_words);
            else batch_compute<false>(h, stages + (size_t)st * stage_words);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
    }
}

// All steps of a batch call in one cooperative launch.  As in the
// single-lattice multi-step kernel, a tile may be staged for step s once the
// tiles of the previous step whose rows it reads -- the tile and its two
// neighbours within the same lattice (periodic in y) -- are finished: the
// publisher warp bumps a tile's counter by kBConsumerWarps after one
// GPU-scope fence when all consumer warps are done with it, and the producer
// waits for the counters (bounded) before issuing the bulk copies.  Every
// CTA handles its contiguous run of the tile list step after step, and all
// CTAs are resident (cooperative launch), so every wait ends.  Members whose
// budget ends within the call are skipped for the remaining steps.
__global__ void __launch_bounds__(kBRunThreads, 2)
    fhp_batch_run_kernel(const BatchLattice* __restrict__ lats, const BatchTile* __restrict__ tiles, int ntiles,
                         int nsteps, unsigned int* __restrict__ done, unsigned int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + kBStages;
    unsigned int* warp_done = reinterpret_cast<unsigned int*>(empty + kBStages);
    StageHeader* headers = reinterpret_cast<StageHeader*>(smem_raw + 128);
    uint32_t* stages = reinterpret_cast<uint32_t*>(smem_raw + kBPrefixBytes);
    const int stage_words = kBStageBudget / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Item i of the CTA is tile list entry blockIdx.x + i * gridDim.x: the
    // neighbours a tile waits for are handled at the same position by the
    // neighbouring CTAs one step earlier, so the waits rarely stall.
    const int first = (int)blockIdx.x;
    const int stride = (int)gridDim.x;
    const int count = ntiles > first ? (ntiles - first + stride - 1) / stride : 0;

    if (threadIdx.x == 0) {
        for (int k = 0; k < kBStages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kBConsumerWarps);
        }
        for (int w = 0; w < kBConsumerWarps; ++w) warp_done[w] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kBConsumerWarps + 1) {
        // Publisher.
        if (lane != 0) return;
        const long long total = (long long)count * nsteps;
        long long published = 0;
        int i_next = 0;
        unsigned long long start = 0;
        while (published < total) {
            unsigned int m = 0xFFFFFFFFu;
            for (int w = 0; w < kBConsumerWarps; ++w) m = min(m, ld_acquire_cta_shared(&warp_done[w]));
            if ((long long)m > published) {
                asm volatile("fence.proxy.async.global;" ::: "memory");
                asm volatile("fence.acq_rel.gpu;" ::: "memory");
                for (; published < (long long)m; ++published) {
                    atomicAdd(&done[first + i_next * stride], (unsigned int)kBConsumerWarps);
                    if (++i_next == count) i_next = 0;
                }
                start = 0;
                continue;
            }
            const unsigned long long now = global_ns();
            if (start == 0) start = now;
            else if (now - start > kWaitLimitNs) {
                if (err) atomicOr(err, 1u);
                return;
            }
            __nanosleep(64);
        }
        return;
    }

    if (warp == kBConsumerWarps) {
        // Producer.
        DescCache c;
        BatchTile rec{0, 0};
        bool ok = true;
        long long k = 0;
        for (int s = 0; ok && s < nsteps; ++s) {
            const unsigned int target = (unsigned int)kBConsumerWarps * (unsigned int)s;
            for (int i = 0; i < count; ++i) {
                const int st = (int)(k % kBStages);
                if ((i & 31) == 0 && i + lane < count) rec = tiles[first + (i + lane) * stride];
                const int bt_lat = __shfl_sync(0xFFFFFFFFu, rec.lattice, i & 31);
                const int bt_tile = __shfl_sync(0xFFFFFFFFu, rec.tile, i & 31);
                if (bt_lat != c.lat) load_desc(c, lats, bt_lat, lane);
                int good = 1;
                if (lane == 0) {
                    if (k >= kBStages) good = mbar_wait_bounded(&empty[st], (uint32_t)(((k / kBStages) - 1) & 1));
                    if (good && s > 0 && s < c.steps) {
                        // Rows of tiles prev, this and next of step s - 1.
                        const int nt = c.ta.ntiles;
                        const int g = c.tile_base + bt_tile;
                        const int prev = c.tile_base + (bt_tile == 0 ? nt - 1 : bt_tile - 1);
                        const int next = c.tile_base + (bt_tile == nt - 1 ? 0 : bt_tile + 1);
                        good = wait_tiles(done, prev, next, g, true, target);
                        // Written through the generic proxy by other CTAs; read
                        // by the bulk copy through the async proxy.
                        if (good) asm volatile("fence.proxy.async.global;" ::: "memory");
                    }
                }
                if (!__shfl_sync(0xFFFFFFFFu, good, 0)) {
                    ok = false;
                    break;
                }
                __syncwarp();  // order lane 0's acquire of "empty" before the lanes rewrite the header
                StageHeader* h = headers + st;
                write_header(h, c, s, bt_tile, err, lane);
                if (lane == 0) {
                    if (h->active) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue_tile<true>(h->a, h->ta, h->a.src, bt_tile, stages + (size_t)st * stage_words,
                                         &full[st]);
                    } else {
                        mbar_arrive_expect_tx(&full[st], 0u);
                    }
                }
                __syncwarp();
                ++k;
            }
        }
        if (lane == 0) {
            if (!ok && err) atomicOr(err, 1u);
            // Never leave while copies into this CTA's shared memory may be in flight.
            for (long long j = (k > kBStages ? k - kBStages : 0); j < k; ++j)
                (void)mbar_wait_bounded(&full[j % kBStages], (uint32_t)((j / kBStages) & 1));
        }
        return;
    }

    // Consumers.
    long long k = 0;
    unsigned int finished = 0;
    for (int s = 0; s < nsteps; ++s) {
        for (int i = 0; i < count; ++i, ++k) {
            const int st = (int)(k % kBStages);
            if (!mbar_wait_bounded(&full[st], (uint32_t)((k / kBStages) & 1))) {
                if (lane == 0 && err) atomicOr(err, 1u);
                return;
            }
            const StageHeader& h = headers[st];
            if (h.active) {
                if (h.force) batch_compute<true>(h, stages + (size_t)st * stage_words);
                else batch_compute<false>(h, stages + (size_t)st * stage_words);
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[st]);
                st_release_cta_shared(&warp_done[warp], ++finished);
            }
        }
    }
}

__global__ void advance_kernel(int* step_base, int by) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *step_base += by;
}

int batch_blocks_per_sm(int dev, cudaError_t* e) {
    static std::mutex m;
    static int cached[64] = {};
    std::lock_guard<std::mutex> lock(m);
    if (dev < 0 || dev >= 64) {
        *e = cudaErrorInvalidDevice;
        return 0;
    }
    if (!cached[dev]) {
        const int smem = kBPrefixBytes + kBStages * kBStageBudget;
        *e = cudaFuncSetAttribute(fhp_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (*e != cudaSuccess) return 0;
        int n = 0;
        *e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fhp_batch_kernel, kBThreads, smem);
        if (*e != cudaSuccess) return 0;
        cached[dev] = n > 0 ? n : 1;
    }
    *e = cudaSuccess;
    return cached[dev];
}

int batch_run_blocks_per_sm(int dev, cudaError_t* e) {
    static std::mutex m;
    static int cached[64] = {};
    std::lock_guard<std::mutex> lock(m);
    if (dev < 0 || dev >= 64) {
        *e = cudaErrorInvalidDevice;
        return 0;
    }
    if (!cached[dev]) {
        const int smem = kBPrefixBytes + kBStages * kBStageBudget;
        *e = cudaFuncSetAttribute(fhp_batch_run_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (*e != cudaSuccess) return 0;
        int n = 0;
        *e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fhp_batch_run_kernel, kBRunThreads, smem);
        if (*e != cudaSuccess) return 0;
        if (n < 1) {
            *e = cudaErrorInvalidConfiguration;
            return 0;
        }
        cached[dev] = n;
    }
    *e = cudaSuccess;
    return cached[dev];
}

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace fhp

// ---------------------------------------------------------------------------
// Host side: the batch object.
// ---------------------------------------------------------------------------
namespace {

struct Member {
    bool used = false;
    fhp::Geometry g;
    uint64_t seed = 0;
    double p = 0.0;
    fhp::ForcingTable ft{};
    size_t off = 0, bytes = 0;    // arena block
    uint32_t* buf[2] = {nullptr, nullptr};
    uint32_t* solid = nullptr;
    unsigned int* flags = nullptr;
    int cur = 0;
    int64_t t = 0;
    int64_t steps_left = -1;      // -1: no budget
    bool has_solid = false;
    int R = 1;
    int tile_base = 0;            // first entry of the member's tiles in the tile list
};

constexpr int64_t kMaxTime = (int64_t)1 << 48;

// Debug builds follow every member block with a canary of kCanaryBytes
// (filled with kCanaryByte), checked by fhp_batch_debug_canaries.
constexpr size_t kCanaryBytes = fhp::kDebugBuild ? 256 : 0;
constexpr unsigned char kCanaryByte = 0xA5;

size_t member_bytes(const fhp::Geometry& g) {
    return 15 * fhp::round256(g.plane_words * sizeof(uint32_t)) + 256 + kCanaryBytes;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

constexpr int kTuneClasses = 32;
constexpr int kTuneMinSteps = 16;   // a trial runs at least this many steps with each candidate
constexpr int kTuneCands = 6;       // (kernel, tile quads, temporal block) candidates a trial compares
constexpr int kDefaultTileQuads = 256;

struct TuneTrial {
    int cls = -1;                    // class being measured, -1: none in flight
    int ncand = 0;
    int kind[kTuneCands] = {};
    int quads[kTuneCands] = {};
    int block[kTuneCands] = {};      // temporal block k (1: none)
    cudaEvent_t ev[kTuneCands][2] = {};   // [candidate][start, end]
    double updates[kTuneCands] = {};
};

struct fhp_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint8_t* arena_base = nullptr;
    bool owns_arena = false;
    fhp::Arena arena;
    std::vector<Member> members;
    // device tables (allocated from the arena, grown on demand)
    size_t lat_off = SIZE_MAX, lat_cap = 0;     // BatchLattice entries
    size_t tile_off = SIZE_MAX, tile_cap = 0;   // BatchTile entries
    size_t misc_off = SIZE_MAX;                 // step base + error word
    fhp::BatchLattice* d_lats = nullptr;
    fhp::BatchTile* d_tiles = nullptr;
    unsigned int* d_done = nullptr;             // per-tile counters of the multi-step kernel
    int step_kernel = FHP_BATCH_KERNEL_AUTO;
    int tuned[kTuneClasses] = {};               // per tile-count class: kernel measured fastest (0: unknown)
    int tuned_quads[kTuneClasses] = {};         // ... and its tile size (quads per tile)
    int tuned_block[kTuneClasses] = {};         // ... and its temporal block (1: none)
    int tile_quads = 0;                         // quads per tile: 0 automatic (tuned with the kernel)
    int temporal_block = 0;                     // 0 automatic (tuned with the kernel), 1 none, 2 or 4
    // blocked passes: member table and tile list (allocated from the arena)
    size_t bmem_off = SIZE_MAX, bmem_cap = 0;
    size_t btile_off = SIZE_MAX, btile_cap = 0;
    fhp::BlockMember* d_bmem = nullptr;
    fhp::BlockTile* d_btiles = nullptr;
    std::vector<fhp::BlockMember> h_bmem;
    std::vector<fhp::BlockTile> h_btiles;
    int cur_quads = kDefaultTileQuads;          // tile size of the current tile list
    TuneTrial trial;
    int* d_step_base = nullptr;
    unsigned int* d_err = nullptr;
    std::vector<fhp::BatchLattice> h_lats;
    std::vector<fhp::BatchTile> h_tiles;
    bool tiles_dirty = true;
    int ntiles = 0;
    int h_counters[2] = {0, 0};                 // source of the step_base upload
    int graph_steps = 64;
    cudaGraphExec_t graph = nullptr;
    int64_t launches = 0;
    std::string err;
};

namespace {

int bfail(fhp_batch* b, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else fhp::set_thread_error(buf);
    return code;
}

int bcuda(fhp_batch* b, cudaError_t e, const char* what) {
    return bfail(b, FHP_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

Member* member(fhp_batch* b, int32_t slot) {
    if (!b || slot < 0 || slot >= (int32_t)b->members.size() || !b->members[slot].used) return nullptr;
    return &b->members[slot];
}

void drop_graph(fhp_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

size_t tile_table_bytes(size_t cap) {
    return fhp::round256(cap * sizeof(fhp::BatchTile)) + fhp::round256(cap * sizeof(unsigned int));
}

// Make sure the device tables can hold `lats` lattices and `tiles` tiles.
int ensure_tables(fhp_batch* b, size_t lats, size_t tiles) {
    if (lats > b->lat_cap) {
        const size_t cap = std::max<size_t>(lats, 2 * b->lat_cap + 16);
        const size_t off = b->arena.allocate(cap * sizeof(fhp::BatchLattice));
        if (off == SIZE_MAX) return bfail(b, FHP_ENOMEM, "batch arena full (descriptor table)");
        if (b->lat_off != SIZE_MAX) b->arena.release(b->lat_off, b->lat_cap * sizeof(fhp::BatchLattice));
        b->lat_off = off;
        b->lat_cap = cap;
        b->d_lats = (fhp::BatchLattice*)(b->arena_base + off);
        drop_graph(b);
    }
    if (tiles > b->tile_cap) {
        // The tile list followed by one completion counter per tile.
        const size_t cap = std::max<size_t>(tiles, 2 * b->tile_cap + 256);
        const size_t off = b->arena.allocate(tile_table_bytes(cap));
        if (off == SIZE_MAX) return bfail(b, FHP_ENOMEM, "batch arena full (tile table)");
        if (b->tile_off != SIZE_MAX) b->arena.release(b->tile_off, tile_table_bytes(b->tile_cap));
        b->tile_off = off;
        b->tile_cap = cap;
        b->d_tiles = (fhp::BatchTile*)(b->arena_base + off);
        b->d_done = (unsigned int*)(b->arena_base + off + fhp::round256(cap * sizeof(fhp::BatchTile)));
        drop_graph(b);
    }
    return FHP_OK;
}

// Rows per tile: about `quads` quads per tile (256: one per consumer
// thread), and the tile's 8 planes within one stage.
int rows_per_tile(const fhp::Geometry& g, int quads = kDefaultTileQuads) {
    const long long row_bytes = 8LL * g.Pq * 4;
    int R = (quads + g.nq - 1) / g.nq;
    const int fit = (int)(fhp::kBStageBudget / row_bytes);
    R = std::min(R, fit);
    R = std::min(R, g.H);
    return R < 1 ? 1 : R;
}

int scratch_bytes_op(fhp_batch* b, size_t bytes, size_t* off) {
    *off = b->arena.allocate(bytes);
    if (*off == SIZE_MAX) return bfail(b, FHP_ENOMEM, "batch arena full (staging of %zu bytes)", bytes);
    return FHP_OK;
}

}  // namespace

extern "C" {

size_t fhp_batch_lattice_bytes(int32_t width, int32_t height) {
    if (width < 32 || width % 32 || height < 2 || height % 2) return 0;
    const fhp::Geometry g = fhp::make_geometry(width, height);
    if (8LL * g.Pq * 4 > fhp::kBStageBudget) return 0;
    return member_bytes(g);
}

int fhp_batch_create(fhp_batch** out, size_t arena_bytes, void* device_memory, void* stream) {
    if (!out) return bfail(nullptr, FHP_EINVAL, "out is NULL");
    *out = nullptr;
    if (arena_bytes < 65536) return bfail(nullptr, FHP_EINVAL, "arena of %zu bytes is too small", arena_bytes);
    fhp_batch* b = new (std::nothrow) fhp_batch();
    if (!b) return bfail(nullptr, FHP_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) {
        delete b;
        return bfail(nullptr, FHP_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    }
    b->stream = (cudaStream_t)stream;
    if (device_memory) {
        if ((uintptr_t)device_memory & 255u) {
            delete b;
            return bfail(nullptr, FHP_EINVAL, "device_memory must be 256-byte aligned");
        }
        b->arena_base = (uint8_t*)device_memory;
        b->owns_arena = false;
    } else {
        e = cudaMalloc((void**)&b->arena_base, arena_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return bfail(nullptr, FHP_ENOMEM, "cudaMalloc(%zu): %s", arena_bytes, cudaGetErrorString(e));
        }
        b->owns_arena = true;
    }
    b->arena.reset(arena_bytes);
    b->misc_off = b->arena.allocate(256);
    b->d_step_base = (int*)(b->arena_base + b->misc_off);
    b->d_err = (unsigned int*)(b->arena_base + b->misc_off + 64);
    e = cudaMemsetAsync(b->arena_base + b->misc_off, 0, 256, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        if (b->owns_arena) cudaFree(b->arena_base);
        delete b;
        return bfail(nullptr, FHP_ECUDA, "initialising the batch: %s", cudaGetErrorString(e));
    }
    *out = b;
    return FHP_OK;
}

void fhp_batch_destroy(fhp_batch* b) {
    if (!b) return;
    DeviceGuard dg(b->device);
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (auto& pair : b->trial.ev)
        for (auto& ev : pair)
            if (ev) cudaEventDestroy(ev);
    if (b->owns_arena && b->arena_base) cudaFree(b->arena_base);
    delete b;
}

const char* fhp_batch_last_error(const fhp_batch* b) { return b ? b->err.c_str() : ""; }

int fhp_batch_add(fhp_batch* b, int32_t width, int32_t height, uint64_t seed, double forcing_p,
                  int32_t* out_slot) {
    if (!b || !out_slot) return bfail(b, FHP_EINVAL, "NULL argument");
    *out_slot = -1;
    if (width < 32 || width % 32 || height < 2 || height % 2)
        return bfail(b, FHP_EINVAL, "invalid lattice %d x %d", width, height);
    if (!(forcing_p >= 0.0 && forcing_p <= 1.0)) return bfail(b, FHP_EINVAL, "forcing probability outside [0, 1]");
    const fhp::Geometry g = fhp::make_geometry(width, height);
    if (8LL * g.Pq * 4 > fhp::kBStageBudget)
        return bfail(b, FHP_EINVAL, "rows of %d nodes are too wide for a batch member", width);
    DeviceGuard dg(b->device);
    Member m;
    m.used = true;
    m.g = g;
    m.seed = seed;
    m.p = forcing_p;
    m.ft = fhp::forcing_table(forcing_p);
    m.bytes = member_bytes(g);
    m.off = b->arena.allocate(m.bytes);
    if (m.off == SIZE_MAX) return bfail(b, FHP_ENOMEM, "batch arena full: a %d x %d lattice needs %zu bytes", width, height, m.bytes);
    const size_t pb = fhp::round256(g.plane_words * sizeof(uint32_t));
    uint8_t* base = b->arena_base + m.off;
    m.buf[0] = (uint32_t*)base;
    m.buf[1] = (uint32_t*)(base + 7 * pb);
    m.solid = (uint32_t*)(base + 14 * pb);
    m.flags = (unsigned int*)(base + 15 * pb);
    m.R = rows_per_tile(g, b->cur_quads);
    cudaError_t e = cudaMemsetAsync(base, 0, m.bytes - kCanaryBytes, b->stream);
    if (e == cudaSuccess && kCanaryBytes)
        e = cudaMemsetAsync(base + m.bytes - kCanaryBytes, kCanaryByte, kCanaryBytes, b->stream);
    if (e != cudaSuccess) {
        b->arena.release(m.off, m.bytes);
        return bcuda(b, e, "clearing a new member");
    }
    int32_t slot = -1;
    for (size_t i = 0; i < b->members.size(); ++i)
        if (!b->members[i].used) { slot = (int32_t)i; break; }
    if (slot < 0) {
        slot = (int32_t)b->members.size();
        b->members.push_back(m);
    } else {
        b->members[slot] = m;
    }
    b->tiles_dirty = true;
    *out_slot = slot;
    return FHP_OK;
}

int fhp_batch_remove(fhp_batch* b, int32_t slot) {
    Member* m = member(b, slot);
    if (!m) return bfail(b, FHP_EINVAL, "no member in slot %d", slot);
    DeviceGuard dg(b->device);
    cudaError_t e = cudaStreamSynchronize(b->stream);  // nothing may still use its memory
    if (e != cudaSuccess) return bcuda(b, e, "synchronizing");
    b->arena.release(m->off, m->bytes);
    *m = Member();
    b->tiles_dirty = true;
    return FHP_OK;
}

int fhp_batch_remove_async(fhp_batch* b, int32_t slot) {
    Member* m = member(b, slot);
    if (!m) return bfail(b, FHP_EINVAL, "no member in slot %d", slot);
    // No wait: any later use of the block is enqueued on the batch's stream
    // behind the work already there.
    b->arena.release(m->off, m->bytes);
    *m = Member();
    b->tiles_dirty = true;
    return FHP_OK;
}

int fhp_batch_coarse_grain_device(fhp_batch* b, int32_t slot, int32_t block, int32_t* counts, float* rho, float* ux,
                                  float* uy, void* stream) {
    Member* m = member(b, slot);
    if (!m) return bfail(b, FHP_EINVAL, "no member in slot %d", slot);
    if (!counts || !rho || !ux || !uy) return bfail(b, FHP_EINVAL, "NULL output buffer");
    if (block < 32 || block % 32 || m->g.W % block || m->g.H % block)
        return bfail(b, FHP_EINVAL, "coarse-grain block %d must be a multiple of 32 dividing %d and %d", block,
                     m->g.W, m->g.H);
    DeviceGuard dg(b->device);
    cudaError_t e = fhp::launch_coarse_grain(m->g, m->buf[m->cur], m->solid, m->has_solid, block, counts, rho, ux, uy,
                                             (cudaStream_t)stream);
    if (e != cudaSuccess) return bcuda(b, e, "launching the coarse-grain kernel");
    ++b->launches;
    return FHP_OK;
}

int fhp_batch_set_state(fhp_batch* b, int32_t slot, const uint8_t* host_bytes) {
    Member* m = member(b, slot);
    if (!m || !host_bytes) return bfail(b, FHP_EINVAL, "invalid slot %d or NULL bytes", slot);
    DeviceGuard dg(b->device);
    const size_t n = (size_t)m->g.W * m->g.H;
    size_t off;
    int rc = scratch_bytes_op(b, n, &off);
    if (rc != FHP_OK) return rc;
    uint8_t* staging = b->arena_base + off;
    cudaError_t e = cudaMemcpyAsync(staging, host_bytes, n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->flags, 0, sizeof(unsigned int), b->stream);
    if (e == cudaSuccess) e = fhp::launch_pack(m->g, staging, m->buf[m->cur], m->solid, m->flags, b->stream);
    unsigned int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, m->flags, sizeof flag, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    b->arena.release(off, n);
    if (e != cudaSuccess) return bcuda(b, e, "setting a member's state");
    ++b->launches;
    m->has_solid = flag != 0;
    return FHP_OK;
}

int fhp_batch_init_random(fhp_batch* b, int32_t slot, double density) {
    Member* m = member(b, slot);
    if (!m || !(density >= 0.0 && density <= 1.0)) return bfail(b, FHP_EINVAL, "invalid slot %d or density", slot);
    DeviceGuard dg(b->device);
    cudaError_t e = fhp::launch_init_random(m->g, m->buf[m->cur], m->solid, m->has_solid, m->seed, density, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "launching the init kernel");
    ++b->launches;
    return FHP_OK;
}

int fhp_batch_load_obstacles(fhp_batch* b, int32_t slot, const uint8_t* host_mask) {
    Member* m = member(b, slot);
    if (!m || !host_mask) return bfail(b, FHP_EINVAL, "invalid slot %d or NULL mask", slot);
    DeviceGuard dg(b->device);
    const size_t n = (size_t)m->g.W * m->g.H;
    size_t off;
    int rc = scratch_bytes_op(b, n, &off);
    if (rc != FHP_OK) return rc;
    uint8_t* staging = b->arena_base + off;
    // Whether any node is solid is decided on the host, so the call does not
    // wait for the device.  The staging block goes back to the arena at once:
    // everything that could reuse it is ordered after the obstacle kernel on
    // the batch's stream.
    bool any = false;
    for (size_t i = 0; i < n && !any; ++i) any = host_mask[i] != 0;
    cudaError_t e = cudaMemcpyAsync(staging, host_mask, n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = fhp::launch_load_obstacles(m->g, staging, m->buf[m->cur], m->solid, m->flags, b->stream);
    b->arena.release(off, n);
    if (e != cudaSuccess) return bcuda(b, e, "loading a member's obstacles");
    ++b->launches;
    m->has_solid = any;
    return FHP_OK;
}

int fhp_batch_load_obstacle_shapes(fhp_batch* b, int32_t slot, const fhp_shape* shapes, int32_t count) {
    Member* m = member(b, slot);
    if (!m) return bfail(b, FHP_EINVAL, "no member in slot %d", slot);
    if (count < 0 || count > FHP_MAX_SHAPES || (count > 0 && !shapes))
        return bfail(b, FHP_EINVAL, "invalid shape list (count %d)", count);
    fhp::ShapeList list{};
    list.n = count;
    for (int i = 0; i < count; ++i) {
        const fhp_shape& sh = shapes[i];
        if ((sh.kind != FHP_SHAPE_DISC && sh.kind != FHP_SHAPE_ROWS) || (sh.kind == FHP_SHAPE_DISC && sh.c < 0))
            return bfail(b, FHP_EINVAL, "invalid shape %d", i);
        list.s[i] = fhp::Shape{sh.kind, sh.a, sh.b, sh.c};
    }
    // Whether any node is solid, decided on the host from the shapes.
    bool any = false;
    for (int i = 0; i < count; ++i) {
        const fhp_shape& sh = shapes[i];
        if (sh.kind == FHP_SHAPE_ROWS) any = any || (std::max(sh.a, 0) < std::min(sh.b, m->g.H));
        else {
            const long long x0 = std::max<long long>((long long)sh.a - sh.c, 0);
            const long long x1 = std::min<long long>((long long)sh.a + sh.c, m->g.W - 1);
            const long long y0 = std::max<long long>((long long)sh.b - sh.c, 0);
            const long long y1 = std::min<long long>((long long)sh.b + sh.c, m->g.H - 1);
            for (long long y = y0; y <= y1 && !any; ++y) {
                const long long dy = y - sh.b, r2 = (long long)sh.c * sh.c - dy * dy;
                const long long dx = sh.a < x0 ? x0 - sh.a : (sh.a > x1 ? sh.a - x1 : 0);
                if (x0 <= x1 && dx * dx <= r2) any = true;
            }
        }
    }
    DeviceGuard dg(b->device);
    cudaError_t e = fhp::launch_obstacle_shapes(m->g, list, m->buf[m->cur], m->solid, nullptr, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "generating a member's obstacles");
    ++b->launches;
    m->has_solid = any;
    return FHP_OK;
}

int fhp_batch_set_rules(fhp_batch* b, int32_t slot, int32_t rules) {
    Member* m = member(b, slot);
    if (!m || (rules != FHP_RULES_FHP_I && rules != FHP_RULES_FHP_II))
        return bfail(b, FHP_EINVAL, "invalid slot %d or rule set %d (members: FHP-I or FHP-II)", slot, rules);
    m->g.rules = rules;
    return FHP_OK;
}

int fhp_batch_get_state(fhp_batch* b, int32_t slot, uint8_t* host_bytes) {
    Member* m = member(b, slot);
    if (!m || !host_bytes) return bfail(b, FHP_EINVAL, "invalid slot %d or NULL bytes", slot);
    DeviceGuard dg(b->device);
    const size_t n = (size_t)m->g.W * m->g.H;
    size_t off;
    int rc = scratch_bytes_op(b, n, &off);
    if (rc != FHP_OK) return rc;
    uint8_t* staging = b->arena_base + off;
    cudaError_t e = fhp::launch_unpack(m->g, m->buf[m->cur], m->solid, staging, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_bytes, staging, n, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    b->arena.release(off, n);
    if (e != cudaSuccess) return bcuda(b, e, "reading a member's state");
    ++b->launches;
    return FHP_OK;
}

int fhp_batch_coarse_grain(fhp_batch* b, int32_t slot, int32_t block, int32_t* counts, float* rho, float* ux,
                           float* uy) {
    Member* m = member(b, slot);
    if (!m) return bfail(b, FHP_EINVAL, "no member in slot %d", slot);
    if (block < 32 || block % 32 || m->g.W % block || m->g.H % block)
        return bfail(b, FHP_EINVAL, "coarse-grain block %d must be a multiple of 32 dividing %d and %d", block,
                     m->g.W, m->g.H);
    DeviceGuard dg(b->device);
    const size_t cells = (size_t)(m->g.W / block) * (m->g.H / block);
    const size_t bc = fhp::round256(cells * 9 * sizeof(int32_t)), bf = fhp::round256(cells * sizeof(float));
    size_t off;
    int rc = scratch_bytes_op(b, bc + 3 * bf, &off);
    if (rc != FHP_OK) return rc;
    uint8_t* s = b->arena_base + off;
    int32_t* dc = (int32_t*)s;
    float* dr = (float*)(s + bc);
    float* dx = (float*)(s + bc + bf);
    float* dy = (float*)(s + bc + 2 * bf);
    cudaError_t e = fhp::launch_coarse_grain(m->g, m->buf[m->cur], m->solid, m->has_solid, block, dc, dr, dx, dy,
                                             b->stream);
    if (e == cudaSuccess && counts) e = cudaMemcpyAsync(counts, dc, cells * 9 * 4, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, dr, cells * 4, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && ux) e = cudaMemcpyAsync(ux, dx, cells * 4, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && uy) e = cudaMemcpyAsync(uy, dy, cells * 4, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    b->arena.release(off, bc + 3 * bf);
    if (e != cudaSuccess) return bcuda(b, e, "coarse-graining a member");
    ++b->launches;
    return FHP_OK;
}

int fhp_batch_set_time(fhp_batch* b, int32_t slot, int64_t t) {
    Member* m = member(b, slot);
    if (!m || t < 0 || t >= kMaxTime) return bfail(b, FHP_EINVAL, "invalid slot or time");
    m->t = t;
    return FHP_OK;
}

int64_t fhp_batch_get_time(const fhp_batch* b, int32_t slot) {
    Member* m = member(const_cast<fhp_batch*>(b), slot);
    return m ? m->t : -1;
}

int fhp_batch_set_steps_left(fhp_batch* b, int32_t slot, int64_t n) {
    Member* m = member(b, slot);
    if (!m || n < -1) return bfail(b, FHP_EINVAL, "invalid slot or step budget");
    m->steps_left = n;
    return FHP_OK;
}

int64_t fhp_batch_get_steps_left(const fhp_batch* b, int32_t slot) {
    Member* m = member(const_cast<fhp_batch*>(b), slot);
    return m ? m->steps_left : -2;
}

int fhp_batch_set_graph_steps(fhp_batch* b, int32_t steps) {
    if (!b || steps < 0) return bfail(b, FHP_EINVAL, "invalid graph step count");
    b->graph_steps = steps;
    drop_graph(b);
    return FHP_OK;
}

namespace {

// Rebuilds the tile list after membership changes (each member's tiles in
// order, starting at its tile_base) and makes sure the device tables fit.
int prepare_tiles(fhp_batch* b) {
    const size_t nm = b->members.size();
    if (b->tiles_dirty) {
        b->h_tiles.clear();
        for (size_t i = 0; i < nm; ++i) {
            Member& m = b->members[i];
            if (!m.used) continue;
            m.tile_base = (int)b->h_tiles.size();
            const int nt = (m.g.H + m.R - 1) / m.R;
            for (int j = 0; j < nt; ++j) b->h_tiles.push_back(fhp::BatchTile{(int)i, j});
        }
        int rc = ensure_tables(b, std::max<size_t>(nm, 1), std::max<size_t>(b->h_tiles.size(), 1));
        if (rc != FHP_OK) return rc;
        cudaError_t e = cudaMemcpyAsync(b->d_tiles, b->h_tiles.data(), b->h_tiles.size() * sizeof(fhp::BatchTile),
                                        cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "uploading the tile list");
        b->ntiles = (int)b->h_tiles.size();
        b->tiles_dirty = false;
    }
    return ensure_tables(b, std::max<size_t>(nm, 1), std::max<size_t>(b->h_tiles.size(), 1));
}

// Tiles of the members at a tile size of `quads` (the tuning classes are
// keyed by the count at the default size, so that a class does not change
// with the size tried).
int tiles_at(const fhp_batch* b, int quads) {
    long long n = 0;
    for (const Member& m : b->members)
        if (m.used) {
            const int R = rows_per_tile(m.g, quads);
            n += (m.g.H + R - 1) / R;
        }
    return (int)std::min<long long>(n, 1 << 30);
}

// Re-tile every member at `quads` quads per tile (results do not depend on
// the tiling).
void apply_tile_quads(fhp_batch* b, int quads) {
    if (quads == b->cur_quads) return;
    b->cur_quads = quads;
    for (Member& m : b->members)
        if (m.used) m.R = rows_per_tile(m.g, quads);
    b->tiles_dirty = true;
}

// Uploads the descriptors of a call of `chunk` steps (each member advances
// min(chunk, its budget) steps); returns the largest count in *max_steps.
// A member's step arguments at its current step (src: the buffer holding it).
void fill_step_args(const fhp_batch* b, const Member& m, fhp::StepArgs& a) {
    a.src = m.buf[m.cur];
    a.dst = m.buf[m.cur ^ 1];
    a.solid = m.solid;
    a.plane_words = m.g.plane_words;
    a.H = m.g.H;
    a.Wq = m.g.Wq;
    a.nq = m.g.nq;
    a.Pq = m.g.Pq;
    a.rows_per_warp = a.groups_per_parity = a.warps_per_row = 1;
    a.key = fhp::Key2{(uint32_t)m.seed, (uint32_t)(m.seed >> 32)};
    a.rest_rules = fhp::rest_rules_mask(m.g);
    a.t_lo = (uint32_t)m.t;
    a.t_hi = (uint32_t)(m.t >> 32);
    a.err = b->d_err;
    a.ft = m.ft;
}

// Descriptors of a call of `chunk` steps: member i advances by
// min(chunk, its budget, caps[i] if caps is given) steps (steps_of[i]).
int upload_descriptors(fhp_batch* b, int chunk, std::vector<int>& steps_of, int* max_steps,
                       const std::vector<int>* caps = nullptr) {
    const size_t nm = b->members.size();
    b->h_lats.assign(nm, fhp::BatchLattice{});
    steps_of.assign(nm, 0);
    *max_steps = 0;
    for (size_t i = 0; i < nm; ++i) {
        const Member& m = b->members[i];
        fhp::BatchLattice& L = b->h_lats[i];
        if (!m.used) continue;
        int64_t k = chunk;
        if (m.steps_left >= 0 && m.steps_left < k) k = m.steps_left;
        if (caps && (*caps)[i] < k) k = (*caps)[i];
        steps_of[i] = (int)k;
        *max_steps = std::max(*max_steps, (int)k);
        fill_step_args(b, m, L.a);
        L.ta.R = m.R;
        L.ta.ntiles = (m.g.H + m.R - 1) / m.R;
        L.ta.nq_magic = ((1ull << 32) + m.g.nq - 1) / m.g.nq;
        L.buf[0] = m.buf[0];
        L.buf[1] = m.buf[1];
        L.t0 = (unsigned long long)m.t;
        L.cur = m.cur;
        L.steps = (int)k;
        L.force = m.ft.q[32] != 0;
        L.tile_base = m.tile_base;
    }
    if (*max_steps == 0) return FHP_OK;
    cudaError_t e = cudaMemcpyAsync(b->d_lats, b->h_lats.data(), nm * sizeof(fhp::BatchLattice),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "uploading the descriptors");
    return FHP_OK;
}

void finish_call(fhp_batch* b, const std::vector<int>& steps_of) {
    for (size_t i = 0; i < b->members.size(); ++i) {
        Member& m = b->members[i];
        if (!m.used) continue;
        const int k = steps_of[i];
        m.t += k;
        m.cur ^= (k & 1);
        if (m.steps_left >= 0) m.steps_left -= k;
    }
}

// One cooperative launch of the multi-step kernel for `max_steps` steps.
int launch_run_call(fhp_batch* b, int max_steps) {
    cudaError_t e;
    const int bps = fhp::batch_run_blocks_per_sm(b->device, &e);
    if (e != cudaSuccess) return bcuda(b, e, "configuring the multi-step batch kernel");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return bcuda(b, e, "querying the SM count");
    const int grid = std::min(b->ntiles, bps * sms);
    e = cudaMemsetAsync(b->d_done, 0, (size_t)b->ntiles * sizeof(unsigned int), b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "clearing the tile counters");
    const fhp::BatchLattice* lats = b->d_lats;
    const fhp::BatchTile* tiles = b->d_tiles;
    int ntiles = b->ntiles;
    int nsteps = max_steps;
    unsigned int* done = b->d_done;
    unsigned int* err = b->d_err;
    void* args[] = {(void*)&lats, (void*)&tiles, (void*)&ntiles, (void*)&nsteps, (void*)&done, (void*)&err};
    const size_t smem = fhp::kBPrefixBytes + fhp::kBStages * fhp::kBStageBudget;
    e = cudaLaunchCooperativeKernel((const void*)fhp::fhp_batch_run_kernel, dim3(grid), dim3(fhp::kBRunThreads), args,
                                    smem, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "launching the multi-step batch kernel");
    ++b->launches;
    return FHP_OK;
}

// The graph of graph_steps launches of the single-step kernel is captured once (with one resident wave
// of CTAs; those without a tile exit at once) and stays valid while the
// membership changes: it reads the tile list and its length from device
// memory.  It is dropped only when the device tables move.
int ensure_graph(fhp_batch* b) {
    if (b->graph || b->graph_steps <= 0) return FHP_OK;
    cudaError_t e = cudaSuccess;
    const int bps = fhp::batch_blocks_per_sm(b->device, &e);
    if (e != cudaSuccess) return bcuda(b, e, "configuring the batch kernel");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return bcuda(b, e, "querying the SM count");
    const int full_grid = bps * sms;
    const size_t smem = fhp::kBPrefixBytes + fhp::kBStages * fhp::kBStageBudget;
    const int G = b->graph_steps;
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bcuda(b, e, "creating the capture stream");
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int o = 0; o < G; ++o)
            fhp::fhp_batch_kernel<<<full_grid, fhp::kBThreads, smem, cs>>>(b->d_lats, b->d_tiles, b->d_step_base, o,
                                                                            b->d_err);
        fhp::advance_kernel<<<1, 32, 0, cs>>>(b->d_step_base, G);
        e = cudaStreamEndCapture(cs, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e == cudaSuccess) e = cudaGraphUpload(b->graph, b->stream);  // not on the first replay's critical path
    if (e != cudaSuccess) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        return bcuda(b, e, "capturing the batch step graph");
    }
    return FHP_OK;
}

// max_steps launches of the single-step kernel, replayed from the captured
// graph in groups of graph_steps.
int launch_step_call(fhp_batch* b, int max_steps) {
    cudaError_t e = cudaSuccess;
    b->h_counters[0] = 0;
    b->h_counters[1] = b->ntiles;
    e = cudaMemcpyAsync(b->d_step_base, b->h_counters, sizeof b->h_counters, cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "uploading the step counters");
    int bps = fhp::batch_blocks_per_sm(b->device, &e);
    if (e != cudaSuccess) return bcuda(b, e, "configuring the batch kernel");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return bcuda(b, e, "querying the SM count");
    // Direct launches size the grid to the tile count; the graph is captured
    // once with one resident wave of CTAs (those without a tile exit at once)
    // and stays valid while the membership changes.
    const int full_grid = bps * sms;
    const int grid = std::min(b->ntiles, full_grid);
    const size_t smem = fhp::kBPrefixBytes + fhp::kBStages * fhp::kBStageBudget;
    int done = 0;
    const int G = b->graph_steps;
    if (G > 0 && max_steps >= G) {
        const int rc = ensure_graph(b);
        if (rc != FHP_OK) return rc;
        while (max_steps - done >= G) {
            e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "launching the batch step graph");
            b->launches += G;
            done += G;
        }
    }
    for (int o = 0; o < max_steps - done; ++o) {
        fhp::fhp_batch_kernel<<<grid, fhp::kBThreads, smem, b->stream>>>(b->d_lats, b->d_tiles, b->d_step_base, o,
                                                                          b->d_err);
        e = cudaGetLastError();
        if (e != cudaSuccess) return bcuda(b, e, "launching the batch kernel");
        ++b->launches;
    }
    return FHP_OK;
}

}  // namespace

namespace {

// Node updates one call issues (members advance steps_of[i] steps).
double issued_updates(const fhp_batch* b, const std::vector<int>& steps_of) {
    double u = 0.0;
    for (size_t i = 0; i < b->members.size(); ++i)
        if (b->members[i].used) u += (double)b->members[i].g.W * b->members[i].g.H * steps_of[i];
    return u;
}

// Online autotuning of the automatic batch kernel choice.  Batches are
// classed by the binary order of magnitude of their tile count; the first
// long enough call in a class runs half its steps with each kernel, timed by
// events on the batch's stream, and a later call reads the events (without
// waiting) and records the kernel with more node updates per millisecond.
int tile_class(int ntiles) {
    int c = 0;
    while (ntiles > 1 && c < kTuneClasses - 1) {
        ntiles >>= 1;
        ++c;
    }
    return c;
}

void collect_trial(fhp_batch* b) {
    TuneTrial& tr = b->trial;
    if (tr.cls < 0) return;
    for (int k = 0; k < tr.ncand; ++k)
        if (cudaEventQuery(tr.ev[k][1]) != cudaSuccess) return;  // not finished yet: look again next call
    int best = -1;
    double best_rate = 0.0;
    for (int k = 0; k < tr.ncand; ++k) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, tr.ev[k][0], tr.ev[k][1]) != cudaSuccess || !(ms > 0.0f)) continue;
        const double rate = tr.updates[k] / ms;
        if (best < 0 || rate > best_rate) {
            best = k;
            best_rate = rate;
        }
    }
    b->tuned[tr.cls] = best >= 0 ? tr.kind[best] : FHP_BATCH_KERNEL_SINGLE_STEP;
    b->tuned_quads[tr.cls] = best >= 0 ? tr.quads[best] : kDefaultTileQuads;
    b->tuned_block[tr.cls] = best >= 0 ? tr.block[best] : 1;
    tr.cls = -1;
}

int ensure_trial_events(fhp_batch* b) {
    for (auto& pair : b->trial.ev)
        for (auto& ev : pair)
            if (!ev) {
                cudaError_t e = cudaEventCreate(&ev);
                if (e != cudaSuccess) return bcuda(b, e, "creating the tuning events");
            }
    return FHP_OK;
}

// One chunk of steps with the given kernel (member i at most caps[i] steps
// if caps is given).
int run_chunk(fhp_batch* b, int chunk, int kind, std::vector<int>& steps_of, double* updates,
              const std::vector<int>* caps = nullptr) {
    int max_steps = 0;
    int rc = upload_descriptors(b, chunk, steps_of, &max_steps, caps);
    if (rc != FHP_OK || max_steps == 0) return rc;
    rc = kind == FHP_BATCH_KERNEL_MULTI_STEP && max_steps >= 2 ? launch_run_call(b, max_steps)
                                                               : launch_step_call(b, max_steps);
    if (rc != FHP_OK) return rc;
    if (updates) *updates = issued_updates(b, steps_of);
    finish_call(b, steps_of);
    return FHP_OK;
}

// Device tables of the blocked passes (member descriptors, tile list), grown
// on demand from the arena; only work on the batch's stream uses them.
int ensure_block_tables(fhp_batch* b, size_t nm, size_t ntiles) {
    if (nm > b->bmem_cap) {
        const size_t cap = std::max<size_t>(nm, 2 * b->bmem_cap + 16);
        const size_t off = b->arena.allocate(cap * sizeof(fhp::BlockMember));
        if (off == SIZE_MAX) return bfail(b, FHP_ENOMEM, "batch arena full (blocked-pass descriptors)");
        if (b->bmem_off != SIZE_MAX) b->arena.release(b->bmem_off, b->bmem_cap * sizeof(fhp::BlockMember));
        b->bmem_off = off;
        b->bmem_cap = cap;
        b->d_bmem = (fhp::BlockMember*)(b->arena_base + off);
    }
    if (ntiles > b->btile_cap) {
        const size_t cap = std::max<size_t>(ntiles, 2 * b->btile_cap + 256);
        const size_t off = b->arena.allocate(cap * sizeof(fhp::BlockTile));
        if (off == SIZE_MAX) return bfail(b, FHP_ENOMEM, "batch arena full (blocked-pass tile list)");
        if (b->btile_off != SIZE_MAX) b->arena.release(b->btile_off, b->btile_cap * sizeof(fhp::BlockTile));
        b->btile_off = off;
        b->btile_cap = cap;
        b->d_btiles = (fhp::BlockTile*)(b->arena_base + off);
    }
    return FHP_OK;
}

// Make room for the blocked passes' tables of the current members (k = 4
// has the most tiles).  Returns false, leaving the batch's error message as
// it was, if the arena cannot hold them: the automatic choice then tunes
// without blocked candidates instead of failing the call.
bool reserve_block_tables(fhp_batch* b) {
    size_t tiles = 0;
    for (const Member& m : b->members) {
        if (!m.used) continue;
        const int R = fhp::batch_block_rows(m.g, 4);
        if (R > 0) tiles += (size_t)((m.g.H + R - 1) / R);
    }
    if (tiles == 0) return false;
    const std::string saved = b->err;
    if (ensure_block_tables(b, b->members.size(), tiles) != FHP_OK) {
        b->err = saved;
        return false;
    }
    return true;
}

// One chunk with temporal blocking k (2 or 4): every member whose rows fit a
// blocked tile (fhp::batch_block_rows) advances by floor(s / k) passes of k
// steps, s = min(chunk, its budget), one launch of the blocked kernel per
// pass over the tiles of all such members; then the remaining steps of every
// member (s mod k, or all s for members that take no pass) run on the batch
// step kernel `kind`.  The result equals s single steps for every member.
int run_blocked_chunk(fhp_batch* b, int chunk, int k, int kind, std::vector<int>& steps_of, double* updates) {
    const size_t nm = b->members.size();
    std::vector<int> passes(nm, 0), caps(nm, 0);
    b->h_bmem.assign(nm, fhp::BlockMember{});
    b->h_btiles.clear();
    int max_passes = 0;
    double upd = 0.0;
    for (size_t i = 0; i < nm; ++i) {
        const Member& m = b->members[i];
        if (!m.used) continue;
        int64_t s = chunk;
        if (m.steps_left >= 0 && m.steps_left < s) s = m.steps_left;
        upd += (double)m.g.W * m.g.H * (double)s;
        const int R = fhp::batch_block_rows(m.g, k);
        const int p = R > 0 ? (int)(s / k) : 0;
        passes[i] = p;
        caps[i] = (int)(s - (int64_t)p * k);
        if (p == 0) continue;
        max_passes = std::max(max_passes, p);
        fhp::BlockMember& M = b->h_bmem[i];
        fill_step_args(b, m, M.a);
        M.buf[0] = m.buf[0];
        M.buf[1] = m.buf[1];
        M.t0 = (unsigned long long)m.t;
        M.cur = m.cur;
        M.passes = p;
        M.R_out = R;
        M.force = m.ft.q[32] != 0;
        const int nt = (m.g.H + R - 1) / R;
        for (int j = 0; j < nt; ++j) b->h_btiles.push_back(fhp::BlockTile{(int)i, j});
    }
    if (max_passes > 0) {
        // CTA c takes tiles c, c + grid, ...: with the list ordered by
        // decreasing work (quads of a pass), every CTA's share comes out about
        // even and the last tiles of a pass are the small ones.
        auto work = [&](const fhp::BlockTile& t) {
            const fhp::BlockMember& M = b->h_bmem[t.lattice];
            const int rows_out = std::min(M.R_out, M.a.H - t.tile * M.R_out);
            return (long long)(rows_out + k) * M.a.nq;
        };
        std::stable_sort(b->h_btiles.begin(), b->h_btiles.end(),
                         [&](const fhp::BlockTile& x, const fhp::BlockTile& y) { return work(x) > work(y); });
        int rc = ensure_block_tables(b, nm, b->h_btiles.size());
        if (rc != FHP_OK) return rc;
        cudaError_t e = cudaMemcpyAsync(b->d_bmem, b->h_bmem.data(), nm * sizeof(fhp::BlockMember),
                                        cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_btiles, b->h_btiles.data(), b->h_btiles.size() * sizeof(fhp::BlockTile),
                                cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "uploading the blocked-pass tables");
        for (int p = 0; p < max_passes; ++p) {
            e = fhp::launch_batch_block(b->d_bmem, b->d_btiles, (int)b->h_btiles.size(), p, k, b->d_err, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "launching the blocked batch kernel");
            ++b->launches;
        }
        for (size_t i = 0; i < nm; ++i) {
            Member& m = b->members[i];
            if (!m.used || passes[i] == 0) continue;
            const int64_t adv = (int64_t)passes[i] * k;
            m.t += adv;
            m.cur ^= passes[i] & 1;   // one write per pass
            if (m.steps_left >= 0) m.steps_left -= adv;
        }
    }
    std::vector<int> rest_of;
    int rc = run_chunk(b, chunk, kind, rest_of, nullptr, &caps);
    if (rc != FHP_OK) return rc;
    steps_of.assign(nm, 0);
    for (size_t i = 0; i < nm; ++i) steps_of[i] = passes[i] * k + (i < rest_of.size() ? rest_of[i] : 0);
    if (updates) *updates = upd;
    return FHP_OK;
}

}  // namespace

namespace {
int batch_step(fhp_batch* b, int64_t n);
}  // namespace

int fhp_batch_step(fhp_batch* b, int64_t n) {
    nvtxRangePushA("fhp_batch_step");
    const int rc = batch_step(b, n);
    nvtxRangePop();
    return rc;
}

namespace {
int batch_step(fhp_batch* b, int64_t n) {
    if (!b || n < 0) return bfail(b, FHP_EINVAL, "invalid arguments");
    DeviceGuard dg(b->device);
    for (auto& m : b->members) {
        if (!m.used) continue;
        int64_t k = n;
        if (m.steps_left >= 0 && m.steps_left < k) k = m.steps_left;
        if (k >= kMaxTime - m.t) return bfail(b, FHP_EINVAL, "a member's step counter would pass 2^48");
    }
    int rc = prepare_tiles(b);
    if (rc != FHP_OK) return rc;
    std::vector<int> steps_of;
    int64_t left = n;
    const int cls = tile_class(tiles_at(b, kDefaultTileQuads));
    if (b->step_kernel == FHP_BATCH_KERNEL_AUTO && b->ntiles > 0) {
        collect_trial(b);
        // Candidates: both kernels, and with an automatic tile size two
        // sizes (256 and 128 quads per tile); with an automatic temporal
        // block also blocked passes of k = 2 and k = 4 steps (remainders on
        // the single-step kernel).  A trial needs parts long enough for the
        // single-step kernel to run as it normally does (from the captured
        // graph).
        TuneTrial& tr = b->trial;
        int nc = 0;
        const int sizes[2] = {kDefaultTileQuads, kDefaultTileQuads / 2};
        for (int si = 0; si < (b->tile_quads ? 1 : 2); ++si)
            for (int kind : {FHP_BATCH_KERNEL_SINGLE_STEP, FHP_BATCH_KERNEL_MULTI_STEP}) {
                tr.kind[nc] = kind;
                tr.quads[nc] = b->tile_quads ? b->tile_quads : sizes[si];
                tr.block[nc] = b->temporal_block > 1 ? b->temporal_block : 1;
                ++nc;
            }
        const int64_t min_part = std::max<int64_t>(kTuneMinSteps, b->graph_steps);
        bool trial = false;
        if (b->tuned[cls] == FHP_BATCH_KERNEL_AUTO && tr.cls < 0) {
            if (b->temporal_block == 0) {
                // A call long enough for all candidates; the blocked ones need
                // their tables in the arena, and without room for them the
                // trial goes on with the others.
                if (n >= (nc + 2) * min_part) {
                    trial = true;
                    if (reserve_block_tables(b))
                        for (int k : {2, 4}) {
                            tr.kind[nc] = FHP_BATCH_KERNEL_SINGLE_STEP;
                            tr.quads[nc] = b->tile_quads ? b->tile_quads : kDefaultTileQuads;
                            tr.block[nc] = k;
                            ++nc;
                        }
                }
            } else {
                trial = n >= nc * min_part;
            }
        }
        if (trial) {
            // A trial: an equal part of the call with each candidate.
            rc = ensure_trial_events(b);
            if (rc != FHP_OK) return rc;
            // One-time host work stays out of the timed parts: the device
            // tables are grown to the largest candidate tiling first (growing
            // them drops the graph), then the graph is captured and both
            // kernels are configured.  Capturing inside a part once made the
            // single-step kernel look slower than it is (64 lattices: 2356
            // GSUPS for the multi-step kernel was chosen over 2756).
            for (int k = 0; k < nc; ++k) {
                apply_tile_quads(b, tr.quads[k]);
                rc = prepare_tiles(b);
                if (rc != FHP_OK) return rc;
            }
            rc = ensure_graph(b);
            if (rc != FHP_OK) return rc;
            {
                cudaError_t e = cudaSuccess;
                (void)fhp::batch_run_blocks_per_sm(b->device, &e);
                if (e == cudaSuccess) e = fhp::configure_batch_block();
                if (e != cudaSuccess) return bcuda(b, e, "configuring the batch kernels");
            }
            // Parts of a multiple of 4 steps: blocked candidates then run no
            // remainder steps.
            const int part = (int)(std::min<int64_t>(n / nc, (int64_t)1 << 20) & ~(int64_t)3);
            tr.ncand = nc;
            for (int k = 0; k < nc; ++k) {
                apply_tile_quads(b, tr.quads[k]);
                rc = prepare_tiles(b);
                if (rc != FHP_OK) return rc;
                cudaEventRecord(tr.ev[k][0], b->stream);
                tr.updates[k] = 0.0;
                rc = tr.block[k] > 1 ? run_blocked_chunk(b, part, tr.block[k], tr.kind[k], steps_of, &tr.updates[k])
                                     : run_chunk(b, part, tr.kind[k], steps_of, &tr.updates[k]);
                if (rc != FHP_OK) return rc;
                cudaError_t e = cudaEventRecord(tr.ev[k][1], b->stream);
                if (e != cudaSuccess) return bcuda(b, e, "recording the tuning events");
            }
            tr.cls = cls;
            left -= (int64_t)nc * part;
        }
    }
    // The tile size for the rest of the call: the caller's, else the one
    // recorded for the class, else the default.
    int quads = b->tile_quads;
    if (!quads) quads = (b->step_kernel == FHP_BATCH_KERNEL_AUTO && b->tuned_quads[cls]) ? b->tuned_quads[cls]
                                                                                             : kDefaultTileQuads;
    apply_tile_quads(b, quads);
    rc = prepare_tiles(b);
    if (rc != FHP_OK) return rc;
    while (left > 0) {
        // Calls are split into chunks of at most 2^24 steps: the multi-step
        // kernel's counters grow by kBConsumerWarps per tile and step.
        static_assert((unsigned long long)fhp::kBConsumerWarps << 24 <= 0xFFFFFFFFull,
                      "tile counters of a 2^24-step chunk must fit in 32 bits");
        const int chunk = (int)std::min<int64_t>(left, (int64_t)1 << 24);
        int kind = b->step_kernel;
        if (kind == FHP_BATCH_KERNEL_AUTO) {
            const int t = b->tuned[cls];
            kind = t == FHP_BATCH_KERNEL_AUTO ? FHP_BATCH_KERNEL_SINGLE_STEP : t;
        }
        // Temporal block: the caller's, else (with the automatic kernel) the
        // one recorded for the class, else none.
        int k = b->temporal_block;
        if (k == 0) k = (b->step_kernel == FHP_BATCH_KERNEL_AUTO && b->tuned_block[cls]) ? b->tuned_block[cls] : 1;
        rc = k > 1 ? run_blocked_chunk(b, chunk, k, kind, steps_of, nullptr) : run_chunk(b, chunk, kind, steps_of, nullptr);
        if (rc != FHP_OK) return rc;
        left -= chunk;
    }
    return FHP_OK;
}

}  // namespace

int fhp_batch_get_tuned_kernel(const fhp_batch* b, int32_t ntiles) {
    if (!b || ntiles < 0) return -1;
    return b->tuned[tile_class(ntiles ? ntiles : tiles_at(b, kDefaultTileQuads))];
}

int fhp_batch_get_tuned_tile_quads(const fhp_batch* b, int32_t ntiles) {
    if (!b || ntiles < 0) return -1;
    return b->tuned_quads[tile_class(ntiles ? ntiles : tiles_at(b, kDefaultTileQuads))];
}

int fhp_batch_set_tile_quads(fhp_batch* b, int32_t quads) {
    if (!b || (quads != 0 && quads != 64 && quads != 128 && quads != 256))
        return bfail(b, FHP_EINVAL, "tile size %d not in {0, 64, 128, 256}", quads);
    b->tile_quads = quads;
    return FHP_OK;
}

int fhp_batch_get_tile_quads(const fhp_batch* b) { return b ? b->cur_quads : -1; }

int fhp_batch_set_temporal_block(fhp_batch* b, int32_t k) {
    if (!b || (k != 0 && k != 1 && k != 2 && k != 4))
        return bfail(b, FHP_EINVAL, "batch temporal block %d not in {0, 1, 2, 4}", k);
    b->temporal_block = k;
    return FHP_OK;
}

int fhp_batch_get_temporal_block(const fhp_batch* b) { return b ? b->temporal_block : -1; }

int fhp_batch_get_tuned_temporal_block(const fhp_batch* b, int32_t ntiles) {
    if (!b || ntiles < 0) return -1;
    return b->tuned_block[tile_class(ntiles ? ntiles : tiles_at(b, kDefaultTileQuads))];
}

int fhp_batch_block_rows(int32_t width, int32_t height, int32_t k) {
    if (width < 32 || width % 32 || height < 2 || height % 2) return 0;
    return fhp::batch_block_rows(fhp::make_geometry(width, height), k);
}

int32_t fhp_batch_tile_count(fhp_batch* b) {
    if (!b) return -1;
    if (prepare_tiles(b) != FHP_OK) return -1;
    return b->ntiles;
}

int fhp_batch_debug_canaries(fhp_batch* b, int32_t* checked, int32_t* corrupted) {
    if (!b || !checked || !corrupted) return bfail(b, FHP_EINVAL, "NULL argument");
    *checked = 0;
    *corrupted = 0;
    if (!kCanaryBytes) return FHP_OK;
    DeviceGuard dg(b->device);
    std::vector<unsigned char> buf(kCanaryBytes);
    for (const Member& m : b->members) {
        if (!m.used) continue;
        cudaError_t e = cudaMemcpyAsync(buf.data(), b->arena_base + m.off + m.bytes - kCanaryBytes, kCanaryBytes,
                                        cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "reading a canary");
        ++*checked;
        for (unsigned char c : buf)
            if (c != kCanaryByte) {
                ++*corrupted;
                break;
            }
    }
    return FHP_OK;
}

int fhp_batch_set_step_kernel(fhp_batch* b, int32_t kind) {
    if (!b || kind < FHP_BATCH_KERNEL_AUTO || kind > FHP_BATCH_KERNEL_MULTI_STEP)
        return bfail(b, FHP_EINVAL, "batch step kernel %d not in {0, 1, 2}", kind);
    b->step_kernel = kind;
    return FHP_OK;
}

int fhp_batch_get_step_kernel(const fhp_batch* b) { return b ? b->step_kernel : -1; }

int fhp_batch_synchronize(fhp_batch* b) {
    if (!b) return bfail(nullptr, FHP_EINVAL, "batch is NULL");
    DeviceGuard dg(b->device);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "synchronizing");
    unsigned int word = 0;
    e = cudaMemcpy(&word, b->d_err, sizeof word, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "reading the error word");
    if (word) {
        cudaMemset(b->d_err, 0, sizeof word);
        if (word & fhp::kErrBounds)
            return bfail(b, FHP_EDEBUG,
                         "a debug-build index check failed (site %u, value %u, error word 0x%08x); the access "
                         "was skipped", (word >> 8) & 0xFFu, word >> 16, word);
        return bfail(b, FHP_ETIMEOUT, "a batch kernel gave up waiting for its input copies");
    }
    return FHP_OK;
}

int32_t fhp_batch_count(const fhp_batch* b) {
    if (!b) return -1;
    int32_t n = 0;
    for (const auto& m : b->members) n += m.used ? 1 : 0;
    return n;
}

size_t fhp_batch_free_bytes(const fhp_batch* b) { return b ? b->arena.free_bytes() : 0; }

int64_t fhp_batch_kernel_launches(const fhp_batch* b) { return b ? b->launches : -1; }

}  // extern "C"
