// fhp_step.cu -- one fused FHP time step on bit-planes.
//
// The unit of work is a quad: 4 consecutive words (128 nodes) of one row y.
// For each quad the step computes S_{t+1}:
//   motion (arXiv:1208.2428 Section 2, Fig. 3): the particle moving along c_i
//     that arrives at (x, y) left (x, y) - c_i; row y-1 feeds the upward
//     movers (NE 3, NW 4), row y the horizontal movers (E 2, W 5) and the rest
//     particle, row y+1 the downward movers (SW 0, SE 1); the half-cell shift
//     of odd rows decides, per direction, whether the source sits one node to
//     the left, at the same x, or one node to the right.  One-node shifts are
//     funnel shifts across the quad's words plus one neighbour word (periodic
//     wrap in x);
//   scattering with bounce-back and forcing (fhp_device.cuh); one Philox
//     block gives the chirality bits of the quad's 128 nodes, a second one its
//     first forcing draws;
//   128-bit stores of the seven planes into the other ping-pong buffer.
//
// Two kernels share that per-quad code:
//   fhp_step_tma_kernel    persistent CTAs walk tiles of R full rows; a
//                          producer warp streams each tile's plane rows into
//                          a 3-stage shared-memory ring with cp.async.bulk
//                          (completion on mbarriers), so loads for the next
//                          tiles are in flight while 8 consumer warps compute;
//   fhp_step_direct_kernel one quad per thread, operands loaded straight into
//                          registers and neighbour words exchanged with
//                          __shfl_sync (used when a row is too wide to stage).
#include <cstdio>
#include <mutex>

#include "fhp_device.cuh"
#include "fhp_internal.h"
#include "fhp_quad.cuh"

namespace fhp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kBlock = 256;             // direct kernel
constexpr int kConsumerWarps = 8;       // bulk-copy kernel: compute warps
constexpr int kTmaThreads = (kConsumerWarps + 1) * 32;  // + one producer warp
constexpr int kRunThreads = (kConsumerWarps + 2) * 32;  // + producer and publisher warps
constexpr int kStages = 3;              // shared-memory ring depth
constexpr int kStageBudget = 32 * 1024; // bytes per stage
constexpr int kBarrierBytes = 128;      // mbarriers at the front of shared memory

// Warp-specialised ring: warp kConsumerWarps (the producer) streams the CTA's
// tiles into kStages shared-memory stages; "full" barriers (one arrival plus
// the copies' bytes) release a stage to the consumer warps, and "empty"
// barriers (one arrival per consumer warp) hand it back.  No block-wide
// barrier is taken after set-up, and every wait is bounded.
// SAT: the FHP-III rule set; its larger scattering network gets one CTA per
// SM and the registers of two.
template <bool SOLID, bool FORCE, bool RAGGED, bool SAT>
__global__ void __launch_bounds__(kTmaThreads, SAT ? 1 : 2) fhp_step_tma_kernel(const StepArgs a, const TileArgs ta) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + kStages;
    uint32_t* stages = reinterpret_cast<uint32_t*>(smem_raw + kBarrierBytes);
    constexpr int NP = SOLID ? 8 : 7;
    const size_t stage_words = (size_t)NP * ta.R * a.Pq;
    if (!dbg_ok(stage_words * 4 <= (size_t)kStageBudget, a.err, kSiteStageFit)) return;
    // Tiles of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int count = (ta.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    auto tile_of = [&](int i) { return (int)blockIdx.x + i * (int)gridDim.x; };
    auto stage_of = [&](int i) { return stages + (size_t)(i % kStages) * stage_words; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kConsumerWarps) {
        if (lane != 0) return;
        int i = 0;
        bool ok = true;
        for (; i < count; ++i) {
            const int s = i % kStages;
            if (i >= kStages && !mbar_wait_bounded(&empty[s], (uint32_t)(((i / kStages) - 1) & 1))) {
                ok = false;
                break;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_tile<SOLID>(a, ta, a.src, tile_of(i), stage_of(i), &full[s]);
        }
        if (!ok && a.err) atomicOr(a.err, 1u);
        // Never leave while copies into this CTA's shared memory may be in flight.
        for (int k = (i > kStages ? i - kStages : 0); k < i; ++k)
            (void)mbar_wait_bounded(&full[k % kStages], (uint32_t)((k / kStages) & 1));
        return;
    }

    const StepVar v{a.dst, a.t_lo, a.t_hi};
    for (int i = 0; i < count; ++i) {
        const int s = i % kStages;
        if (!mbar_wait_bounded_call(&full[s], (uint32_t)((i / kStages) & 1))) {
            if (lane == 0 && a.err) atomicOr(a.err, 1u);
            return;
        }
        compute_tile<SOLID, FORCE, RAGGED, SAT>(a, v, ta, tile_of(i), stage_of(i), (int)threadIdx.x,
                                                kConsumerWarps * 32);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ---------------------------------------------------------------------------
// Multi-step kernel: all n steps in one cooperative launch.  Tiles of step s
// depend only on the three tiles of step s-1 that hold their source rows
// (tile j reads rows y0-1 .. y0+R of the previous state), so instead of a
// grid-wide barrier per step every tile carries a counter of consumer warps
// that finished it (bumped by a publisher warp after a GPU-scope fence, so
// neither the compute warps nor stage reuse wait on a fence); the producer of
// (s, j) waits (bounded) until tiles j-1, j, j+1 reached kConsumerWarps * s
// before streaming its inputs.  That also
// makes the write of (s, j) safe: the three tiles that read the old rows of j
// (at step s-1) have finished.  All CTAs are co-resident (cooperative launch)
// and each walks its items in step order, so every wait is for an item that
// is already running or finished.
// ---------------------------------------------------------------------------
struct RunArgs {
    uint32_t* buf0;          // state S_{t0} (also StepArgs::src)
    uint32_t* buf1;          // the other buffer (StepArgs::dst)
    unsigned int* done;      // per-tile finished-warp counters, zero at launch
    int nsteps;
    unsigned long long t0;
};

template <bool SOLID, bool FORCE, bool RAGGED, bool SAT>
__global__ void __launch_bounds__(kRunThreads, SAT ? 1 : 2) fhp_run_kernel(const StepArgs a, const TileArgs ta,
                                                                           const RunArgs ra) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + kStages;  // all consumer warps finished the stage's tile
    // warp_done[w]: number of items consumer warp w has finished (written
    // with release, read by the publisher with acquire).
    unsigned int* warp_done = reinterpret_cast<unsigned int*>(empty + kStages);
    uint32_t* stages = reinterpret_cast<uint32_t*>(smem_raw + kBarrierBytes);
    constexpr int NP = SOLID ? 8 : 7;
    const size_t stage_words = (size_t)NP * ta.R * a.Pq;
    if (!dbg_ok(stage_words * 4 <= (size_t)kStageBudget, a.err, kSiteStageFit)) return;
    const int count = (ta.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        for (int w = 0; w < kConsumerWarps; ++w) warp_done[w] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kConsumerWarps + 1) {
        // Publisher: every item all consumer warps have finished gets its
        // tile counter bumped after one GPU-scope fence; when it falls
        // behind, one fence covers several items.  The compute warps never
        // wait on a fence and stage reuse never waits on the publisher.
        if (lane != 0) return;
        const long long total = (long long)count * ra.nsteps;
        long long published = 0;
        int i_next = 0;  // tile index (within this CTA) of item `published`
        unsigned long long start = 0;
        while (published < total) {
            unsigned int m = 0xFFFFFFFFu;
            for (int w = 0; w < kConsumerWarps; ++w) m = min(m, ld_acquire_cta_shared(&warp_done[w]));
            if ((long long)m > published) {
                asm volatile("fence.proxy.async.global;" ::: "memory");
                asm volatile("fence.acq_rel.gpu;" ::: "memory");
                for (; published < (long long)m; ++published) {
                    atomicAdd(&ra.done[(int)blockIdx.x + i_next * (int)gridDim.x], (unsigned int)kConsumerWarps);
                    if (++i_next == count) i_next = 0;
                }
                start = 0;
                continue;
            }
            const unsigned long long now = global_ns();
            if (start == 0) start = now;
            else if (now - start > kWaitLimitNs) {
                if (a.err) atomicOr(a.err, 1u);
                return;
            }
            __nanosleep(64);
        }
        return;
    }

    if (warp == kConsumerWarps) {
        if (lane != 0) return;
        // Item k = s * count + i goes to stage k % kStages; its "full" phase
        // parity is (k / kStages) & 1, and it may reuse the stage once the
        // "empty" phase of item k - kStages (parity flipped) has completed.
        long long k = 0;
        int st = 0;
        uint32_t par = 0;
        bool ok = true;
        for (int s = 0; ok && s < ra.nsteps; ++s) {
            const uint32_t* src = (s & 1) ? ra.buf1 : ra.buf0;
            const unsigned int target = (unsigned int)kConsumerWarps * (unsigned int)s;
            for (int i = 0; i < count; ++i) {
                const int tile = (int)blockIdx.x + i * (int)gridDim.x;
                if (k >= kStages && !mbar_wait_bounded(&empty[st], par ^ 1u)) {
                    ok = false;
                    break;
                }
                if (s > 0) {
                    // Tiles prev, tile, next of step s - 1 hold the source rows.
                    const int prev = tile == 0 ? ta.ntiles - 1 : tile - 1;
                    const int next = tile == ta.ntiles - 1 ? 0 : tile + 1;
                    if (!wait_tiles(ra.done, prev, next, tile, true, target)) {
                        ok = false;
                        break;
                    }
                    // The rows were written through the generic proxy by other
                    // warps and CTAs; the bulk copy reads them through the
                    // async proxy.
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_tile<SOLID>(a, ta, src, tile, stages + (size_t)st * stage_words, &full[st]);
                ++k;
                if (++st == kStages) {
                    st = 0;
                    par ^= 1u;
                }
            }
        }
        if (!ok && a.err) atomicOr(a.err, 1u);
        // Never leave while copies into this CTA's shared memory may be in flight.
        for (long long j = (k > kStages ? k - kStages : 0); j < k; ++j)
            (void)mbar_wait_bounded(&full[j % kStages], (uint32_t)((j / kStages) & 1));
        return;
    }

    int st = 0;
    uint32_t par = 0;
    unsigned int finished = 0;
    for (int s = 0; s < ra.nsteps; ++s) {
        const unsigned long long t = ra.t0 + (unsigned long long)s;
        const StepVar v{(s & 1) ? ra.buf0 : ra.buf1, (uint32_t)t, (uint32_t)(t >> 32)};
        for (int i = 0; i < count; ++i) {
            const int tile = (int)blockIdx.x + i * (int)gridDim.x;
            if (!mbar_wait_bounded(&full[st], par)) {
                if (lane == 0 && a.err) atomicOr(a.err, 1u);
                return;
            }
            compute_tile<SOLID, FORCE, RAGGED, SAT>(a, v, ta, tile, stages + (size_t)st * stage_words,
                                                    (int)threadIdx.x, kConsumerWarps * 32);
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[st]);                        // the stage may be refilled
                st_release_cta_shared(&warp_done[warp], ++finished);  // this warp's rows are written
            }
            if (++st == kStages) {
                st = 0;
                par ^= 1u;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Direct kernel: one quad per thread, neighbour words by warp shuffles.
// ---------------------------------------------------------------------------
struct Lane {
    int y, q;
    bool active;
    int src_left, src_right;     // lanes holding the quads to the left / right
    bool glob_left, glob_right;  // neighbour quad outside the warp: load it
};

__device__ __forceinline__ Lane map_lane(const StepArgs& a) {
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    Lane L;
    if (a.nq >= 32) {
        const long long y = gw / a.warps_per_row;
        const int seg = (int)(gw - y * a.warps_per_row);
        const int q = seg * 32 + lane;
        L.active = y < a.H && q < a.nq;
        L.y = y < a.H ? (int)y : 0;
        L.q = q < a.nq ? q : a.nq - 1;
        L.src_left = lane == 0 ? 0 : lane - 1;
        L.src_right = lane == 31 ? 31 : lane + 1;
        L.glob_left = lane == 0;
        L.glob_right = lane == 31 || q == a.nq - 1;
    } else {
        const int par = (int)(gw / a.groups_per_parity);
        const int grp = (int)(gw - (long long)par * a.groups_per_parity);
        const int r = lane / a.nq;
        const int qi = lane - r * a.nq;
        const int m = grp * a.rows_per_warp + r;
        L.active = par < 2 && r < a.rows_per_warp && m < (a.H >> 1);
        L.y = L.active ? 2 * m + par : (par & 1);
        L.q = qi;
        L.src_left = qi == 0 ? lane + a.nq - 1 : lane - 1;
        L.src_right = qi == a.nq - 1 ? lane - (a.nq - 1) : lane + 1;
        L.glob_left = false;
        L.glob_right = false;
    }
    return L;
}

template <bool RAGGED>
__device__ __forceinline__ uint32_t left_word(uint4 v, uint32_t fallback, const Lane& L, int m) {
    uint32_t offer = v.w;  // the quad's last valid word, for the lane to the right
    if (RAGGED) offer = m == 4 ? v.w : m == 3 ? v.z : m == 2 ? v.y : v.x;
    const uint32_t left = __shfl_sync(kFull, offer, L.src_left);
    return L.glob_left ? fallback : left;
}

__device__ __forceinline__ uint32_t right_word(uint4 v, uint32_t fallback, const Lane& L) {
    const uint32_t right = __shfl_sync(kFull, v.x, L.src_right);
    return L.glob_right ? fallback : right;
}

template <bool SOLID, bool FORCE, bool RAGGED, bool ODD, bool SAT>
__device__ __forceinline__ void direct_quad(const StepArgs& a, const Lane& L) {
    const size_t pw = a.plane_words;
    // Debug builds: an index outside the lattice reads row 0 / quad 0 instead
    // and stores nothing (the lanes must still take part in the shuffles).
    const bool in_range = dbg_ok(L.y >= 0 && L.y < a.H && L.q >= 0 && L.q < a.nq, a.err, kSiteDirectQuad);
    const int y = in_range ? L.y : 0;
    const int ym = y == 0 ? a.H - 1 : y - 1;
    const int yp = y == a.H - 1 ? 0 : y + 1;
    const int qi = in_range ? L.q : 0;
    const int w = 4 * qi;
    const uint32_t* rm = a.src + (size_t)ym * a.Pq;  // row y-1 of plane 0
    const uint32_t* r0 = a.src + (size_t)y * a.Pq;   // row y
    const uint32_t* rp = a.src + (size_t)yp * a.Pq;  // row y+1
    const int m = RAGGED ? (qi == a.nq - 1 ? a.Wq - w : 4) : 4;
    const int wl = qi == 0 ? a.Wq - 1 : w - 1;
    const int wr = qi == a.nq - 1 ? 0 : w + 4;

    const uint4 i3 = ld4(rm + 3 * pw + w), i4 = ld4(rm + 4 * pw + w);
    const uint4 i2 = ld4(r0 + 2 * pw + w), i5 = ld4(r0 + 5 * pw + w);
    const uint4 i6 = ld4(r0 + 6 * pw + w);
    const uint4 i0 = ld4(rp + 0 * pw + w), i1 = ld4(rp + 1 * pw + w);
    uint4 sd = make_uint4(0u, 0u, 0u, 0u);
    if (SOLID) sd = ld4(a.solid + (size_t)y * a.Pq + w);

    uint4 n0, n1, n2, n3, n4, n5;
    if (!ODD) {
        uint32_t f2 = 0, f3 = 0, f1 = 0, f5 = 0;
        if (L.glob_left) { f2 = r0[2 * pw + wl]; f3 = rm[3 * pw + wl]; f1 = rp[1 * pw + wl]; }
        if (L.glob_right) f5 = r0[5 * pw + wr];
        n2 = pull_left(i2, left_word<RAGGED>(i2, f2, L, m));
        n3 = pull_left(i3, left_word<RAGGED>(i3, f3, L, m));
        n1 = pull_left(i1, left_word<RAGGED>(i1, f1, L, m));
        n5 = pull_right<RAGGED>(i5, right_word(i5, f5, L), m);
        n4 = i4;
        n0 = i0;
    } else {
        uint32_t f2 = 0, f5 = 0, f4 = 0, f0 = 0;
        if (L.glob_left) f2 = r0[2 * pw + wl];
        if (L.glob_right) { f5 = r0[5 * pw + wr]; f4 = rm[4 * pw + wr]; f0 = rp[0 * pw + wr]; }
        n2 = pull_left(i2, left_word<RAGGED>(i2, f2, L, m));
        n5 = pull_right<RAGGED>(i5, right_word(i5, f5, L), m);
        n4 = pull_right<RAGGED>(i4, right_word(i4, f4, L), m);
        n0 = pull_right<RAGGED>(i0, right_word(i0, f0, L), m);
        n3 = i3;
        n1 = i1;
    }
    const StepVar v{a.dst, a.t_lo, a.t_hi};
    finish_quad<SOLID, FORCE, RAGGED, SAT>(a, v, L.q, y, m, n0, n1, n2, n3, n4, n5, i6, sd, L.active && in_range);
}

// SAT: the FHP-III rule set (its larger scattering network gets twice the
// registers).
template <bool SOLID, bool FORCE, bool RAGGED, bool SAT>
__global__ void __launch_bounds__(kBlock, SAT ? 2 : 4) fhp_step_direct_kernel(const StepArgs a) {
    const Lane L = map_lane(a);
    if (L.y & 1) direct_quad<SOLID, FORCE, RAGGED, true, SAT>(a, L);
    else direct_quad<SOLID, FORCE, RAGGED, false, SAT>(a, L);
}

__global__ void philox_kernel(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                              uint32_t* __restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
        const uint4 r = philox4x32_10(c, Key2{key[2 * i], key[2 * i + 1]});
        out[4 * i] = r.x;
        out[4 * i + 1] = r.y;
        out[4 * i + 2] = r.z;
        out[4 * i + 3] = r.w;
    }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct DeviceInfo {
    int sms = 0;
    int tma_blocks_per_sm[16] = {};  // per kernel variant (sat, solid, force, ragged)
    bool configured[16] = {};
    int run_blocks_per_sm[16] = {};
    bool run_configured[16] = {};
};
std::mutex g_dev_mutex;
DeviceInfo g_dev[64];

template <bool SOLID, bool FORCE, bool RAGGED, bool SAT>
cudaError_t launch_tma_variant(const StepArgs& a, const TileArgs& ta, size_t smem, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const int variant = (SAT ? 8 : 0) | (SOLID ? 4 : 0) | (FORCE ? 2 : 0) | (RAGGED ? 1 : 0);
    auto kernel = fhp_step_tma_kernel<SOLID, FORCE, RAGGED, SAT>;
    int blocks_per_sm, sms;
    {
        std::lock_guard<std::mutex> lock(g_dev_mutex);
        DeviceInfo& d = g_dev[dev];
        if (!d.sms) {
            e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
        }
        if (!d.configured[variant]) {
            const int max_smem = kBarrierBytes + kStages * kStageBudget;
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
            if (e != cudaSuccess) return e;
            int n = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kTmaThreads, max_smem);
            if (e != cudaSuccess) return e;
            d.tma_blocks_per_sm[variant] = n > 0 ? n : 1;
            d.configured[variant] = true;
        }
        blocks_per_sm = d.tma_blocks_per_sm[variant];
        sms = d.sms;
    }
    const int grid = min(ta.ntiles, blocks_per_sm * sms);
    kernel<<<grid, kTmaThreads, smem, s>>>(a, ta);
    return cudaGetLastError();
}

template <bool SOLID, bool FORCE, bool RAGGED, bool SAT>
cudaError_t launch_run_variant(const StepArgs& a, const TileArgs& ta, const RunArgs& ra, size_t smem,
                               cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const int variant = (SAT ? 8 : 0) | (SOLID ? 4 : 0) | (FORCE ? 2 : 0) | (RAGGED ? 1 : 0);
    auto kernel = fhp_run_kernel<SOLID, FORCE, RAGGED, SAT>;
    int blocks_per_sm, sms;
    {
        std::lock_guard<std::mutex> lock(g_dev_mutex);
        DeviceInfo& d = g_dev[dev];
        if (!d.sms) {
            e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
        }
        if (!d.run_configured[variant]) {
            const int max_smem = kBarrierBytes + kStages * kStageBudget;
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
            if (e != cudaSuccess) return e;
            int n = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kRunThreads, max_smem);
            if (e != cudaSuccess) return e;
            d.run_blocks_per_sm[variant] = n > 0 ? n : 1;
            d.run_configured[variant] = true;
        }
        blocks_per_sm = d.run_blocks_per_sm[variant];
        sms = d.sms;
    }
    // Every CTA must be resident at once (they wait on each other's tiles):
    // a cooperative launch with at most the co-resident number of CTAs.
    const int grid = min(ta.ntiles, blocks_per_sm * sms);
    StepArgs a_copy = a;
    TileArgs ta_copy = ta;
    RunArgs ra_copy = ra;
    void* args[] = {&a_copy, &ta_copy, &ra_copy};
    e = cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(kRunThreads), args, smem, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <bool SOLID, bool FORCE>
cudaError_t launch_run(const StepArgs& a, const TileArgs& ta, const RunArgs& ra, size_t smem, bool ragged,
                       bool sat, cudaStream_t s) {
    if (sat)
        return ragged ? launch_run_variant<SOLID, FORCE, true, true>(a, ta, ra, smem, s)
                      : launch_run_variant<SOLID, FORCE, false, true>(a, ta, ra, smem, s);
    return ragged ? launch_run_variant<SOLID, FORCE, true, false>(a, ta, ra, smem, s)
                  : launch_run_variant<SOLID, FORCE, false, false>(a, ta, ra, smem, s);
}

template <bool SOLID, bool FORCE>
cudaError_t launch_tma(const StepArgs& a, const TileArgs& ta, size_t smem, bool ragged, bool sat, cudaStream_t s) {
    if (sat)
        return ragged ? launch_tma_variant<SOLID, FORCE, true, true>(a, ta, smem, s)
                      : launch_tma_variant<SOLID, FORCE, false, true>(a, ta, smem, s);
    return ragged ? launch_tma_variant<SOLID, FORCE, true, false>(a, ta, smem, s)
                  : launch_tma_variant<SOLID, FORCE, false, false>(a, ta, smem, s);
}

template <bool SOLID, bool FORCE>
cudaError_t launch_direct(const StepArgs& a, bool ragged, bool sat, long long warps, cudaStream_t s) {
    const long long threads = warps * 32;
    const unsigned grid = (unsigned)((threads + kBlock - 1) / kBlock);
    if (sat) {
        if (ragged) fhp_step_direct_kernel<SOLID, FORCE, true, true><<<grid, kBlock, 0, s>>>(a);
        else fhp_step_direct_kernel<SOLID, FORCE, false, true><<<grid, kBlock, 0, s>>>(a);
    } else {
        if (ragged) fhp_step_direct_kernel<SOLID, FORCE, true, false><<<grid, kBlock, 0, s>>>(a);
        else fhp_step_direct_kernel<SOLID, FORCE, false, false><<<grid, kBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// Rows per tile of the bulk-copy kernel, or 0 if one row does not fit a stage.
int tile_rows(const Geometry& g, bool has_solid) {
    const int np = has_solid ? 8 : 7;
    const long long row_bytes = (long long)np * g.Pq * 4;
    if (row_bytes > kStageBudget) return 0;
    int R = (int)(kStageBudget / row_bytes);
    return R < g.H ? R : g.H;
}

}  // namespace

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                          cudaStream_t stream) {
    long long blocks = (n + kBlock - 1) / kBlock;
    if (blocks > 4096) blocks = 4096;
    philox_kernel<<<(unsigned)blocks, kBlock, 0, stream>>>(ctr, key, out, (long long)n);
    return cudaGetLastError();
}

Geometry make_geometry(int W, int H) {
    Geometry g;
    g.W = W;
    g.H = H;
    g.Wq = W / 32;
    g.nq = (g.Wq + 3) / 4;
    g.Pq = 4 * g.nq;
    g.plane_words = (size_t)H * g.Pq;
    return g;
}

int resolved_step_kernel(const Geometry& g, bool has_solid, int requested) {
    const int R = tile_rows(g, has_solid);
    if (R == 0 || requested == kStepDirect) return kStepDirect;
    if (requested == kStepRing || requested == kStepRun) return requested;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return kStepDirect;
    {
        std::lock_guard<std::mutex> lock(g_dev_mutex);
        if (!g_dev[dev].sms && cudaDeviceGetAttribute(&g_dev[dev].sms, cudaDevAttrMultiProcessorCount, dev) !=
                                   cudaSuccess)
            return kStepDirect;
        sms = g_dev[dev].sms;
    }
    // Few tiles per CTA and step: launch gaps and per-step pipeline refills
    // dominate, so run all steps in one launch (measured on GB300: 903 vs 682
    // GSUPS on 4096 x 1024, 235 vs 171 on 2048 x 512).  Many tiles per CTA:
    // the per-step overhead is small and the single-step ring streams best.
    // A lattice of a handful of tiles is faster with the direct kernel.
    const int ntiles = (g.H + R - 1) / R;
    if (ntiles < 8) return kStepDirect;
    return ntiles <= 12 * 2 * sms ? kStepRun : kStepRing;
}

int run_tiles(const Geometry& g, bool has_solid) {
    const int R = tile_rows(g, has_solid);
    return R > 0 ? (g.H + R - 1) / R : 0;
}

cudaError_t launch_run(const Geometry& g, uint32_t* buf0, uint32_t* buf1, const uint32_t* solid,
                       bool has_solid, bool force, const ForcingTable& ft, Key2 key, uint64_t t0,
                       int nsteps, unsigned int* done, cudaStream_t stream, unsigned int* err) {
    const int R = tile_rows(g, has_solid);
    if (R == 0 || nsteps <= 0) return cudaErrorInvalidValue;
    StepArgs a;
    a.src = buf0;
    a.dst = buf1;
    a.solid = solid;
    a.plane_words = g.plane_words;
    a.H = g.H;
    a.Wq = g.Wq;
    a.nq = g.nq;
    a.Pq = g.Pq;
    a.rows_per_warp = a.groups_per_parity = a.warps_per_row = 1;
    a.key = key;
    a.y_base = g.row_base;
    a.rest_rules = rest_rules_mask(g);
    a.t_lo = (uint32_t)t0;
    a.t_hi = (uint32_t)(t0 >> 32);
    a.err = err;
    a.ft = ft;
    TileArgs ta;
    ta.R = R;
    ta.ntiles = (g.H + R - 1) / R;
    ta.nq_magic = ((1ull << 32) + g.nq - 1) / g.nq;
    RunArgs ra;
    ra.buf0 = buf0;
    ra.buf1 = buf1;
    ra.done = done;
    ra.nsteps = nsteps;
    ra.t0 = t0;
    cudaError_t e = cudaMemsetAsync(done, 0, (size_t)ta.ntiles * sizeof(unsigned int), stream);
    if (e != cudaSuccess) return e;
    const size_t smem = kBarrierBytes + (size_t)kStages * (has_solid ? 8 : 7) * R * g.Pq * 4;
    const bool ragged = (g.Wq % 4) != 0;
    const bool sat = g.rules == 3;
    if (has_solid)
        return force ? launch_run<true, true>(a, ta, ra, smem, ragged, sat, stream)
                     : launch_run<true, false>(a, ta, ra, smem, ragged, sat, stream);
    return force ? launch_run<false, true>(a, ta, ra, smem, ragged, sat, stream)
                 : launch_run<false, false>(a, ta, ra, smem, ragged, sat, stream);
}

cudaError_t launch_step(const Geometry& g, const uint32_t* src, uint32_t* dst,
                        const uint32_t* solid, bool has_solid, bool force,
                        const ForcingTable& ft, Key2 key, uint64_t t, cudaStream_t stream,
                        unsigned int* err, int kernel) {
    StepArgs a;
    a.src = src;
    a.dst = dst;
    a.solid = solid;
    a.plane_words = g.plane_words;
    a.H = g.H;
    a.Wq = g.Wq;
    a.nq = g.nq;
    a.Pq = g.Pq;
    a.key = key;
    a.y_base = g.row_base;
    a.rest_rules = rest_rules_mask(g);
    a.t_lo = (uint32_t)t;
    a.t_hi = (uint32_t)(t >> 32);
    a.err = err;
    a.ft = ft;
    const bool ragged = (g.Wq % 4) != 0;
    const int R = tile_rows(g, has_solid);
    if (resolved_step_kernel(g, has_solid, kernel) != kStepDirect) {
        TileArgs ta;
        ta.R = R;
        ta.ntiles = (g.H + R - 1) / R;
        ta.nq_magic = ((1ull << 32) + g.nq - 1) / g.nq;
        a.rows_per_warp = a.groups_per_parity = a.warps_per_row = 1;
        const size_t smem = kBarrierBytes + (size_t)kStages * (has_solid ? 8 : 7) * R * g.Pq * 4;
        const bool sat = g.rules == 3;
        if (has_solid)
            return force ? launch_tma<true, true>(a, ta, smem, ragged, sat, stream)
                         : launch_tma<true, false>(a, ta, smem, ragged, sat, stream);
        return force ? launch_tma<false, true>(a, ta, smem, ragged, sat, stream)
                     : launch_tma<false, false>(a, ta, smem, ragged, sat, stream);
    }
    long long warps;
    if (g.nq >= 32) {
        a.warps_per_row = (g.nq + 31) / 32;
        a.rows_per_warp = 1;
        a.groups_per_parity = 1;
        warps = (long long)g.H * a.warps_per_row;
    } else {
        a.warps_per_row = 1;
        a.rows_per_warp = 32 / g.nq;
        a.groups_per_parity = ((g.H / 2) + a.rows_per_warp - 1) / a.rows_per_warp;
        warps = 2LL * a.groups_per_parity;
    }
    if (has_solid)
        return force ? launch_direct<true, true>(a, ragged, g.rules == 3, warps, stream)
                     : launch_direct<true, false>(a, ragged, g.rules == 3, warps, stream);
    return force ? launch_direct<false, true>(a, ragged, g.rules == 3, warps, stream)
                 : launch_direct<false, false>(a, ragged, g.rules == 3, warps, stream);
}

}  // namespace fhp
