// fhp_batch_block.cu -- temporal blocking inside batches: one pass advances
// the members it lists by k (2 or 4) FHP steps.
//
// A member's rows are cut into tiles of R_out full rows (R_out even, chosen
// per member so that R_out + 2k staged rows of the member's row pitch fit
// one staged plane, kBBPlaneWords).  A CTA stages a tile with k rows above
// and below (periodic in y; rows are whole, so the periodic wrap in x stays
// inside the staged row and no column halo exists), applies the step k times
// in shared memory -- step j updates rows [j, R_in - j) of the block, the
// rows whose value equals the true S_{t+j} -- and stores the R_out rows of
// the last step to the member's other state buffer.  Motion, scattering,
// bounce-back and forcing are the per-quad code of every other kernel, with
// the random streams keyed on the global (quad, row, step), so a member's
// state after a pass equals k single steps bit for bit.  While step k runs,
// the CTA's next tile is already being copied (bulk copies of whole rows,
// completing on an mbarrier) into the buffer step k does not read.
//
// Tiles of one pass are independent (they read S_t and write S_{t+k} of
// their own member), so CTAs walk the pass's tile list with a stride of the
// grid and never wait for each other.
#include <cstdio>
#include <mutex>

#include "fhp_debug.cuh"
#include "fhp_device.cuh"
#include "fhp_internal.h"
#include "fhp_quad.cuh"

namespace fhp {
namespace {

constexpr int kBBThreads = 384;   // 12 warps: an inner step of a tile is ~700 quads
constexpr int kBBHeaderBytes = (int)((sizeof(BlockMember) + 127) / 128 * 128);
constexpr int kBBPrefix = 128 + 2 * kBBHeaderBytes;   // mbarrier, then two headers
// Shared memory: the staging mbarrier, two headers, then buffers A and B (7
// planes each) and two solid planes (one per tile parity), each plane
// kBBPlaneWords words.
constexpr size_t kBBSmem = kBBPrefix + (size_t)16 * kBBPlaneWords * 4;
static_assert(kBBSmem <= 227 * 1024, "the staged block must fit one CTA's shared memory");

__device__ __forceinline__ int bb_wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// Header of tile `tl` for pass `pass` (warp 0): the member's descriptor with
// src / dst / step of this pass, y0, the tile's row counts and whether the
// member takes this pass.
__device__ void bb_header(const BlockMember* __restrict__ mem, BlockTile tl, int pass, int k, BlockMember* h,
                          int lane) {
    const uint32_t* srcw = reinterpret_cast<const uint32_t*>(mem + tl.lattice);
    uint32_t* dstw = reinterpret_cast<uint32_t*>(h);
    constexpr int kWords = (int)(sizeof(BlockMember) / 4);
    for (int w = lane; w < kWords; w += 32) dstw[w] = srcw[w];
    __syncwarp();
    if (lane == 0) {
        const int par = (h->cur + pass) & 1;
        const unsigned long long t = h->t0 + (unsigned long long)pass * (unsigned long long)k;
        h->a.src = h->buf[par];
        h->a.dst = h->buf[par ^ 1];
        h->a.t_lo = (uint32_t)t;
        h->a.t_hi = (uint32_t)(t >> 32);
        h->y0 = tl.tile * h->R_out;
        h->rows_out = min(h->R_out, h->a.H - h->y0);
        h->active = pass < h->passes && dbg_ok_v(tl.tile >= 0 && h->y0 < h->a.H && h->R_out >= 1 &&
                                                     (h->rows_out + 2 * k) * h->a.Pq <= kBBPlaneWords,
                                                 h->a.err, kSiteBatchBlockHeader, (unsigned int)tl.tile);
    }
    __syncwarp();
}

// Stage the tile of header h (one thread): the seven planes of the member's
// state at the pass start into A, its solid plane into S, as bulk copies of
// whole rows; block row r is member row y0 - k + r (periodic), so each plane
// takes one copy per contiguous run of rows (one, or two where the block
// wraps around the member's last row).  The copies complete on `bar`; an
// inactive tile arrives on it with no bytes.
__device__ void bb_issue(const BlockMember& h, int k, uint32_t* A, uint32_t* S, uint64_t* bar) {
    if (!h.active) {
        mbar_arrive_expect_tx(bar, 0u);
        return;
    }
    const StepArgs& a = h.a;
    const int H = a.H, Pq = a.Pq;
    const int rows_in = h.rows_out + 2 * k;
    const uint32_t row_bytes = (uint32_t)Pq * 4u;
    mbar_arrive_expect_tx(bar, 8u * (uint32_t)rows_in * row_bytes);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int slot = 0; slot < 8; ++slot) {
        const uint32_t* plane = slot < 7 ? a.src + (size_t)slot * a.plane_words : a.solid;
        uint32_t* sp = slot < 7 ? A + (size_t)slot * kBBPlaneWords : S;
        int r = 0;
        while (r < rows_in) {
            const int yy = bb_wrap(h.y0 - k + r, H);
            const int run = min(rows_in - r, H - yy);   // contiguous rows up to the member's last row
            if (!dbg_ok_v(run >= 1 && (r + run) * Pq <= kBBPlaneWords, a.err, kSiteBatchBlockStage,
                          (unsigned int)r))
                break;   // (the barrier then waits for fewer bytes than announced and gives up)
            bulk_copy_g2s(sp + r * Pq, plane + (size_t)yy * Pq, (uint32_t)run * row_bytes, bar);
            r += run;
        }
    }
}

// Inner step j (1..k) of the staged block: rows [j, rows_in - j) from `src`
// (solid plane S) into `dst` (shared memory), or, at j = k, rows
// [k, k + rows_out) into the member's dst buffer in global memory.
template <bool FORCE>
__device__ __forceinline__ void bb_step(const BlockMember& h, int k, int j, const uint32_t* src, const uint32_t* S,
                                        uint32_t* dst) {
    const StepArgs& a = h.a;
    const int nq = a.nq, Pq = a.Pq, Wq = a.Wq, H = a.H;
    const int rows_in = h.rows_out + 2 * k;
    const int r0 = j, r1 = rows_in - j;
    const bool last = j == k;
    const unsigned long long t = (((unsigned long long)a.t_hi << 32) | a.t_lo) + (unsigned long long)(j - 1);
    const StepVar v{a.dst, (uint32_t)t, (uint32_t)(t >> 32)};
    // Items (row, quad): even block rows first, then odd ones.  Block row r
    // is member row y0 - k + r with y0 - k and H even, so the parity of r is
    // the row parity that selects the shift pattern.  A thread's items are
    // threadIdx.x + i * blockDim.x; their (row, quad) pairs advance by a
    // fixed step, so only the first item of each half is divided out.
    const int first_even = (r0 + 1) & ~1, first_odd = r0 | 1;
    const int n_even = (r1 - first_even + 1) >> 1, n_odd = (r1 - first_odd + 1) >> 1;
    const int even_items = n_even * nq;
    const int items = (n_even + n_odd) * nq;
    const int T = (int)blockDim.x;
    const int dk = T / nq, dq = T - dk * nq;
    const int ybase = h.y0 - k;
    constexpr int PW = kBBPlaneWords;
    int it = (int)threadIdx.x;
    int odd = it >= even_items;
    int kk = (odd ? it - even_items : it) / nq;
    int q = (odd ? it - even_items : it) - kk * nq;
    while (it < items) {
        const int r = (odd ? first_odd : first_even) + 2 * kk;
        int y = ybase + r;
        if (H >= k) {
            if (y < 0) y += H;
            if (y >= H) y -= H;
        } else {
            y = bb_wrap(y, H);
        }
        const int w = 4 * q;
        const int m = q == nq - 1 ? Wq - w : 4;
        const int wl = q == 0 ? Wq - 1 : w - 1;
        const int wr = q == nq - 1 ? 0 : w + 4;
        if (dbg_ok_v(r >= 1 && (r + 2) * Pq <= PW && w + 3 < Pq && wl >= 0 && wl < Wq && wr < Wq && y >= 0 && y < H,
                     a.err, kSiteBatchBlockQuad, (unsigned int)(r | (j << 12)))) {
            const uint32_t* rowm = src + (r - 1) * Pq;
            const uint32_t* row0 = src + r * Pq;
            const uint32_t* rowp = src + (r + 1) * Pq;
            const uint4 i3 = ld4(rowm + 3 * PW + w), i4 = ld4(rowm + 4 * PW + w);
            const uint4 i2 = ld4(row0 + 2 * PW + w), i5 = ld4(row0 + 5 * PW + w);
            const uint4 i6 = ld4(row0 + 6 * PW + w);
            const uint4 i0 = ld4(rowp + 0 * PW + w), i1 = ld4(rowp + 1 * PW + w);
            const uint4 sd = ld4(S + r * Pq + w);
            uint4 n0, n1, n2, n3, n4, n5;
            if (!odd) {
                // Even row: E, NE, SE come from x-1; W from x+1; NW, SW from x.
                n2 = pull_left(i2, row0[2 * PW + wl]);
                n3 = pull_left(i3, rowm[3 * PW + wl]);
                n1 = pull_left(i1, rowp[1 * PW + wl]);
                n5 = pull_right<true>(i5, row0[5 * PW + wr], m);
                n4 = i4;
                n0 = i0;
            } else {
                // Odd row: E from x-1; W, NW, SW from x+1; NE, SE from x.
                n2 = pull_left(i2, row0[2 * PW + wl]);
                n5 = pull_right<true>(i5, row0[5 * PW + wr], m);
                n4 = pull_right<true>(i4, rowm[4 * PW + wr], m);
                n0 = pull_right<true>(i0, rowp[0 * PW + wr], m);
                n3 = i3;
                n1 = i1;
            }
            uint4 o[7];
            collide_quad<true, FORCE>(a, v, q, y, n0, n1, n2, n3, n4, n5, i6, sd, o);
            if (last) {
                store_quad<true>(a, v.dst, q, y, m, o);
            } else {
                // (the padding words of a ragged last quad carry don't-care
                // values here: no valid word reads them, and the global store
                // zeroes them)
                uint32_t* drow = dst + r * Pq + w;
#pragma unroll
                for (int p = 0; p < 7; ++p) st4(drow + p * PW, o[p]);
            }
        }
        it += T;
        if (!odd && it >= even_items) {
            odd = 1;
            kk = (it - even_items) / nq;
            q = (it - even_items) - kk * nq;
        } else {
            q += dq;
            kk += dk;
            if (q >= nq) {
                q -= nq;
                ++kk;
            }
        }
    }
}

__global__ void __launch_bounds__(kBBThreads, 1)
    fhp_batch_block_kernel(const BlockMember* __restrict__ mem, const BlockTile* __restrict__ tiles, int ntiles,
                           int pass, int k, unsigned int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    auto hdr = [&](int i) { return reinterpret_cast<BlockMember*>(smem_raw + 128 + i * kBBHeaderBytes); };
    uint32_t* A = reinterpret_cast<uint32_t*>(smem_raw + kBBPrefix);
    uint32_t* B = A + 7 * kBBPlaneWords;
    auto S = [&](int i) { return B + (7 + i) * kBBPlaneWords; };
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    int tile = (int)blockIdx.x;
    if (tile >= ntiles) return;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) {
        bb_header(mem, tiles[tile], pass, k, hdr(0), lane);
        if (lane == 0) bb_issue(*hdr(0), k, A, S(0), bar);
    }
    int hb = 0;
    uint32_t phase = 0;
    for (; tile < ntiles; tile += (int)gridDim.x) {
        // Every thread waits (bounded) for the tile's copies; the CTA then
        // agrees, so that either all threads go on or all leave together.
        const bool got = mbar_wait_bounded(bar, phase);
        if (!__syncthreads_and(got)) {
            if (threadIdx.x == 0) {
                if (err) atomicOr(err, 1u);
                (void)mbar_wait_bounded(bar, phase);   // never leave with copies in flight
            }
            return;
        }
        phase ^= 1u;
        const BlockMember& h = *hdr(hb);
        // h.active and h.force are the same for every thread of the CTA (one
        // header), so the barriers below are taken by all threads or by none.
        if (h.active) {
            // Steps 1 .. k-1 alternate A -> B -> A ...; k is even, so step
            // k-1 writes B and step k reads B (and S(hb)) while A and
            // S(hb ^ 1) take the next tile.
            for (int j = 1; j < k; ++j) {
                const uint32_t* src = (j & 1) ? A : B;
                uint32_t* dst = (j & 1) ? B : A;
                if (h.force) bb_step<true>(h, k, j, src, S(hb), dst);
                else bb_step<false>(h, k, j, src, S(hb), dst);
                __syncthreads();
            }
        }
        const int next = tile + (int)gridDim.x;
        if (next < ntiles && warp == 0) {
            bb_header(mem, tiles[next], pass, k, hdr(hb ^ 1), lane);
            if (lane == 0) bb_issue(*hdr(hb ^ 1), k, A, S(hb ^ 1), bar);
        }
        if (h.active) {
            if (h.force) bb_step<true>(h, k, k, B, S(hb), nullptr);
            else bb_step<false>(h, k, k, B, S(hb), nullptr);
        }
        hb ^= 1;
        // (the next iteration's wait orders the step-k reads of B and S(hb)
        // before any thread overwrites them: its __syncthreads_and)
    }
}

std::mutex g_bb_mutex;
int g_bb_sms[64] = {};
bool g_bb_configured[64] = {};

}  // namespace

int batch_block_rows(const Geometry& g, int k) {
    if ((k != 2 && k != 4) || g.rules == 3) return 0;
    // Largest even R_out with (R_out + 2k) rows of the member's pitch in one
    // staged plane; a tile never needs more rows than the member has.
    int R = kBBPlaneWords / g.Pq - 2 * k;
    R &= ~1;
    if (R > g.H) R = g.H;
    // Below 4k output rows per tile the recomputed rows (k (k + 1) per tile)
    // cost more than a third of the work: not worth a blocked pass.
    return R >= 4 * k || R == g.H ? R : 0;
}

namespace {
cudaError_t configured_sms(int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(g_bb_mutex);
        if (!g_bb_sms[dev]) {
            e = cudaDeviceGetAttribute(&g_bb_sms[dev], cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
        }
        if (!g_bb_configured[dev]) {
            e = cudaFuncSetAttribute(fhp_batch_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kBBSmem);
            if (e != cudaSuccess) return e;
            g_bb_configured[dev] = true;
        }
        *sms = g_bb_sms[dev];
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t configure_batch_block() {
    int sms = 0;
    return configured_sms(&sms);
}

cudaError_t launch_batch_block(const BlockMember* d_members, const BlockTile* d_tiles, int ntiles, int pass, int k,
                               unsigned int* err, cudaStream_t stream) {
    if (ntiles <= 0) return cudaSuccess;
    if (k != 2 && k != 4) return cudaErrorInvalidValue;
    int sms = 0;
    const cudaError_t e = configured_sms(&sms);
    if (e != cudaSuccess) return e;
    const int grid = ntiles < sms ? ntiles : sms;
    fhp_batch_block_kernel<<<grid, kBBThreads, kBBSmem, stream>>>(d_members, d_tiles, ntiles, pass, k, err);
    return cudaGetLastError();
}

}  // namespace fhp
