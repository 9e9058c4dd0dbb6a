// fhp_block.cu -- temporal blocking: k FHP steps per pass over the lattice.
//
// One pass reads S_t and writes S_{t+k} (k = 2, 4 or 8).  The lattice is cut
// into tiles of R_out rows x QO quads (a quad is 4 words = 128 nodes).  A CTA
// loads a tile with a halo of k rows above and below and ceil(k/4) quads on
// either side into shared memory (periodic wrap in x and y), then applies the step k times in shared memory: step j
// updates rows [j, R_in - j) of the staged block from one buffer into the
// other, so the region whose values equal the true S_{t+j} shrinks by one
// row and one word per step at every edge; step k computes only the
// R_out x QO interior and stores it to global memory.  Motion, scattering, bounce-back and
// forcing are the same per-quad code as the single-step kernels, with the
// random streams keyed on the global (quad, row, step), so results are
// bit-identical for every k.  While step k runs, the next tile is already
// being copied (cp.async, 16 bytes per copy, issued by every thread) into the
// buffer step k does not read.
#include <cstdio>
#include <mutex>

#include "fhp_debug.cuh"
#include "fhp_device.cuh"
#include "fhp_internal.h"
#include "fhp_quad.cuh"

namespace fhp {
namespace {

constexpr int kBlockThreads = 512;
constexpr int kQI = 18;                     // staged quads per row (interior + halo)
constexpr int kRin = 44;                    // staged rows (R_out + 2k)
constexpr int kRowWords = kQI * 4;          // words of one staged row
constexpr int kBarBytes = 128;

// Halo width.  Vertically a node's value depends on rows within one row per
// step, so k rows suffice.  Horizontally motion moves one node per step, but
// forcing decides the nodes of a 32-node word together (one draw sequence
// walks the word's candidates), so a wrong node anywhere in a word can change
// every node of it: the region that is not yet exact grows by one whole word
// per step.  k steps therefore need k words = ceil(k / 4) quads on each side.
struct BlockArgs {
    int k;            // steps per pass
    int hq;           // halo quads per side, ceil(k / 4)
    int qo;           // interior quads per tile, kQI - 2 hq
    int R_out;        // interior rows per tile
    int row_tiles;    // ceil(H / R_out)
    int col_tiles;    // ceil(nq / qo)
    int ntiles;       // row_tiles * col_tiles
    unsigned long long t0;
};

__device__ __forceinline__ int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)), "l"(gmem_src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Stage the tile (row tile tr, column tile tc): the seven state planes into
// buffer A, the solid plane into S; row r of the block is global row
// y0 - k + r, quad qi is global quad q0 - hq + qi (both periodic).  Every
// thread issues asynchronous 16-byte copies (cp.async) of whole quads; the
// caller waits for them (cp.async.wait_group) before the block is read.
template <bool SOLID>
__device__ void stage_tile(const StepArgs& a, const BlockArgs& b, int tile, uint32_t* A, uint32_t* S) {
    constexpr int NP = SOLID ? 8 : 7;
    const int tr = tile / b.col_tiles, tc = tile - tr * b.col_tiles;
    const int y0 = tr * b.R_out, q0 = tc * b.qo;
    const int rows = min(b.R_out, a.H - y0) + 2 * b.k;
    const int qo = min(b.qo, a.nq - q0);
    const int qi_n = qo + 2 * b.hq;
    const size_t pws = (size_t)kRin * kRowWords;
    // thread -> (quad column, row lane); rows are walked by row lanes
    const int col = threadIdx.x % kQI, lanes = blockDim.x / kQI, rl = threadIdx.x / kQI;
    if (col < qi_n && rl < lanes) {
        const int q = wrap(q0 - b.hq + col, a.nq);
        for (int job = rl; job < NP * rows; job += lanes) {
            const int slot = job / rows, r = job - slot * rows;
            const int y = wrap(y0 - b.k + r, a.H);
            if (!dbg_ok(r < kRin && col < kQI && q >= 0 && q < a.nq, a.err, kSiteBlockStage)) continue;
            const uint32_t* plane = slot < 7 ? a.src + (size_t)slot * a.plane_words : a.solid;
            uint32_t* srow = (slot < 7 ? A + slot * pws : S) + (size_t)r * kRowWords;
            cp_async16(srow + 4 * col, plane + (size_t)y * a.Pq + 4 * q);
        }
    }
    cp_async_commit();
}

// One step of the staged block: rows [r0, r1) x quads [c0, c1) of the block
// from buffer `src` (solid plane `S`) into buffer `dst`, or into global
// memory when `last`.
template <bool SOLID, bool FORCE>
__device__ __forceinline__ void block_step(const StepArgs& a, const BlockArgs& b, int tile, int j,
                                           const uint32_t* src, const uint32_t* S, uint32_t* dst, bool last,
                                           uint32_t* gdst) {
    const int tr = tile / b.col_tiles, tc = tile - tr * b.col_tiles;
    const int y0 = tr * b.R_out, q0 = tc * b.qo;
    const int rows = min(b.R_out, a.H - y0) + 2 * b.k;
    const int qo = min(b.qo, a.nq - q0);
    const int qi_n = qo + 2 * b.hq;
    const int r0 = j, r1 = rows - j;                 // rows of the block updated at step j
    const int c0 = last ? b.hq : 0, c1 = last ? b.hq + qo : qi_n;
    const int width = c1 - c0;
    const unsigned long long t = b.t0 + (unsigned long long)(j - 1);
    const StepVar v{gdst, (uint32_t)t, (uint32_t)(t >> 32)};
    const size_t pws = (size_t)kRin * kRowWords;    // words per staged plane
    // Thread -> (quad column c, row lane); a row lane walks rows of one
    // parity, even block rows first then odd ones (the rows of one group
    // share their global parity, which selects the shift pattern).
    const int lanes = blockDim.x / kQI;
    const int cl = threadIdx.x % kQI, rl = threadIdx.x / kQI;
    const int c = c0 + cl;
    if (cl >= width || rl >= lanes) return;
    const int first_even = (r0 + 1) & ~1;
    const int first_odd = r0 | 1;
    const int n_even = (r1 - first_even + 1) / 2;
    const int n_odd = (r1 - first_odd + 1) / 2;
    const int q = wrap(q0 - b.hq + c, a.nq);
    for (int it = rl; it < n_even + n_odd; it += lanes) {
        const int r = it < n_even ? first_even + 2 * it : first_odd + 2 * (it - n_even);
        const int y = wrap(y0 - b.k + r, a.H);
        const int w = 4 * c;
        if (!dbg_ok(r >= 1 && r + 1 < kRin && c < kQI, a.err, kSiteBlockStage)) continue;
        const uint32_t* rowm = src + (size_t)(r - 1) * kRowWords;
        const uint32_t* row0 = src + (size_t)r * kRowWords;
        const uint32_t* rowp = src + (size_t)(r + 1) * kRowWords;
        const uint4 i3 = ld4(rowm + 3 * pws + w), i4 = ld4(rowm + 4 * pws + w);
        const uint4 i2 = ld4(row0 + 2 * pws + w), i5 = ld4(row0 + 5 * pws + w);
        const uint4 i6 = ld4(row0 + 6 * pws + w);
        const uint4 i0 = ld4(rowp + 0 * pws + w), i1 = ld4(rowp + 1 * pws + w);
        uint4 sd = make_uint4(0u, 0u, 0u, 0u);
        if (SOLID) sd = ld4(S + (size_t)r * kRowWords + w);
        // neighbour words outside the staged block are unknown: use 0 (the
        // values they feed lie outside the valid region)
        const bool has_l = c > 0, has_r = c < qi_n - 1;
        uint4 n0, n1, n2, n3, n4, n5;
        if ((y & 1) == 0) {
            n2 = pull_left(i2, has_l ? row0[2 * pws + w - 1] : 0u);
            n3 = pull_left(i3, has_l ? rowm[3 * pws + w - 1] : 0u);
            n1 = pull_left(i1, has_l ? rowp[1 * pws + w - 1] : 0u);
            n5 = pull_right<false>(i5, has_r ? row0[5 * pws + w + 4] : 0u, 4);
            n4 = i4;
            n0 = i0;
        } else {
            n2 = pull_left(i2, has_l ? row0[2 * pws + w - 1] : 0u);
            n5 = pull_right<false>(i5, has_r ? row0[5 * pws + w + 4] : 0u, 4);
            n4 = pull_right<false>(i4, has_r ? rowm[4 * pws + w + 4] : 0u, 4);
            n0 = pull_right<false>(i0, has_r ? rowp[0 * pws + w + 4] : 0u, 4);
            n3 = i3;
            n1 = i1;
        }
        uint4 o[7];
        collide_quad<SOLID, FORCE>(a, v, q, y, n0, n1, n2, n3, n4, n5, i6, sd, o);
        if (last) {
            store_quad<false>(a, gdst, q, y, 4, o);
        } else {
            uint32_t* drow = dst + (size_t)r * kRowWords + w;
#pragma unroll
            for (int k2 = 0; k2 < 7; ++k2) st4(drow + k2 * pws, o[k2]);
        }
    }
}

template <bool SOLID, bool FORCE>
__global__ void __launch_bounds__(kBlockThreads, 1) fhp_block_kernel(const StepArgs a, const BlockArgs b) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const size_t pws = (size_t)kRin * kRowWords;
    uint32_t* A = reinterpret_cast<uint32_t*>(smem_raw + kBarBytes);  // 7 state planes
    uint32_t* B = A + 7 * pws;                                          // 7 state planes
    uint32_t* S[2] = {B + 7 * pws, B + 8 * pws};                        // solid plane, per tile parity
    int tile = blockIdx.x;
    int sbuf = 0;
    if (tile < b.ntiles) stage_tile<SOLID>(a, b, tile, A, S[0]);
    for (; tile < b.ntiles; tile += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        // Steps 1 .. k-1 alternate A -> B -> A ...; k is even, so step k-1
        // writes B and step k reads B (and S[sbuf]) while A and S[sbuf ^ 1]
        // take the next tile.
        for (int j = 1; j < b.k; ++j) {
            const uint32_t* src = (j & 1) ? A : B;
            uint32_t* dst = (j & 1) ? B : A;
            block_step<SOLID, FORCE>(a, b, tile, j, src, S[sbuf], dst, false, nullptr);
            __syncthreads();
        }
        const int next = tile + gridDim.x;
        if (next < b.ntiles) stage_tile<SOLID>(a, b, next, A, S[sbuf ^ 1]);
        block_step<SOLID, FORCE>(a, b, tile, b.k, B, S[sbuf], nullptr, true, a.dst);
        sbuf ^= 1;
    }
    cp_async_wait_all();
}

std::mutex g_block_mutex;
int g_block_sms[64] = {};
bool g_block_configured[64][2][2] = {};

template <bool SOLID, bool FORCE>
cudaError_t launch_block_variant(const StepArgs& a, const BlockArgs& b, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const size_t smem = kBarBytes + (size_t)16 * kRin * kRowWords * 4;
    int sms;
    {
        std::lock_guard<std::mutex> lock(g_block_mutex);
        if (!g_block_sms[dev]) {
            e = cudaDeviceGetAttribute(&g_block_sms[dev], cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
        }
        if (!g_block_configured[dev][SOLID][FORCE]) {
            e = cudaFuncSetAttribute(fhp_block_kernel<SOLID, FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return e;
            g_block_configured[dev][SOLID][FORCE] = true;
        }
        sms = g_block_sms[dev];
    }
    const int grid = min(b.ntiles, sms);
    fhp_block_kernel<SOLID, FORCE><<<grid, kBlockThreads, smem, s>>>(a, b);
    return cudaGetLastError();
}

}  // namespace

bool block_supported(const Geometry& g, int k) {
    return (k == 2 || k == 4 || k == 8) && g.Wq % 4 == 0 && g.nq >= 4 && g.H >= 2 * k + 2 && 2 * k < kRin &&
           g.rules != 3;   // FHP-III: not in the blocked kernel
}

cudaError_t launch_block(const Geometry& g, const uint32_t* src, uint32_t* dst, const uint32_t* solid,
                         bool has_solid, bool force, const ForcingTable& ft, Key2 key, uint64_t t0, int k,
                         cudaStream_t stream, unsigned int* err) {
    if (!block_supported(g, k)) return cudaErrorInvalidValue;
    StepArgs a;
    a.src = src;
    a.dst = dst;
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
    BlockArgs b;
    b.k = k;
    b.hq = (k + 3) / 4;
    b.qo = kQI - 2 * b.hq;
    b.R_out = kRin - 2 * k;
    b.row_tiles = (g.H + b.R_out - 1) / b.R_out;
    b.col_tiles = (g.nq + b.qo - 1) / b.qo;
    b.ntiles = b.row_tiles * b.col_tiles;
    b.t0 = t0;
    if (has_solid) return force ? launch_block_variant<true, true>(a, b, stream)
                                : launch_block_variant<true, false>(a, b, stream);
    return force ? launch_block_variant<false, true>(a, b, stream) : launch_block_variant<false, false>(a, b, stream);
}

}  // namespace fhp
