// fhp_wave.cu -- temporal blocking by row wavefronts: K FHP steps per pass
// over full-width row bands, with the intermediate time levels kept in
// shared-memory row rings.
//
// The lattice is cut into horizontal bands, one per CTA (persistent CTAs
// loop over the bands).  For a band of rows [y0, y1) the pass computes
// S_{t+K} from S_t:
//   level 0  rows y0-K .. y1+K-1 of S_t, streamed in row order by a producer
//            warp into a ring of D0 shared-memory slots (cp.async.bulk of the
//            seven state planes and the solid plane of one row, completion
//            on one mbarrier per slot);
//   level j  (1 <= j < K) rows y0-(K-j) .. y1+(K-j)-1 of S_{t+j}, each
//            computed from rows y-1, y, y+1 of level j-1 and kept in a ring
//            of D slots;
//   level K  rows y0 .. y1-1 of S_{t+K}, stored to global memory.
// Rows are whole lattice rows, so the periodic wrap in x needs no halo; only
// the 2(K-1) rows of levels below K outside the band are computed twice (by
// this band and its neighbour).
//
// Work is split among warps by (level j, column c of 32 quads, row parity p
// when P = 2): warp (j, c, p) computes quads 32c .. 32c+31 of the rows of
// level j whose index is p mod P, in increasing order.  There is no CTA-wide
// barrier inside a band: every warp publishes the number of rows it has
// finished in a shared-memory counter (release), and a warp waits (acquire,
// bounded) only for what it reads -- rows i .. i+2 of level j-1 in its own
// and the two neighbouring columns -- and, before overwriting a ring slot,
// for the rows of level j+1 that read the slot's old row.  Level 1 waits for
// the producer's copies on the slots' mbarriers instead.  Every dependency
// points to a smaller row index, so the waits always end.
//
// The per-quad code (motion with the odd-row shift, scattering, bounce-back,
// forcing, counter-based random streams keyed on the global quad, row and
// step) is the one of the single-step kernels, so results are bit-identical
// to K single steps.
#include <cstdio>
#include <mutex>

#include "fhp_debug.cuh"
#include "fhp_device.cuh"
#include "fhp_internal.h"
#include "fhp_quad.cuh"

namespace fhp {
namespace {

constexpr int kWaveMaxComputeWarps = 16;
constexpr int kWaveThreads = (kWaveMaxComputeWarps + 1) * 32;  // + producer warp
constexpr int kWaveCounterBytes = 256;                           // row counters [K+1][C][P]
constexpr int kWaveBarrierBytes = 256;                           // one mbarrier per level-0 slot
constexpr int kWaveMaxD0 = kWaveBarrierBytes / 8;
constexpr int kWaveHeaderBytes = kWaveCounterBytes + kWaveBarrierBytes;

struct WaveArgs {
    int C;             // columns of 32 quads per row
    int P;             // warps per (level, column): rows of index p mod P
    int D0;            // level-0 ring slots (8 planes each)
    int D;             // ring slots per intermediate level (7 planes each)
    int nbands;        // bands of rows (band b: rows [b H / nbands, (b+1) H / nbands))
    unsigned long long t0;
};

__device__ __forceinline__ int wrap_row(int y, int H) {
    y %= H;
    return y < 0 ? y + H : y;
}

// Rows 0..m of a level done by the warp of parity p (rows of index p mod P).
__device__ __forceinline__ unsigned int rows_upto(int m, int p, int P) {
    return m < p ? 0u : (unsigned int)((m - p) / P + 1);
}

__device__ __forceinline__ unsigned int ld_relaxed_shared(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.relaxed.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_shared(unsigned int* p, unsigned int v) {
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}

// Wait until, in the columns c-1, c, c+1 (periodic) of one level's counters,
// the rows of index 0..m of every parity are counted.  Lane 0 polls with
// relaxed loads and then takes one CTA-scope fence (acquire); __syncwarp
// orders the other lanes' later reads after it.  Warp-uniform result; false
// after kWaitLimitNs.
__device__ __forceinline__ bool wait_rows(const unsigned int* level, int c, int C, int P, int m, int lane) {
    int ok = 1;
    if (m >= 0 && lane == 0) {
        const int cl = c == 0 ? C - 1 : c - 1, cr = c == C - 1 ? 0 : c + 1;
        unsigned long long start = 0;
        for (;;) {
            bool ready = true;
            for (int p = 0; p < P; ++p) {
                const unsigned int need = rows_upto(m, p, P);
                ready = ready && ld_relaxed_shared(level + c * P + p) >= need &&
                        ld_relaxed_shared(level + cl * P + p) >= need &&
                        ld_relaxed_shared(level + cr * P + p) >= need;
            }
            if (ready) break;
            const unsigned long long now = global_ns();
            if (start == 0) start = now;
            else if (now - start > kWaitLimitNs) {
                ok = 0;
                break;
            }
            __nanosleep(64);   // leave the issue slots to the warps that compute
        }
        __threadfence_block();
    }
    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
    __syncwarp();
    return ok != 0;
}

// The inputs of one quad of a level row: the quad's words of the seven
// planes of rows y-1, y, y+1 of the previous level (planes Pq words apart),
// already shifted by the motion step, and its solid words.
struct QuadIn {
    uint4 n0, n1, n2, n3, n4, n5, i6, sd;
};

// Shared-memory reads only (the solid words of a level-1 row come with the
// staged row; the other levels read theirs from global memory in wave_finish,
// after the quad has released its input rows).
template <bool SOLID, bool RAGGED>
__device__ __forceinline__ QuadIn wave_load(const StepArgs& a, const uint32_t* rm, const uint32_t* r0,
                                            const uint32_t* rp, const uint32_t* sd_smem, int y, int q) {
    const int Pq = a.Pq;
    const int w = 4 * q;
    const int m = RAGGED ? (q == a.nq - 1 ? a.Wq - w : 4) : 4;
    const int wl = q == 0 ? a.Wq - 1 : w - 1;       // word left of the quad (periodic)
    const int wr = q == a.nq - 1 ? 0 : w + 4;       // word right of the quad (periodic)
    const uint4 i3 = ld4(rm + 3 * Pq + w), i4 = ld4(rm + 4 * Pq + w);
    const uint4 i2 = ld4(r0 + 2 * Pq + w), i5 = ld4(r0 + 5 * Pq + w);
    const uint4 i0 = ld4(rp + 0 * Pq + w), i1 = ld4(rp + 1 * Pq + w);
    QuadIn in;
    in.i6 = ld4(r0 + 6 * Pq + w);
    in.sd = make_uint4(0u, 0u, 0u, 0u);
    if (SOLID && sd_smem) in.sd = ld4(sd_smem + w);
    if ((y & 1) == 0) {
        // Even row: E, NE, SE come from x-1; W from x+1; NW, SW from x.
        in.n2 = pull_left(i2, r0[2 * Pq + wl]);
        in.n3 = pull_left(i3, rm[3 * Pq + wl]);
        in.n1 = pull_left(i1, rp[1 * Pq + wl]);
        in.n5 = pull_right<RAGGED>(i5, r0[5 * Pq + wr], m);
        in.n4 = i4;
        in.n0 = i0;
    } else {
        // Odd row: E from x-1; W, NW, SW from x+1; NE, SE from x.
        in.n2 = pull_left(i2, r0[2 * Pq + wl]);
        in.n5 = pull_right<RAGGED>(i5, r0[5 * Pq + wr], m);
        in.n4 = pull_right<RAGGED>(i4, rm[4 * Pq + wr], m);
        in.n0 = pull_right<RAGGED>(i0, rp[0 * Pq + wr], m);
        in.n3 = i3;
        in.n1 = i1;
    }
    return in;
}

// Scattering, bounce-back and forcing of the quad; LAST stores the result to
// global memory, else into `out` (a level slot).
template <bool SOLID, bool FORCE, bool RAGGED>
__device__ __forceinline__ void wave_finish(const StepArgs& a, const StepVar& v, const QuadIn& in,
                                            const uint32_t* sd_global, uint32_t* out, bool last, int y, int q) {
    uint4 sd = in.sd;
    if (SOLID && sd_global) sd = __ldg(reinterpret_cast<const uint4*>(sd_global + 4 * q));
    uint4 o[7];
    collide_quad<SOLID, FORCE>(a, v, q, y, in.n0, in.n1, in.n2, in.n3, in.n4, in.n5, in.i6, sd, o);
    if (last) {
        const int m = RAGGED ? (q == a.nq - 1 ? a.Wq - 4 * q : 4) : 4;
        store_quad<RAGGED>(a, v.dst, q, y, m, o);
    } else {
#pragma unroll
        for (int k = 0; k < 7; ++k) st4(out + k * a.Pq + 4 * q, o[k]);
    }
}

template <int K, bool SOLID, bool FORCE, bool RAGGED>
__global__ void __launch_bounds__(kWaveThreads, 1) fhp_wave_kernel(const StepArgs a, const WaveArgs wa) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // Row counters: rd[j] counts rows of level j whose inputs have been read,
    // wr[j] rows of level j written to its ring (per column and parity).
    unsigned int* rd = reinterpret_cast<unsigned int*>(smem_raw);                     // [K+1][C][P]
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + kWaveCounterBytes);         // [D0]
    uint32_t* ring0 = reinterpret_cast<uint32_t*>(smem_raw + kWaveHeaderBytes);        // D0 x 8 planes
    const int Pq = a.Pq;
    const size_t slot0_words = (size_t)8 * Pq;
    const size_t slot_words = (size_t)7 * Pq;
    uint32_t* ring = ring0 + (size_t)wa.D0 * slot0_words;                               // (K-1) x D x 7 planes
    const int C = wa.C, P = wa.P;
    const int ncomp = K * C * P;
    unsigned int* wr = rd + (K + 1) * C * P;                                            // [K+1][C][P]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ int abort_flag;
    {
        unsigned int dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        const size_t need = (size_t)kWaveHeaderBytes +
                            ((size_t)wa.D0 * slot0_words + (size_t)(K - 1) * wa.D * slot_words) * 4;
        if (!dbg_ok(need <= dyn && wa.D0 <= kWaveMaxD0 && (K + 1) * C * P * 8 <= kWaveCounterBytes, a.err,
                    kSiteWaveSmem))
            return;
    }

    if (threadIdx.x == 0) abort_flag = 0;
    for (int band = blockIdx.x; band < wa.nbands; band += gridDim.x) {
        const int y0 = (int)(((long long)band * a.H) / wa.nbands);
        const int y1 = (int)(((long long)(band + 1) * a.H) / wa.nbands);
        const int B = y1 - y0;
        for (int i = threadIdx.x; i < 2 * (K + 1) * C * P; i += blockDim.x) rd[i] = 0;
        if (threadIdx.x == 0) {
            for (int s = 0; s < wa.D0; ++s) mbar_init(&full[s], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        const bool aborted = abort_flag != 0;

        if (warp == ncomp) {
            // Producer: level-0 rows i = 0 .. B+2K-1 (lattice rows y0-K+i).
            if (lane == 0 && !aborted) {
                const int n0 = B + 2 * K;
                const uint32_t row_bytes = (uint32_t)Pq * 4u;
                constexpr int NP = SOLID ? 8 : 7;
                int i = 0;
                bool ok = true;
                for (; i < n0; ++i) {
                    const int s = i % wa.D0;
                    if (i >= wa.D0) {
                        // The slot's old row i - D0 is read by level-1 rows i-D0-2 .. i-D0.
                        const unsigned int* lv1 = rd + 1 * C * P;
                        const int m = i - wa.D0;
                        unsigned long long start = 0;
                        for (;;) {
                            bool ready = true;
                            for (int c = 0; c < C && ready; ++c)
                                for (int p = 0; p < P && ready; ++p)
                                    ready = ld_relaxed_shared(lv1 + c * P + p) >= rows_upto(m, p, P);
                            if (ready) break;
                            const unsigned long long now = global_ns();
                            if (start == 0) start = now;
                            else if (now - start > kWaitLimitNs) {
                                ok = false;
                                break;
                            }
                            __nanosleep(64);
                        }
                        if (!ok) break;
                        __threadfence_block();   // acquire: the readers are done with the slot
                    }
                    const int y = wrap_row(y0 - K + i, a.H);
                    uint32_t* dst = ring0 + (size_t)s * slot0_words;
                    // Generic-proxy reads of the slot's old row are ordered
                    // before the bulk copy's writes.
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive_expect_tx(&full[s], (uint32_t)NP * row_bytes);
#pragma unroll
                    for (int pl = 0; pl < NP; ++pl) {
                        const uint32_t* plane = pl < 7 ? a.src + (size_t)pl * a.plane_words : a.solid;
                        bulk_copy_g2s(dst + (size_t)pl * Pq, plane + (size_t)y * Pq, row_bytes, &full[s]);
                    }
                }
                if (!ok) {
                    if (a.err) atomicOr(a.err, 1u);
                    atomicOr(&abort_flag, 1);
                }
                // Never leave the band while copies into shared memory may be in flight.
                for (int k = (i > wa.D0 ? i - wa.D0 : 0); k < i; ++k)
                    (void)mbar_wait_bounded(&full[k % wa.D0], (uint32_t)((k / wa.D0) & 1));
            }
        } else if (warp < ncomp && !aborted) {
            const int j = 1 + warp / (C * P);
            const int rem = warp - (j - 1) * C * P;
            const int c = rem / P, p = rem - c * P;
            const int q = c * 32 + lane;
            const bool active = q < a.nq && dbg_ok(4 * q + 3 < Pq && a.Wq <= Pq, a.err, kSiteWaveQuad);
            const int nj = B + 2 * (K - j);
            const int start = y0 - (K - j);
            const unsigned long long t = wa.t0 + (unsigned long long)(j - 1);
            const StepVar v{a.dst, (uint32_t)t, (uint32_t)(t >> 32)};
            uint32_t* my_ring = j < K ? ring + ((size_t)(j - 1) * wa.D) * slot_words : nullptr;
            const uint32_t* prev_ring = j > 1 ? ring + ((size_t)(j - 2) * wa.D) * slot_words : nullptr;
            bool ok = true;
            for (int i = p; i < nj; i += P) {
                // Inputs: rows i, i+1, i+2 of level j-1 (lattice rows y-1, y, y+1).
                const uint32_t *rm, *r0, *rp, *sd_smem, *sd_global;
                const int y = wrap_row(start + i, a.H);
                if (j == 1) {
                    // Every row's slot phase is waited for in row order (the
                    // first iteration also covers the rows below it), so a
                    // slot's previous use has completed before its next one
                    // is tested and the phase parity cannot alias.
                    for (int r = (i == p ? 0 : i); r <= i + 2 && ok; ++r) {
                        const uint32_t par = (uint32_t)((r / wa.D0) & 1);
                        ok = mbar_wait_bounded(&full[r % wa.D0], par);
                    }
                    ok = __all_sync(0xFFFFFFFFu, ok);
                    rm = ring0 + (size_t)(i % wa.D0) * slot0_words;
                    r0 = ring0 + (size_t)((i + 1) % wa.D0) * slot0_words;
                    rp = ring0 + (size_t)((i + 2) % wa.D0) * slot0_words;
                    sd_smem = r0 + 7 * (size_t)Pq;
                    sd_global = nullptr;
                } else {
                    ok = wait_rows(wr + (j - 1) * C * P, c, C, P, i + 2, lane);
                    rm = prev_ring + (size_t)(i % wa.D) * slot_words;
                    r0 = prev_ring + (size_t)((i + 1) % wa.D) * slot_words;
                    rp = prev_ring + (size_t)((i + 2) % wa.D) * slot_words;
                    sd_smem = nullptr;
                    sd_global = a.solid + (size_t)y * Pq;
                }
                // Output slot: its old row i - D is read by level j+1 rows i-D-2 .. i-D.
                if (ok && j < K) ok = wait_rows(rd + (j + 1) * C * P, c, C, P, i - wa.D, lane);
                if (!ok) break;
                const unsigned int count = (unsigned int)(i / P + 1);
                QuadIn in;
                if (active) in = wave_load<SOLID, RAGGED>(a, rm, r0, rp, sd_smem, y, q);
                // The inputs are in registers: the level below may reuse their slots.
                __syncwarp();
                if (lane == 0) st_release_shared(rd + j * C * P + c * P + p, count);
                if (active) {
                    // One copy of the collision code serves every level (the
                    // store target is a warp-uniform choice).
                    wave_finish<SOLID, FORCE, RAGGED>(a, v, in, sd_global,
                                                      j < K ? my_ring + (size_t)(i % wa.D) * slot_words : nullptr,
                                                      j == K, y, q);
                }
                if (j < K) {
                    __syncwarp();
                    if (lane == 0) st_release_shared(wr + j * C * P + c * P + p, count);
                }
            }
            if (!ok && lane == 0) {
                if (a.err) atomicOr(a.err, 1u);
                atomicOr(&abort_flag, 1);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int s = 0; s < wa.D0; ++s)
                asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&full[s])) : "memory");
        }
        __syncthreads();
    }
}

struct WaveConfig {
    int C, P, D0, D;
    size_t smem;
};

size_t wave_smem(const Geometry& g, int K, int D0, int D) {
    return (size_t)kWaveHeaderBytes + (size_t)D0 * 8 * g.Pq * 4 + (size_t)(K - 1) * D * 7 * g.Pq * 4;
}

constexpr size_t kWaveMaxSmem = 224 * 1024;   // dynamic; the static abort flag needs a few bytes more

// Columns, warps per column and ring depths for a lattice, or false if the
// rows do not fit shared memory or need more warps than a CTA has.
bool wave_config(const Geometry& g, int K, WaveConfig* out) {
    if (K < 2 || K > 4 || g.rules == 3) return false;
    const int C = (g.nq + 31) / 32;
    for (int P = 2; P >= 1; --P) {
        if (K * C * P > kWaveMaxComputeWarps) continue;
        // Preferred depths leave slack between the levels; the minimum ones
        // (D0 = P + 3, D = 3) still let every wait end.
        const int pref[2][2] = {{P + 5, 2 * P + 2}, {P + 3, 3}};
        for (const auto& d : pref) {
            const int D0 = d[0], D = d[1];
            if (D0 > kWaveMaxD0) continue;
            const size_t smem = wave_smem(g, K, D0, D);
            if (smem <= kWaveMaxSmem) {
                *out = WaveConfig{C, P, D0, D, smem};
                return true;
            }
        }
    }
    return false;
}

std::mutex g_wave_mutex;
int g_wave_sms[64] = {};
bool g_wave_configured[64][3][2][2][2] = {};

template <int K, bool SOLID, bool FORCE, bool RAGGED>
cudaError_t launch_wave_variant(const StepArgs& a, const Geometry& g, const WaveConfig& cfg, uint64_t t0,
                                cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    auto kernel = fhp_wave_kernel<K, SOLID, FORCE, RAGGED>;
    int sms;
    {
        std::lock_guard<std::mutex> lock(g_wave_mutex);
        if (!g_wave_sms[dev]) {
            e = cudaDeviceGetAttribute(&g_wave_sms[dev], cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
        }
        bool& configured = g_wave_configured[dev][K - 2][SOLID][FORCE][RAGGED];
        if (!configured) {
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWaveMaxSmem);
            if (e != cudaSuccess) return e;
            configured = true;
        }
        sms = g_wave_sms[dev];
    }
    const int threads = (K * cfg.C * cfg.P + 1) * 32;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, cfg.smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // One band per CTA, bands of at least 8 rows.
    const int max_bands = g.H / 8 > 0 ? g.H / 8 : 1;
    const int grid = std::min(per_sm * sms, max_bands);
    WaveArgs wa;
    wa.C = cfg.C;
    wa.P = cfg.P;
    wa.D0 = cfg.D0;
    wa.D = cfg.D;
    wa.nbands = grid;
    wa.t0 = t0;
    kernel<<<grid, threads, cfg.smem, s>>>(a, wa);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_wave_k(const StepArgs& a, const Geometry& g, const WaveConfig& cfg, bool has_solid, bool force,
                          uint64_t t0, cudaStream_t s) {
    const bool ragged = (g.Wq % 4) != 0;
    if (has_solid) {
        if (force) return ragged ? launch_wave_variant<K, true, true, true>(a, g, cfg, t0, s)
                                 : launch_wave_variant<K, true, true, false>(a, g, cfg, t0, s);
        return ragged ? launch_wave_variant<K, true, false, true>(a, g, cfg, t0, s)
                      : launch_wave_variant<K, true, false, false>(a, g, cfg, t0, s);
    }
    if (force) return ragged ? launch_wave_variant<K, false, true, true>(a, g, cfg, t0, s)
                             : launch_wave_variant<K, false, true, false>(a, g, cfg, t0, s);
    return ragged ? launch_wave_variant<K, false, false, true>(a, g, cfg, t0, s)
                  : launch_wave_variant<K, false, false, false>(a, g, cfg, t0, s);
}

}  // namespace

bool wave_supported(const Geometry& g, int k) {
    WaveConfig cfg;
    return wave_config(g, k, &cfg);
}

cudaError_t launch_wave(const Geometry& g, const uint32_t* src, uint32_t* dst, const uint32_t* solid,
                        bool has_solid, bool force, const ForcingTable& ft, Key2 key, uint64_t t0, int k,
                        cudaStream_t stream, unsigned int* err) {
    WaveConfig cfg;
    if (!wave_config(g, k, &cfg)) return cudaErrorInvalidValue;
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
    switch (k) {
        case 2: return launch_wave_k<2>(a, g, cfg, has_solid, force, t0, stream);
        case 3: return launch_wave_k<3>(a, g, cfg, has_solid, force, t0, stream);
        case 4: return launch_wave_k<4>(a, g, cfg, has_solid, force, t0, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fhp
