// fhp_resident.cu -- lattices that fit in the SMs' shared memory: the whole
// lattice stays on chip for all steps of a call.
//
// One cooperative launch, one CTA per SM.  CTA b owns rows [y0, y1) of the
// lattice (a contiguous strip) and keeps them, with one extra row below and
// above, in two shared-memory buffers (steps alternate between them).  A step
// pulls the movers from the rows y-1 (north-going planes 3, 4), y (planes 2,
// 5, 6) and y+1 (south-going planes 0, 1) of the staged strip, scatters with
// the same per-quad code as every other step kernel (random words keyed on
// the lattice's row, so results are identical), and writes the new state of
// the owned rows into the other buffer.  Only the strip's edge rows travel
// between steps: after step s each CTA publishes its lowest row (planes 0, 1,
// needed by the CTA below) and highest row (planes 3, 4, needed by the CTA
// above) to a global exchange buffer (double-buffered by step parity) and
// bumps its step counter after a GPU-scope fence; before step s + 1 a CTA
// waits (bounded) for the counters of its two neighbours and copies their
// published rows into its extra rows.  HBM and L2 see the lattice once at the
// start and once at the end of the call, plus 4 rows per CTA and step.
//
// A second kernel keeps two ghost rows per side and exchanges every second
// step (below); it halves the hand-offs between SMs, which dominate a step of
// a strip of a few rows, for 1/n more arithmetic (n rows per strip).
#include <cuda_runtime.h>

#include <mutex>

#include "fhp_device.cuh"
#include "fhp_internal.h"
#include "fhp_quad.cuh"

namespace fhp {
namespace {

constexpr int kResThreads = 384;   // 12 warps: 3 per SM sub-partition at <= 168 registers
constexpr int kResSmemLimit = 220 * 1024;

struct ResArgs {
    uint32_t* buf0;        // state at t0; also the result when nsteps is even
    uint32_t* buf1;        // the result when nsteps is odd
    uint32_t* halo;        // exchange rows: [2 parities][G][2 sides][2 planes][Pq] words
    unsigned int* flags;   // [G] step counters, zero at launch
    int nsteps;
    unsigned long long t0;
    int nmax;              // most rows any CTA owns
};

__device__ __forceinline__ void st_release_gpu(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint4 ldcg4(const uint32_t* p) { return __ldcg(reinterpret_cast<const uint4*>(p)); }

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Spin (no sleep: a hand-off per step is on the critical path) until both
// neighbours' counters reach `target`; acquire loads order the reads of their
// rows after it.  Gives up (false) after kWaitLimitNs.
__device__ __noinline__ bool wait_neighbours(const unsigned int* flags, int p, int q, unsigned int target) {
    unsigned long long start = 0;
    for (unsigned int spin = 0;; ++spin) {
        if (ld_acquire_gpu(flags + p) >= target && ld_acquire_gpu(flags + q) >= target) return true;
        if ((spin & 255u) == 255u) {
            const unsigned long long now = global_ns();
            if (start == 0) start = now;
            else if (now - start > kWaitLimitNs) return false;
        }
    }
}

// One quad (quad q of strip row rr, lattice row y0 + rr) of a step: pulls the
// movers from the staged rows of `src`, scatters, and writes the seven planes
// of the new state into `dst` (padding words of a ragged row stay zero).
// (Local row lr of the staged buffers, lattice row y, `Srow` its solid row.)
template <bool SOLID, bool FORCE, bool RAGGED>
__device__ __forceinline__ void resident_quad_at(const StepArgs& a, const StepVar& v, const uint32_t* src,
                                                 uint32_t* dst, const uint32_t* Srow, size_t pstride, int lr, int y,
                                                 int q, uint4 (&o)[7]) {
    const int Pq = a.Pq;
    const int w = 4 * q;
    const int m = RAGGED ? (q == a.nq - 1 ? a.Wq - w : 4) : 4;
    const int wl = q == 0 ? a.Wq - 1 : w - 1;
    const int wr = q == a.nq - 1 ? 0 : w + 4;
    const uint32_t* rm = src + (size_t)(lr - 1) * Pq;   // row y - 1
    const uint32_t* r0 = src + (size_t)lr * Pq;         // row y
    const uint32_t* rp = src + (size_t)(lr + 1) * Pq;   // row y + 1
    const uint4 i3 = ld4(rm + 3 * pstride + w), i4 = ld4(rm + 4 * pstride + w);
    const uint4 i2 = ld4(r0 + 2 * pstride + w), i5 = ld4(r0 + 5 * pstride + w);
    const uint4 i6 = ld4(r0 + 6 * pstride + w);
    const uint4 i0 = ld4(rp + 0 * pstride + w), i1 = ld4(rp + 1 * pstride + w);
    uint4 sd = make_uint4(0u, 0u, 0u, 0u);
    if (SOLID) sd = ld4(Srow + w);
    uint4 n0, n1, n2, n3, n4, n5;
    if ((y & 1) == 0) {
        n2 = pull_left(i2, r0[2 * pstride + wl]);
        n3 = pull_left(i3, rm[3 * pstride + wl]);
        n1 = pull_left(i1, rp[1 * pstride + wl]);
        n5 = pull_right<RAGGED>(i5, r0[5 * pstride + wr], m);
        n4 = i4;
        n0 = i0;
    } else {
        n2 = pull_left(i2, r0[2 * pstride + wl]);
        n5 = pull_right<RAGGED>(i5, r0[5 * pstride + wr], m);
        n4 = pull_right<RAGGED>(i4, rm[4 * pstride + wr], m);
        n0 = pull_right<RAGGED>(i0, rp[0 * pstride + wr], m);
        n3 = i3;
        n1 = i1;
    }
    collide_quad<SOLID, FORCE>(a, v, q, y, n0, n1, n2, n3, n4, n5, i6, sd, o);
    if (RAGGED && m < 4) {
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            if (m < 2) o[k].y = 0u;
            if (m < 3) o[k].z = 0u;
            o[k].w = 0u;
        }
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) st4(dst + k * pstride + (size_t)lr * Pq + w, o[k]);
}

// One step's work items in two classes: the edge items (the rows the
// neighbours need) first; then, when publishing, a GPU-scope fence and the
// release of the step counter by one thread; then the rest.  (Running the
// rest on other warps while the edge warps publish measured no faster.)
template <class EdgeF, class RestF>
__device__ __forceinline__ void edge_then_rest(int ne, int nr, bool publish, unsigned int* counter,
                                               unsigned int value, EdgeF&& edge, RestF&& rest) {
    const int tid = (int)threadIdx.x;
    if (!publish) {
        for (int i = tid; i < ne + nr; i += kResThreads) {
            if (i < ne) edge(i);
            else rest(i - ne);
        }
        return;
    }
    for (int i = tid; i < ne; i += kResThreads) edge(i);
    __syncthreads();
    if (tid == 0) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");   // the edge rows, then the counter
        st_release_gpu(counter, value);
    }
    for (int i = tid; i < nr; i += kResThreads) rest(i);
}

template <bool SOLID, bool FORCE, bool RAGGED>
__global__ void __launch_bounds__(kResThreads, 1) fhp_resident_kernel(const StepArgs a, const ResArgs ra) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_ok;
    const int G = (int)gridDim.x, b = (int)blockIdx.x;
    const int y0 = (int)(((long long)b * a.H) / G), y1 = (int)(((long long)(b + 1) * a.H) / G);
    const int n = y1 - y0;
    const int Pq = a.Pq, q4 = Pq / 4;
    const int rows = ra.nmax + 2;
    const size_t pstride = (size_t)rows * Pq;          // words per staged plane
    uint32_t* X[2];
    X[0] = reinterpret_cast<uint32_t*>(smem_raw);
    X[1] = X[0] + 7 * pstride;
    uint32_t* S = X[1] + 7 * pstride;                  // solid rows of the strip (SOLID only)
    const int below = b == 0 ? G - 1 : b - 1, above = b == G - 1 ? 0 : b + 1;
    const int tid = (int)threadIdx.x;

    // Stage the owned rows, the two extra rows for step 0 and the solid rows.
    for (int i = tid; i < 7 * n * q4; i += kResThreads) {
        const int p = i / (n * q4), rem = i - p * n * q4, lr = rem / q4 + 1, w = 4 * (rem % q4);
        st4(X[0] + p * pstride + (size_t)lr * Pq + w,
            ld4(ra.buf0 + (size_t)p * a.plane_words + (size_t)(y0 + lr - 1) * Pq + w));
    }
    {
        const int yb = y0 == 0 ? a.H - 1 : y0 - 1, ya = y1 == a.H ? 0 : y1;
        for (int i = tid; i < 4 * q4; i += kResThreads) {
            const int k = i / q4, w = 4 * (i % q4);
            const int p = k < 2 ? 3 + k : k - 2;         // planes 3, 4 from below; 0, 1 from above
            const int y = k < 2 ? yb : ya, lr = k < 2 ? 0 : n + 1;
            st4(X[0] + p * pstride + (size_t)lr * Pq + w, ld4(ra.buf0 + (size_t)p * a.plane_words + (size_t)y * Pq + w));
        }
    }
    if (SOLID)
        for (int i = tid; i < n * q4; i += kResThreads) {
            const int rr = i / q4, w = 4 * (i % q4);
            st4(S + (size_t)rr * Pq + w, ld4(a.solid + (size_t)(y0 + rr) * Pq + w));
        }
    __syncthreads();

    // Each step computes the strip's edge rows first and publishes them, so
    // that the neighbours can go on while the interior rows are computed.
    const int n_edge = n == 1 ? 1 : 2;                     // strip rows 0 and n - 1
    const int n_int = n - n_edge;                          // strip rows 1 .. n - 2
    bool ok = true;
    for (int s = 0; s < ra.nsteps; ++s) {
        const int cur = s & 1, nxt = cur ^ 1;
        if (s > 0) {
            // The neighbours' edge rows of the state after step s - 1.
            if (tid == 0) s_ok = wait_neighbours(ra.flags, below, above, (unsigned int)s) ? 1 : 0;
            __syncthreads();
            if (!s_ok) {
                ok = false;
                break;
            }
            const uint32_t* hb = ra.halo + (((size_t)(s & 1) * G + below) * 2 + 1) * 2 * Pq;  // below's top row
            const uint32_t* ha = ra.halo + (((size_t)(s & 1) * G + above) * 2 + 0) * 2 * Pq;  // above's bottom row
            for (int i = tid; i < 4 * q4; i += kResThreads) {
                const int k = i / q4, w = 4 * (i % q4);
                if (k < 2) st4(X[cur] + (3 + k) * pstride + w, ldcg4(hb + (size_t)k * Pq + w));
                else st4(X[cur] + (k - 2) * pstride + (size_t)(n + 1) * Pq + w, ldcg4(ha + (size_t)(k - 2) * Pq + w));
            }
            __syncthreads();
        }
        const unsigned long long t = ra.t0 + (unsigned long long)s;
        const StepVar v{nullptr, (uint32_t)t, (uint32_t)(t >> 32)};
        const bool publish = s + 1 < ra.nsteps;
        uint32_t* hb = ra.halo + (((size_t)((s + 1) & 1) * G + b) * 2 + 0) * 2 * Pq;   // bottom row: planes 0, 1
        uint32_t* ht = ra.halo + (((size_t)((s + 1) & 1) * G + b) * 2 + 1) * 2 * Pq;   // top row: planes 3, 4
        edge_then_rest(
            n_edge * a.nq, n_int * a.nq, publish, ra.flags + b, (unsigned int)(s + 1),
            [&](int it) {
                // Edge rows, written to shared memory and, for the neighbours, to
                // the exchange buffer.
                const int rr = it < a.nq ? 0 : n - 1, q = it < a.nq ? it : it - a.nq;
                uint4 o[7];
                resident_quad_at<SOLID, FORCE, RAGGED>(a, v, X[cur], X[nxt], S + (size_t)rr * Pq, pstride, rr + 1,
                                                       y0 + rr, q, o);
                if (publish) {
                    if (rr == 0) {
                        st4(hb + 4 * q, o[0]);
                        st4(hb + (size_t)Pq + 4 * q, o[1]);
                    }
                    if (rr == n - 1) {
                        st4(ht + 4 * q, o[3]);
                        st4(ht + (size_t)Pq + 4 * q, o[4]);
                    }
                }
            },
            [&](int it) {
                // Interior rows (their parity alternates with the strip row).
                const int rr = 1 + it / a.nq, q = it % a.nq;
                uint4 o[7];
                resident_quad_at<SOLID, FORCE, RAGGED>(a, v, X[cur], X[nxt], S + (size_t)rr * Pq, pstride, rr + 1,
                                                       y0 + rr, q, o);
            });
        __syncthreads();
    }
    if (!ok) {
        if (tid == 0 && a.err) atomicOr(a.err, 1u);
        return;
    }
    // The owned rows of the final state.
    const uint32_t* fin = X[ra.nsteps & 1];
    uint32_t* out = (ra.nsteps & 1) ? ra.buf1 : ra.buf0;
    for (int i = tid; i < 7 * n * q4; i += kResThreads) {
        const int p = i / (n * q4), rem = i - p * n * q4, lr = rem / q4 + 1, w = 4 * (rem % q4);
        st4(out + (size_t)p * a.plane_words + (size_t)(y0 + lr - 1) * Pq + w, ld4(fin + p * pstride + (size_t)lr * Pq + w));
    }
}

// Ghost-row variant: each strip also keeps the GH rows beyond each edge and
// computes them itself, so that the strips exchange rows once every GH steps
// instead of every step.  In step j of a round of GH steps the rows that can
// still be computed exactly lose one at each end; after the round exactly the
// owned rows are exact, and fresh ghost rows come from the neighbours: the
// GH - 1 inner ghost rows with all seven planes, the outermost only with the
// two planes that stream inwards (3, 4 below the strip, 0, 1 above it).
// Needs strips of at least 2 GH rows.
//
// One side's exchange slots (Pq words each), 7 (GH - 1) + 2 of them:
//   bottom edge (for the strip below): rows 0 .. GH-2 planes 0..6, then row
//     GH-1 planes 0, 1;
//   top edge (for the strip above): row 0 planes 3, 4, then rows 1 .. GH-1
//     planes 0..6;
// rows counted upwards from the edge row block's lowest row.
template <int GH>
__host__ __device__ constexpr int ghost_slots() { return 7 * (GH - 1) + 2; }

template <bool SOLID, bool FORCE, bool RAGGED, int GH>
__global__ void __launch_bounds__(kResThreads, 1) fhp_resident_ghost_kernel(const StepArgs a, const ResArgs ra) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_ok;
    const int G = (int)gridDim.x, b = (int)blockIdx.x;
    const int y0 = (int)(((long long)b * a.H) / G), y1 = (int)(((long long)(b + 1) * a.H) / G);
    const int n = y1 - y0;
    const int L = n + 2 * GH;                          // staged rows: GH ghost rows, n owned, GH ghost rows
    const int Pq = a.Pq, q4 = Pq / 4, nq = a.nq;
    const size_t pstride = (size_t)(ra.nmax + 2 * GH) * Pq;
    uint32_t* X[2];
    X[0] = reinterpret_cast<uint32_t*>(smem_raw);
    X[1] = X[0] + 7 * pstride;
    uint32_t* S = X[1] + 7 * pstride;                  // solid rows of all L staged rows (SOLID only)
    const int below = b == 0 ? G - 1 : b - 1, above = b == G - 1 ? 0 : b + 1;
    const int tid = (int)threadIdx.x;
    const size_t side_words = (size_t)ghost_slots<GH>() * Pq;   // one side's exchange slots
    auto lattice_row = [&](int lr) {                   // lattice row of staged row lr (periodic)
        int y = (y0 - GH + lr) % a.H;
        return y < 0 ? y + a.H : y;
    };

    for (int i = tid; i < 7 * L * q4; i += kResThreads) {
        const int p = i / (L * q4), rem = i - p * L * q4, lr = rem / q4, w = 4 * (rem % q4);
        st4(X[0] + p * pstride + (size_t)lr * Pq + w,
            ld4(ra.buf0 + (size_t)p * a.plane_words + (size_t)lattice_row(lr) * Pq + w));
    }
    if (SOLID)
        for (int i = tid; i < L * q4; i += kResThreads) {
            const int lr = i / q4, w = 4 * (i % q4);
            st4(S + (size_t)lr * Pq + w, ld4(a.solid + (size_t)lattice_row(lr) * Pq + w));
        }
    __syncthreads();

    bool ok = true;
    int cur = 0;
    const int rounds = (ra.nsteps + GH - 1) / GH;
    for (int r = 0; r < rounds; ++r) {
        if (r > 0) {
            if (tid == 0) s_ok = wait_neighbours(ra.flags, below, above, (unsigned int)r) ? 1 : 0;
            __syncthreads();
            if (!s_ok) {
                ok = false;
                break;
            }
            // Ghost rows: the top GH owned rows of the strip below, the bottom
            // GH owned rows of the strip above (both in ascending row order).
            const uint32_t* hb = ra.halo + (((size_t)(r & 1) * G + below) * 2 + 1) * side_words;
            const uint32_t* ha = ra.halo + (((size_t)(r & 1) * G + above) * 2 + 0) * side_words;
            constexpr int ns = ghost_slots<GH>();
            for (int i = tid; i < 2 * ns * q4; i += kResThreads) {
                const int side = i / (ns * q4), rem = i - side * ns * q4, slot = rem / q4, w = 4 * (rem % q4);
                int lr, p;
                if (side == 0) {           // below's top edge
                    lr = slot < 2 ? 0 : 1 + (slot - 2) / 7;
                    p = slot < 2 ? 3 + slot : (slot - 2) % 7;
                } else {                   // above's bottom edge
                    lr = GH + n + (slot < 7 * (GH - 1) ? slot / 7 : GH - 1);
                    p = slot < 7 * (GH - 1) ? slot % 7 : slot - 7 * (GH - 1);
                }
                st4(X[cur] + p * pstride + (size_t)lr * Pq + w,
                    ldcg4((side == 0 ? hb : ha) + (size_t)slot * Pq + w));
            }
            __syncthreads();
        }
        const int steps_here = min(GH, ra.nsteps - r * GH);
        for (int j = 0; j < steps_here; ++j) {
            const unsigned long long t = ra.t0 + (unsigned long long)(r * GH + j);
            const StepVar v{nullptr, (uint32_t)t, (uint32_t)(t >> 32)};
            const uint32_t* src = X[cur];
            uint32_t* dst = X[cur ^ 1];
            auto row_item = [&](int lr, int q) {
                uint4 o[7];
                resident_quad_at<SOLID, FORCE, RAGGED>(a, v, src, dst, S + (size_t)lr * Pq, pstride, lr,
                                                       lattice_row(lr), q, o);
            };
            // A round's last step (j = GH - 1, rows GH .. GH + n - 1, the owned
            // ones) publishes the edge rows GH .. 2GH - 1 and n .. n + GH - 1;
            // earlier steps compute rows j + 1 .. L - 2 - j.
            const bool publish = j == GH - 1 && r + 1 < rounds;
            if (publish) {
                uint32_t* eb = ra.halo + (((size_t)((r + 1) & 1) * G + b) * 2 + 0) * side_words;
                uint32_t* et = ra.halo + (((size_t)((r + 1) & 1) * G + b) * 2 + 1) * side_words;
                edge_then_rest(
                    2 * GH * nq, (n - 2 * GH) * nq, true, ra.flags + b, (unsigned int)(r + 1),
                    [&](int it) {
                        const int side = it / (GH * nq), rem = it - side * GH * nq;
                        const int row = rem / nq, q = rem % nq;
                        const int lr = side == 0 ? GH + row : n + row;
                        uint4 o[7];
                        resident_quad_at<SOLID, FORCE, RAGGED>(a, v, src, dst, S + (size_t)lr * Pq, pstride, lr,
                                                               lattice_row(lr), q, o);
                        if (side == 0) {
                            uint32_t* e = eb + (size_t)row * 7 * Pq + 4 * q;
                            if (row < GH - 1) {
#pragma unroll
                                for (int k = 0; k < 7; ++k) st4(e + (size_t)k * Pq, o[k]);
                            } else {
                                st4(e, o[0]);
                                st4(e + Pq, o[1]);
                            }
                        } else if (row == 0) {
                            st4(et + 4 * q, o[3]);
                            st4(et + Pq + 4 * q, o[4]);
                        } else {
                            uint32_t* e = et + (size_t)(2 + 7 * (row - 1)) * Pq + 4 * q;
#pragma unroll
                            for (int k = 0; k < 7; ++k) st4(e + (size_t)k * Pq, o[k]);
                        }
                    },
                    [&](int it) { row_item(2 * GH + it / nq, it % nq); });
            } else {
                const int lo = j + 1, nitems = (L - 2 - 2 * j) * nq;
                for (int it = tid; it < nitems; it += kResThreads) row_item(lo + it / nq, it % nq);
            }
            __syncthreads();
            cur ^= 1;
        }
    }
    if (!ok) {
        if (tid == 0 && a.err) atomicOr(a.err, 1u);
        return;
    }
    const uint32_t* fin = X[cur];
    uint32_t* out = (ra.nsteps & 1) ? ra.buf1 : ra.buf0;
    for (int i = tid; i < 7 * n * q4; i += kResThreads) {
        const int p = i / (n * q4), rem = i - p * n * q4, lr = GH + rem / q4, w = 4 * (rem % q4);
        st4(out + (size_t)p * a.plane_words + (size_t)(y0 + lr - GH) * Pq + w,
            ld4(fin + p * pstride + (size_t)lr * Pq + w));
    }
}

std::mutex g_res_mutex;
int g_res_sms[64] = {};
bool g_res_configured[64][2][2][2][2] = {};

template <bool SOLID, bool FORCE, bool RAGGED, int GH>
cudaError_t launch_resident_variant(const StepArgs& a, const ResArgs& ra, int grid, size_t smem, cudaStream_t s) {
    const void* fn = GH == 1 ? (const void*)fhp_resident_kernel<SOLID, FORCE, RAGGED>
                             : (const void*)fhp_resident_ghost_kernel<SOLID, FORCE, RAGGED, GH>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(g_res_mutex);
        if (!g_res_configured[dev][SOLID][FORCE][RAGGED][GH - 1]) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kResSmemLimit);
            if (e != cudaSuccess) return e;
            g_res_configured[dev][SOLID][FORCE][RAGGED][GH - 1] = true;
        }
    }
    StepArgs a_ = a;
    ResArgs ra_ = ra;
    void* args[] = {(void*)&a_, (void*)&ra_};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kResThreads), args, smem, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int GH>
cudaError_t launch_resident_gh(const StepArgs& a, const ResArgs& ra, int grid, size_t smem, bool has_solid,
                               bool force, bool ragged, cudaStream_t s) {
    if (has_solid) {
        if (force) return ragged ? launch_resident_variant<true, true, true, GH>(a, ra, grid, smem, s)
                                 : launch_resident_variant<true, true, false, GH>(a, ra, grid, smem, s);
        return ragged ? launch_resident_variant<true, false, true, GH>(a, ra, grid, smem, s)
                      : launch_resident_variant<true, false, false, GH>(a, ra, grid, smem, s);
    }
    if (force) return ragged ? launch_resident_variant<false, true, true, GH>(a, ra, grid, smem, s)
                             : launch_resident_variant<false, true, false, GH>(a, ra, grid, smem, s);
    return ragged ? launch_resident_variant<false, false, true, GH>(a, ra, grid, smem, s)
                  : launch_resident_variant<false, false, false, GH>(a, ra, grid, smem, s);
}

}  // namespace

// CTAs of the resident kernel: one per SM, at most one per row.
int resident_grid(const Geometry& g) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lock(g_res_mutex);
    if (!g_res_sms[dev] && cudaDeviceGetAttribute(&g_res_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return g.H < g_res_sms[dev] ? g.H : g_res_sms[dev];
}

// Shared memory of one CTA: two staged copies of its strip (nmax owned rows,
// 1 extra row per side for gh = 1, gh ghost rows per side otherwise; 7 planes)
// and its solid rows.
size_t resident_smem(const Geometry& g, bool has_solid, int grid, int gh) {
    if (grid <= 0) return 0;
    const int nmax = (g.H + grid - 1) / grid;
    const int staged = nmax + 2 * gh;
    const int solid_rows = has_solid ? (gh == 1 ? nmax : staged) : 0;
    return (size_t)(2 * 7 * staged + solid_rows) * g.Pq * 4;
}

// Exchange buffer words: 2 parities x G CTAs x 2 sides x (2 planes of one row
// for gh = 1, 7 (gh - 1) + 2 row planes otherwise) x Pq words.  The step
// counters take G more words.
size_t resident_halo_words(const Geometry& g, int gh) {
    const size_t per_side = (size_t)(7 * (gh - 1) + 2) * g.Pq;
    return (size_t)2 * resident_grid(g) * 2 * per_side;
}

bool resident_supported(const Geometry& g, bool has_solid, size_t staging_bytes, int gh) {
    if (gh != 1 && gh != 2) return false;
    const int grid = resident_grid(g);
    if (grid <= 0) return false;
    if (gh > 1 && g.H / grid < 2 * gh) return false;   // every strip holds its 2 gh edge rows
    return resident_smem(g, has_solid, grid, gh) <= (size_t)kResSmemLimit &&
           resident_halo_words(g, gh) * sizeof(uint32_t) <= staging_bytes;
}

cudaError_t launch_resident(const Geometry& g, uint32_t* buf0, uint32_t* buf1, const uint32_t* solid, bool has_solid,
                            bool force, const ForcingTable& ft, Key2 key, uint64_t t0, int nsteps, int gh,
                            uint32_t* halo, unsigned int* flags, cudaStream_t stream, unsigned int* err) {
    const int grid = resident_grid(g);
    if (grid <= 0 || nsteps <= 0 || (gh != 1 && gh != 2) || (gh > 1 && g.H / grid < 2 * gh))
        return cudaErrorInvalidValue;
    const size_t smem = resident_smem(g, has_solid, grid, gh);
    if (smem > (size_t)kResSmemLimit) return cudaErrorInvalidValue;
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
    ResArgs ra;
    ra.buf0 = buf0;
    ra.buf1 = buf1;
    ra.halo = halo;
    ra.flags = flags;
    ra.nsteps = nsteps;
    ra.t0 = t0;
    ra.nmax = (g.H + grid - 1) / grid;
    cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)grid * sizeof(unsigned int), stream);
    if (e != cudaSuccess) return e;
    const bool ragged = g.Wq % 4 != 0;
    return gh == 1 ? launch_resident_gh<1>(a, ra, grid, smem, has_solid, force, ragged, stream)
                   : launch_resident_gh<2>(a, ra, grid, smem, has_solid, force, ragged, stream);
}

}  // namespace fhp
