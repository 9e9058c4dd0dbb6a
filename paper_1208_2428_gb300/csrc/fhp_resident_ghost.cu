// fhp_resident_ghost.cu -- the shared-memory resident kernel with two ghost
// rows per strip side: strips exchange rows every second step (its own
// translation unit so that the library's kernels compile in parallel).
#include <cuda_runtime.h>

#include "fhp_resident.cuh"

namespace fhp {
namespace {

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

bool g_ghost_configured[64][2][2][2] = {};

template <bool SOLID, bool FORCE, bool RAGGED>
cudaError_t launch_ghost_variant(const StepArgs& a, const ResArgs& ra, int grid, size_t smem, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    return launch_resident_coop((const void*)fhp_resident_ghost_kernel<SOLID, FORCE, RAGGED, 2>,
                                &g_ghost_configured[dev][SOLID][FORCE][RAGGED], a, ra, grid, smem, s);
}

}  // namespace

cudaError_t launch_resident_ghost2(const StepArgs& a, const ResArgs& ra, int grid, size_t smem, bool has_solid,
                                   bool force, bool ragged, cudaStream_t s) {
    if (has_solid) {
        if (force) return ragged ? launch_ghost_variant<true, true, true>(a, ra, grid, smem, s)
                                 : launch_ghost_variant<true, true, false>(a, ra, grid, smem, s);
        return ragged ? launch_ghost_variant<true, false, true>(a, ra, grid, smem, s)
                      : launch_ghost_variant<true, false, false>(a, ra, grid, smem, s);
    }
    if (force) return ragged ? launch_ghost_variant<false, true, true>(a, ra, grid, smem, s)
                             : launch_ghost_variant<false, true, false>(a, ra, grid, smem, s);
    return ragged ? launch_ghost_variant<false, false, true>(a, ra, grid, smem, s)
                  : launch_ghost_variant<false, false, false>(a, ra, grid, smem, s);
}

}  // namespace fhp
