// fhp_resident.cuh -- pieces shared by the shared-memory resident kernels
// (one-row exchange in fhp_resident.cu, two ghost rows per strip side in
// fhp_resident_ghost.cu): launch constants, kernel arguments, the bounded
// neighbour wait and the per-quad step on staged strip rows.
#pragma once

#include <cuda_runtime.h>

#include "fhp_device.cuh"
#include "fhp_internal.h"
#include "fhp_quad.cuh"

namespace fhp {

constexpr int kResThreads = 384;   // 12 warps: 3 per SM sub-partition at <= 168 registers
                                   // (both kernels use at most 160: no spills)
constexpr int kResSmemLimit = 220 * 1024;

struct ResArgs {
    uint32_t* buf0;        // state at t0; also the result when nsteps is even
    uint32_t* buf1;        // the result when nsteps is odd
    uint32_t* halo;        // exchange rows: [2 parities][G][2 sides][row planes][Pq] words (2 row
                           // planes per side for the one-row exchange, 9 for two ghost rows)
    unsigned int* flags;   // [G] step counters, zero at launch
    int nsteps;
    unsigned long long t0;
    int nmax;              // most rows any CTA owns
};

// Launches the two-ghost-row kernel (fhp_resident_ghost.cu) for the
// lattice's variant (obstacles, forcing, partial last quad).
cudaError_t launch_resident_ghost2(const StepArgs& a, const ResArgs& ra, int grid, size_t smem, bool has_solid,
                                   bool force, bool ragged, cudaStream_t s);

// Sets the dynamic shared-memory limit of `fn` once per device and launches
// it cooperatively with the kernel arguments (a, ra).
cudaError_t launch_resident_coop(const void* fn, bool* configured, const StepArgs& a, const ResArgs& ra, int grid,
                                 size_t smem, cudaStream_t s);

namespace {

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

}  // namespace
}  // namespace fhp
