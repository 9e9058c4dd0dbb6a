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
#include <cuda_runtime.h>

#include <mutex>

#include "fhp_device.cuh"
#include "fhp_internal.h"
#include "fhp_quad.cuh"

namespace fhp {
namespace {

constexpr int kResThreads = 256;
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

// One quad (quad q of strip row rr, lattice row y0 + rr) of a step: pulls the
// movers from the staged rows of `src`, scatters, and writes the seven planes
// of the new state into `dst` (padding words of a ragged row stay zero).
template <bool SOLID, bool FORCE, bool RAGGED>
__device__ __forceinline__ void resident_quad(const StepArgs& a, const StepVar& v, const uint32_t* src, uint32_t* dst,
                                              const uint32_t* S, size_t pstride, int y0, int rr, int q,
                                              uint4 (&o)[7]) {
    const int Pq = a.Pq;
    const int lr = rr + 1, y = y0 + rr, w = 4 * q;
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
    if (SOLID) sd = ld4(S + (size_t)rr * Pq + w);
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
            if (tid == 0) s_ok = wait_tiles(ra.flags, below, above, 0, false, (unsigned int)s) ? 1 : 0;
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
        // Edge rows, written to shared memory and, for the neighbours, to the
        // exchange buffer.
        for (int it = tid; it < n_edge * a.nq; it += kResThreads) {
            const int rr = it < a.nq ? 0 : n - 1, q = it < a.nq ? it : it - a.nq;
            uint4 o[7];
            resident_quad<SOLID, FORCE, RAGGED>(a, v, X[cur], X[nxt], S, pstride, y0, rr, q, o);
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
        }
        __syncthreads();
        if (publish && tid == 0) {
            asm volatile("fence.acq_rel.gpu;" ::: "memory");   // the edge rows, then the counter
            st_release_gpu(ra.flags + b, (unsigned int)(s + 1));
        }
        // Interior rows (their global parity alternates with the strip row).
        for (int it = tid; it < n_int * a.nq; it += kResThreads) {
            const int rr = 1 + it / a.nq, q = it % a.nq;
            uint4 o[7];
            resident_quad<SOLID, FORCE, RAGGED>(a, v, X[cur], X[nxt], S, pstride, y0, rr, q, o);
        }
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

std::mutex g_res_mutex;
int g_res_sms[64] = {};
bool g_res_configured[64][2][2][2] = {};

template <bool SOLID, bool FORCE, bool RAGGED>
cudaError_t launch_resident_variant(const StepArgs& a, const ResArgs& ra, int grid, size_t smem, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(g_res_mutex);
        if (!g_res_configured[dev][SOLID][FORCE][RAGGED]) {
            e = cudaFuncSetAttribute(fhp_resident_kernel<SOLID, FORCE, RAGGED>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kResSmemLimit);
            if (e != cudaSuccess) return e;
            g_res_configured[dev][SOLID][FORCE][RAGGED] = true;
        }
    }
    StepArgs a_ = a;
    ResArgs ra_ = ra;
    void* args[] = {(void*)&a_, (void*)&ra_};
    e = cudaLaunchCooperativeKernel((const void*)fhp_resident_kernel<SOLID, FORCE, RAGGED>, dim3(grid),
                                    dim3(kResThreads), args, smem, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
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

size_t resident_smem(const Geometry& g, bool has_solid, int grid) {
    if (grid <= 0) return 0;
    const int nmax = (g.H + grid - 1) / grid;
    return (size_t)(2 * 7 * (nmax + 2) + (has_solid ? nmax : 0)) * g.Pq * 4;
}

// Exchange buffer words the resident kernel needs (2 parities x G CTAs x 2
// sides x 2 planes x Pq words); the step counters take G more words.
size_t resident_halo_words(const Geometry& g) { return (size_t)2 * resident_grid(g) * 2 * 2 * g.Pq; }

bool resident_supported(const Geometry& g, bool has_solid, size_t staging_bytes) {
    const int grid = resident_grid(g);
    return grid > 0 && resident_smem(g, has_solid, grid) <= (size_t)kResSmemLimit &&
           resident_halo_words(g) * sizeof(uint32_t) <= staging_bytes;
}

cudaError_t launch_resident(const Geometry& g, uint32_t* buf0, uint32_t* buf1, const uint32_t* solid, bool has_solid,
                            bool force, const ForcingTable& ft, Key2 key, uint64_t t0, int nsteps, uint32_t* halo,
                            unsigned int* flags, cudaStream_t stream, unsigned int* err) {
    const int grid = resident_grid(g);
    const size_t smem = resident_smem(g, has_solid, grid);
    if (grid <= 0 || smem > (size_t)kResSmemLimit || nsteps <= 0) return cudaErrorInvalidValue;
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
    if (has_solid) {
        if (force) return ragged ? launch_resident_variant<true, true, true>(a, ra, grid, smem, stream)
                                 : launch_resident_variant<true, true, false>(a, ra, grid, smem, stream);
        return ragged ? launch_resident_variant<true, false, true>(a, ra, grid, smem, stream)
                      : launch_resident_variant<true, false, false>(a, ra, grid, smem, stream);
    }
    if (force) return ragged ? launch_resident_variant<false, true, true>(a, ra, grid, smem, stream)
                             : launch_resident_variant<false, true, false>(a, ra, grid, smem, stream);
    return ragged ? launch_resident_variant<false, false, true>(a, ra, grid, smem, stream)
                  : launch_resident_variant<false, false, false>(a, ra, grid, smem, stream);
}

}  // namespace fhp
