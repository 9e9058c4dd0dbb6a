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
// A second kernel (fhp_resident_ghost.cu) keeps two ghost rows per side and
// exchanges every second step; it halves the hand-offs between SMs, which
// dominate a step of a strip of a few rows, for 1/n more arithmetic (n rows
// per strip).  This file also holds the host side of both.
#include <cuda_runtime.h>

#include <mutex>

#include "fhp_resident.cuh"

namespace fhp {
namespace {

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

std::mutex g_res_mutex;
int g_res_sms[64] = {};
bool g_res_configured[64][2][2][2] = {};

template <bool SOLID, bool FORCE, bool RAGGED>
cudaError_t launch_resident_variant(const StepArgs& a, const ResArgs& ra, int grid, size_t smem, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    return launch_resident_coop((const void*)fhp_resident_kernel<SOLID, FORCE, RAGGED>,
                                &g_res_configured[dev][SOLID][FORCE][RAGGED], a, ra, grid, smem, s);
}

cudaError_t launch_resident_one(const StepArgs& a, const ResArgs& ra, int grid, size_t smem, bool has_solid,
                                bool force, bool ragged, cudaStream_t s) {
    if (has_solid) {
        if (force) return ragged ? launch_resident_variant<true, true, true>(a, ra, grid, smem, s)
                                 : launch_resident_variant<true, true, false>(a, ra, grid, smem, s);
        return ragged ? launch_resident_variant<true, false, true>(a, ra, grid, smem, s)
                      : launch_resident_variant<true, false, false>(a, ra, grid, smem, s);
    }
    if (force) return ragged ? launch_resident_variant<false, true, true>(a, ra, grid, smem, s)
                             : launch_resident_variant<false, true, false>(a, ra, grid, smem, s);
    return ragged ? launch_resident_variant<false, false, true>(a, ra, grid, smem, s)
                  : launch_resident_variant<false, false, false>(a, ra, grid, smem, s);
}

}  // namespace

cudaError_t launch_resident_coop(const void* fn, bool* configured, const StepArgs& a, const ResArgs& ra, int grid,
                                 size_t smem, cudaStream_t s) {
    {
        std::lock_guard<std::mutex> lock(g_res_mutex);
        if (!*configured) {
            const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kResSmemLimit);
            if (e != cudaSuccess) return e;
            *configured = true;
        }
    }
    StepArgs a_ = a;
    ResArgs ra_ = ra;
    void* args[] = {(void*)&a_, (void*)&ra_};
    const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kResThreads), args, smem, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

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
    if ((gh != 1 && gh != 2) || g.rules == 3) return false;   // FHP-III: not in the resident kernels
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
    return gh == 1 ? launch_resident_one(a, ra, grid, smem, has_solid, force, ragged, stream)
                   : launch_resident_ghost2(a, ra, grid, smem, has_solid, force, ragged, stream);
}

}  // namespace fhp
