// fhp_step.cu -- one fused FHP time step on bit-planes (k = 1).
//
// One thread owns one quad (4 consecutive words = 128 nodes) of one row y and
// writes S_{t+1} for it:
//   motion (arXiv:1208.2428 Section 2, Fig. 3): the particle moving along c_i
//     that arrives at (x, y) left (x, y) - c_i; rows y-1, y, y+1 each feed the
//     directions that point away from them, and the half-cell shift of odd
//     rows decides, per direction, whether the source sits one node to the
//     left, at the same x, or one node to the right;
//   the one-node shifts are funnel shifts across the words of the quad; the
//     word beyond the quad comes from the neighbouring lane (__shfl_sync) or,
//     at a warp or row edge, from a global load (periodic wrap in x);
//   scattering with bounce-back and forcing (device functions of
//     fhp_device.cuh); one Philox block gives the chirality bits of the
//     quad's 128 nodes, a second one its forcing draws;
//   128-bit loads and stores of the seven planes (two ping-pong buffers).
// The row parity is uniform within a warp: wide rows (>= 32 quads) give each
// warp 32 quads of one row; narrow rows pack whole rows of one parity into a
// warp.
#include "fhp_device.cuh"
#include "fhp_internal.h"

namespace fhp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kBlock = 256;

struct Lane {
    int y, q;
    bool active;
    int src_left, src_right;   // lanes holding the quads to the left / right
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

__device__ __forceinline__ uint4 ld4(const uint32_t* p) {
    return *reinterpret_cast<const uint4*>(p);
}

__device__ __forceinline__ void st4(uint32_t* p, uint4 v) {
    *reinterpret_cast<uint4*>(p) = v;
}

// New bit x takes old bit x-1.  `m` = number of valid words in this quad.
template <bool RAGGED>
__device__ __forceinline__ uint4 from_left(uint4 v, uint32_t fallback, const Lane& L, int m) {
    uint32_t offer = v.w;
    if (RAGGED) offer = m == 4 ? v.w : m == 3 ? v.z : m == 2 ? v.y : v.x;
    uint32_t left = __shfl_sync(kFull, offer, L.src_left);
    if (L.glob_left) left = fallback;
    return make_uint4(__funnelshift_l(left, v.x, 1), __funnelshift_l(v.x, v.y, 1),
                      __funnelshift_l(v.y, v.z, 1), __funnelshift_l(v.z, v.w, 1));
}

// New bit x takes old bit x+1.
template <bool RAGGED>
__device__ __forceinline__ uint4 from_right(uint4 v, uint32_t fallback, const Lane& L, int m) {
    uint32_t right = __shfl_sync(kFull, v.x, L.src_right);
    if (L.glob_right) right = fallback;
    uint32_t n0 = v.y, n1 = v.z, n2 = v.w;
    if (RAGGED) {
        if (m == 1) n0 = right;
        if (m == 2) n1 = right;
        if (m == 3) n2 = right;
    }
    return make_uint4(__funnelshift_r(v.x, n0, 1), __funnelshift_r(v.y, n1, 1),
                      __funnelshift_r(v.z, n2, 1), __funnelshift_r(v.w, right, 1));
}

template <bool SOLID, bool FORCE, bool RAGGED, bool ODD>
__device__ __forceinline__ void step_quad(const StepArgs& a, const Lane& L) {
    const size_t pw = a.plane_words;
    const int y = L.y;
    const int ym = y == 0 ? a.H - 1 : y - 1;
    const int yp = y == a.H - 1 ? 0 : y + 1;
    const int w = 4 * L.q;
    const uint32_t* rm = a.src + (size_t)ym * a.Pq;  // row y-1 of plane 0
    const uint32_t* r0 = a.src + (size_t)y * a.Pq;   // row y
    const uint32_t* rp = a.src + (size_t)yp * a.Pq;  // row y+1
    const int m = RAGGED ? (L.q == a.nq - 1 ? a.Wq - w : 4) : 4;
    const int wl = L.q == 0 ? a.Wq - 1 : w - 1;      // word left of the quad (periodic)
    const int wr = L.q == a.nq - 1 ? 0 : w + 4;      // word right of the quad (periodic)

    // Rows y-1 feed the upward movers (NE 3, NW 4), row y the horizontal movers
    // (E 2, W 5) and the rest particle, row y+1 the downward movers (SW 0, SE 1).
    const uint4 i3 = ld4(rm + 3 * pw + w), i4 = ld4(rm + 4 * pw + w);
    const uint4 i2 = ld4(r0 + 2 * pw + w), i5 = ld4(r0 + 5 * pw + w);
    const uint4 i6 = ld4(r0 + 6 * pw + w);
    const uint4 i0 = ld4(rp + 0 * pw + w), i1 = ld4(rp + 1 * pw + w);
    uint4 sd = make_uint4(0u, 0u, 0u, 0u);
    if (SOLID) sd = ld4(a.solid + (size_t)y * a.Pq + w);

    uint4 n0, n1, n2, n3, n4, n5;
    if (!ODD) {
        // Even row: E, NE, SE come from x-1; W from x+1; NW, SW from x.
        uint32_t f2 = 0, f3 = 0, f1 = 0, f5 = 0;
        if (L.glob_left) { f2 = r0[2 * pw + wl]; f3 = rm[3 * pw + wl]; f1 = rp[1 * pw + wl]; }
        if (L.glob_right) f5 = r0[5 * pw + wr];
        n2 = from_left<RAGGED>(i2, f2, L, m);
        n3 = from_left<RAGGED>(i3, f3, L, m);
        n1 = from_left<RAGGED>(i1, f1, L, m);
        n5 = from_right<RAGGED>(i5, f5, L, m);
        n4 = i4;
        n0 = i0;
    } else {
        // Odd row: E from x-1; W, NW, SW from x+1; NE, SE from x.
        uint32_t f2 = 0, f5 = 0, f4 = 0, f0 = 0;
        if (L.glob_left) f2 = r0[2 * pw + wl];
        if (L.glob_right) { f5 = r0[5 * pw + wr]; f4 = rm[4 * pw + wr]; f0 = rp[0 * pw + wr]; }
        n2 = from_left<RAGGED>(i2, f2, L, m);
        n5 = from_right<RAGGED>(i5, f5, L, m);
        n4 = from_right<RAGGED>(i4, f4, L, m);
        n0 = from_right<RAGGED>(i0, f0, L, m);
        n3 = i3;
        n1 = i1;
    }

    const uint4 chi = rng_block((uint32_t)L.q, (uint32_t)y, a.t_lo, a.t_hi, 0u, a.key);
    uint4 gate = make_uint4(0u, 0u, 0u, 0u);
    if (FORCE) gate = rng_block((uint32_t)L.q, (uint32_t)y, a.t_lo, a.t_hi, 1u, a.key);

    uint4 o0, o1, o2, o3, o4, o5, o6;
#define FHP_WORD(J, C)                                                                          \
    {                                                                                           \
        Planes7 in{n0.C, n1.C, n2.C, n3.C, n4.C, n5.C, i6.C};                                   \
        Planes7 out = scatter(in, sd.C, chi.C);                                                 \
        if (FORCE) {                                                                            \
            const uint32_t cand = ~sd.C & out.m5 & ~out.m2;                                     \
            const uint32_t u = gate.C;                                                          \
            if (cand != 0u && (unsigned long long)u < a.ft.q[32]) {                             \
                const uint32_t f = forced_mask(cand, u, a.ft, [&](uint32_t d) {                 \
                    return word_of(rng_block((uint32_t)L.q, (uint32_t)y, a.t_lo, a.t_hi, 1u + d, \
                                             a.key), J);                                        \
                });                                                                             \
                out.m5 ^= f;                                                                    \
                out.m2 ^= f;                                                                    \
            }                                                                                   \
        }                                                                                       \
        o0.C = out.m0; o1.C = out.m1; o2.C = out.m2; o3.C = out.m3;                             \
        o4.C = out.m4; o5.C = out.m5; o6.C = out.rest;                                          \
    }
    FHP_WORD(0, x)
    FHP_WORD(1, y)
    FHP_WORD(2, z)
    FHP_WORD(3, w)
#undef FHP_WORD

    if (!L.active) return;
    if (RAGGED && m < 4) {
        // Keep the padding words of the last quad zero.
        if (m < 2) { o0.y = o1.y = o2.y = o3.y = o4.y = o5.y = o6.y = 0u; }
        if (m < 3) { o0.z = o1.z = o2.z = o3.z = o4.z = o5.z = o6.z = 0u; }
        o0.w = o1.w = o2.w = o3.w = o4.w = o5.w = o6.w = 0u;
    }
    uint32_t* d = a.dst + (size_t)y * a.Pq + w;
    st4(d + 0 * pw, o0);
    st4(d + 1 * pw, o1);
    st4(d + 2 * pw, o2);
    st4(d + 3 * pw, o3);
    st4(d + 4 * pw, o4);
    st4(d + 5 * pw, o5);
    st4(d + 6 * pw, o6);
}

template <bool SOLID, bool FORCE, bool RAGGED>
__global__ void __launch_bounds__(kBlock) fhp_step_kernel(const StepArgs a) {
    const Lane L = map_lane(a);
    if (L.y & 1) step_quad<SOLID, FORCE, RAGGED, true>(a, L);
    else step_quad<SOLID, FORCE, RAGGED, false>(a, L);
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

template <bool SOLID, bool FORCE>
cudaError_t launch_variant(const StepArgs& a, bool ragged, long long warps, cudaStream_t s) {
    const long long threads = warps * 32;
    const unsigned grid = (unsigned)((threads + kBlock - 1) / kBlock);
    if (ragged) fhp_step_kernel<SOLID, FORCE, true><<<grid, kBlock, 0, s>>>(a);
    else fhp_step_kernel<SOLID, FORCE, false><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
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

cudaError_t launch_step(const Geometry& g, const uint32_t* src, uint32_t* dst,
                        const uint32_t* solid, bool has_solid, bool force,
                        const ForcingTable& ft, Key2 key, uint64_t t, cudaStream_t stream) {
    StepArgs a;
    a.src = src;
    a.dst = dst;
    a.solid = solid;
    a.plane_words = g.plane_words;
    a.H = g.H;
    a.Wq = g.Wq;
    a.nq = g.nq;
    a.Pq = g.Pq;
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
    a.key = key;
    a.t_lo = (uint32_t)t;
    a.t_hi = (uint32_t)(t >> 32);
    a.ft = ft;
    const bool ragged = (g.Wq % 4) != 0;
    if (has_solid) {
        return force ? launch_variant<true, true>(a, ragged, warps, stream)
                     : launch_variant<true, false>(a, ragged, warps, stream);
    }
    return force ? launch_variant<false, true>(a, ragged, warps, stream)
                 : launch_variant<false, false>(a, ragged, warps, stream);
}

}  // namespace fhp
