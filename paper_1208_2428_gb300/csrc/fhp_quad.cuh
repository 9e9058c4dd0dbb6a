// fhp_quad.cuh -- per-quad building blocks shared by the step kernels
// (fhp_step.cu), the temporally blocked kernel (fhp_block.cu) and the batch
// kernels (fhp_batch.cu): 128-bit plane access, the one-node shifts of the
// motion step, scattering plus forcing of one quad (4 words = 128 nodes), the
// mbarrier / bulk-copy helpers (inline PTX) of the shared-memory pipelines,
// and the completion counters of the multi-step kernels.
#pragma once

#include "fhp_debug.cuh"
#include "fhp_device.cuh"
#include "fhp_internal.h"

namespace fhp {
namespace {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s bound on any wait

__device__ __forceinline__ uint4 ld4(const uint32_t* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ void st4(uint32_t* p, uint4 v) { *reinterpret_cast<uint4*>(p) = v; }

// New bit x takes old bit x-1; `left` is the word left of the quad.
__device__ __forceinline__ uint4 pull_left(uint4 v, uint32_t left) {
    return make_uint4(__funnelshift_l(left, v.x, 1), __funnelshift_l(v.x, v.y, 1),
                      __funnelshift_l(v.y, v.z, 1), __funnelshift_l(v.z, v.w, 1));
}

// New bit x takes old bit x+1; `right` is the word right of the quad's last
// valid word (m valid words; the rest of a ragged last quad is padding).
template <bool RAGGED>
__device__ __forceinline__ uint4 pull_right(uint4 v, uint32_t right, int m) {
    uint32_t n0 = v.y, n1 = v.z, n2 = v.w;
    if (RAGGED) {
        if (m == 1) n0 = right;
        if (m == 2) n1 = right;
        if (m == 3) n2 = right;
    }
    return make_uint4(__funnelshift_r(v.x, n0, 1), __funnelshift_r(v.y, n1, 1),
                      __funnelshift_r(v.z, n2, 1), __funnelshift_r(v.w, right, 1));
}

// Where one step writes and which step it is (varies per step in the
// multi-step kernel; the single-step kernels take it from StepArgs).
struct StepVar {
    uint32_t* dst;
    uint32_t t_lo, t_hi;
};

// Compile-time flag carried by a value (selects code inside collide_quad).
template <bool B>
struct Flag {
    static constexpr bool value = B;
};

// Scattering, bounce-back and forcing of one quad (global quad index q of
// row y at step v.t) whose movers have already been pulled (n0..n5), with
// rest plane i6 and solid plane sd; the seven result planes go to o[0..6].
// SAT selects the FHP-III (collision-saturated) rule set at compile time;
// otherwise FHP-II or FHP-I by the lattice's rest-particle mask.
//
// Two uniform branches select code with constants in it: the rule set (one
// per launch or batch tile), and whether any quad of the active lanes holds a
// solid node -- most warps hold none, and their words then skip the
// bounce-back multiplexers (the result is the same: a word without solid
// nodes takes the fluid branch of every multiplexer).  On the 16384 x 4096
// cylinder the two changes here (this one and the forcing pre-check below)
// raised the multi-step kernel from 3159 to 3310 GSUPS and the 512-lattice
// batch from 2484 to 2640; the resident kernel on the 4096 x 1024 channel
// (p = 1e-3) went from 845 to 890.
//
// Forcing: a word enters the candidate walk only if its first draw u is
// below K (P + 1) for its K candidates, an upper bound of Q_K (the walk's
// own first test, u < Q_K, decides exactly inside); a word without
// candidates never enters.  The bound needs no table read, so the ~99.7 % of
// words it rejects cost a popcount, a multiply and a compare.
template <bool SOLID, bool FORCE, bool SAT = false>
__device__ __forceinline__ void collide_quad(const StepArgs& a, const StepVar& v, int q, int y, uint4 n0, uint4 n1,
                                             uint4 n2, uint4 n3, uint4 n4, uint4 n5, uint4 i6, uint4 sd,
                                             uint4 (&o)[7]) {
    const uint4 chi = rng_block((uint32_t)q, (uint32_t)(y + a.y_base), v.t_lo, v.t_hi, 0u, a.key);
    uint4 gate = make_uint4(0u, 0u, 0u, 0u);
    if (FORCE) gate = rng_block((uint32_t)q, (uint32_t)(y + a.y_base), v.t_lo, v.t_hi, 1u, a.key);

#define FHP_WORD(J, C, RR, S)                                                                   \
    {                                                                                           \
        Planes7 in{n0.C, n1.C, n2.C, n3.C, n4.C, n5.C, i6.C};                                   \
        Planes7 out = SAT ? scatter_saturated(in, S ? sd.C : 0u, chi.C)                         \
                          : scatter(in, S ? sd.C : 0u, chi.C, RR);                              \
        if (FORCE) {                                                                            \
            const uint32_t cand = (S ? ~sd.C : 0xFFFFFFFFu) & out.m5 & ~out.m2;                 \
            const uint32_t u = gate.C;                                                          \
            if ((unsigned long long)u < (unsigned long long)__popc(cand) * a.ft.p_plus_1) {     \
                const uint32_t f = forced_mask(cand, u, a.ft, [&](uint32_t d) {                 \
                    return word_of(rng_block((uint32_t)q, (uint32_t)(y + a.y_base), v.t_lo, v.t_hi, 1u + d,   \
                                             a.key), J);                                        \
                });                                                                             \
                out.m5 ^= f;                                                                    \
                out.m2 ^= f;                                                                    \
            }                                                                                   \
        }                                                                                       \
        o[0].C = out.m0; o[1].C = out.m1; o[2].C = out.m2; o[3].C = out.m3;                     \
        o[4].C = out.m4; o[5].C = out.m5; o[6].C = out.rest;                                    \
    }
    auto words = [&](auto solid, auto rest) {
        constexpr bool S = decltype(solid)::value;
        constexpr uint32_t RR = decltype(rest)::value ? 0xFFFFFFFFu : 0u;
        FHP_WORD(0, x, RR, S)
        FHP_WORD(1, y, RR, S)
        FHP_WORD(2, z, RR, S)
        FHP_WORD(3, w, RR, S)
    };
#undef FHP_WORD
    // (Not for FHP-III: a second copy of its larger network measured 11 %
    // slower on the cylinder.)
    bool solid_here = SOLID;
    if (SOLID && !SAT) solid_here = __any_sync(__activemask(), (sd.x | sd.y | sd.z | sd.w) != 0u);
    if (SAT || a.rest_rules != 0u) {
        if (solid_here) words(Flag<SOLID>{}, Flag<true>{});
        else words(Flag<false>{}, Flag<true>{});
    } else {
        if (solid_here) words(Flag<SOLID>{}, Flag<false>{});
        else words(Flag<false>{}, Flag<false>{});
    }
}

// Store a quad's seven result planes to global memory (the padding words of
// a ragged last quad are written as zero).
template <bool RAGGED>
__device__ __forceinline__ void store_quad(const StepArgs& a, uint32_t* dst, int q, int y, int m, uint4 (&o)[7]) {
    if (RAGGED && m < 4) {
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            if (m < 2) o[k].y = 0u;
            if (m < 3) o[k].z = 0u;
            o[k].w = 0u;
        }
    }
    if (!dbg_ok(y >= 0 && y < a.H && q >= 0 && q < a.nq, a.err, kSiteStoreQuad)) return;
    const size_t pw = a.plane_words;
    uint32_t* d = dst + (size_t)y * a.Pq + 4 * q;
#pragma unroll
    for (int k = 0; k < 7; ++k) st4(d + k * pw, o[k]);
}

// Collide and store one quad.
template <bool SOLID, bool FORCE, bool RAGGED, bool SAT = false>
__device__ __forceinline__ void finish_quad(const StepArgs& a, const StepVar& v, int q, int y, int m, uint4 n0,
                                            uint4 n1, uint4 n2, uint4 n3, uint4 n4, uint4 n5, uint4 i6,
                                            uint4 sd, bool active) {
    uint4 o[7];
    collide_quad<SOLID, FORCE, SAT>(a, v, q, y, n0, n1, n2, n3, n4, n5, i6, sd, o);
    if (active) store_quad<RAGGED>(a, v.dst, q, y, m, o);
}

// ---------------------------------------------------------------------------
// Bulk-copy kernel: mbarrier / cp.async.bulk helpers (inline PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// The same test, suspending the thread for up to about `hint_ns` while the
// phase is incomplete (the barrier's completion wakes it earlier).  Used by
// watchers that are not participants of the barrier: for them the phase
// parity can alias once the barrier has moved on by two phases, so they take
// the result as a wake-up only and read their own counters for the truth.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The waiting loop of mbar_wait_bounded, out of line (rarely entered).
__device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity) {
    const unsigned long long start = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - start > kWaitLimitNs) return false;
    }
}

// Wait for phase `parity` of `bar`; gives up (returns false) after
// kWaitLimitNs.  The first test is inline, so a phase that has already
// completed costs no call (the call's calling convention made the batch
// kernels' consumers spill registers: 2638 -> 3064 GSUPS on the 512-lattice
// ensemble, 3306 -> 3430 for the multi-step kernel on the cylinder).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    return mbar_try_wait(bar, parity) || mbar_wait_slow(bar, parity);
}

// The same wait entirely out of line: for the single-step ring kernel's
// consumers, where the inline test made the register allocation spill
// (3370 -> 3190 GSUPS on the paper-size lattice).
__device__ __noinline__ bool mbar_wait_bounded_call(uint64_t* bar, uint32_t parity) {
    return mbar_try_wait(bar, parity) || mbar_wait_slow(bar, parity);
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Stage layout: slot k (plane k for k < 7, the solid plane for k = 7) holds
// R rows of Pq words; staged row r of every slot feeds output row y0 + r, so
// slots 3, 4 hold source rows y0 + r - 1 and slots 0, 1 rows y0 + r + 1.
template <bool SOLID>
__device__ void issue_tile(const StepArgs& a, const TileArgs& ta, const uint32_t* src, int tile,
                           uint32_t* stage, uint64_t* bar) {
    constexpr int NP = SOLID ? 8 : 7;
    const int y0 = tile * ta.R;
    const int rows = min(ta.R, a.H - y0);
    const uint32_t row_bytes = (uint32_t)a.Pq * 4u;
    mbar_arrive_expect_tx(bar, (uint32_t)NP * (uint32_t)rows * row_bytes);
#pragma unroll
    for (int slot = 0; slot < NP; ++slot) {
        const uint32_t* plane = slot < 7 ? src + (size_t)slot * a.plane_words : a.solid;
        const int shift = (slot == 3 || slot == 4) ? -1 : (slot == 0 || slot == 1) ? 1 : 0;
        int r = 0;
        while (r < rows) {
            int yy = y0 + shift + r;
            if (yy < 0) yy += a.H;
            if (yy >= a.H) yy -= a.H;
            const int run = min(rows - r, a.H - yy);  // contiguous rows up to the end of the plane
            if (!dbg_ok(yy >= 0 && yy < a.H && run >= 1 && r + run <= ta.R, a.err, kSiteIssueTile)) break;
            bulk_copy_g2s(stage + ((size_t)slot * ta.R + r) * a.Pq, plane + (size_t)yy * a.Pq,
                          (uint32_t)run * row_bytes, bar);
            r += run;
        }
    }
}

template <bool SOLID, bool FORCE, bool RAGGED, bool SAT = false>
__device__ __forceinline__ void quad_from_stage(const StepArgs& a, const StepVar& v, const TileArgs& ta,
                                                const uint32_t* stage, int r, int y, int q) {
    const int Pq = a.Pq, R = ta.R;
    const int w = 4 * q;
    const int m = RAGGED ? (q == a.nq - 1 ? a.Wq - w : 4) : 4;
    const int wl = q == 0 ? a.Wq - 1 : w - 1;       // word left of the quad (periodic)
    const int wr = q == a.nq - 1 ? 0 : w + 4;       // word right of the quad (periodic)
    if (!dbg_ok(r >= 0 && r < R && q >= 0 && q < a.nq && w + 3 < Pq && wl >= 0 && wl < a.Wq && wr < a.Wq, a.err,
                kSiteStageQuad))
        return;
    const uint32_t* s0 = stage + (size_t)r * Pq;    // slot 0, row r
    const size_t slot = (size_t)R * Pq;
    const uint4 i0 = ld4(s0 + 0 * slot + w), i1 = ld4(s0 + 1 * slot + w);
    const uint4 i2 = ld4(s0 + 2 * slot + w), i3 = ld4(s0 + 3 * slot + w);
    const uint4 i4 = ld4(s0 + 4 * slot + w), i5 = ld4(s0 + 5 * slot + w);
    const uint4 i6 = ld4(s0 + 6 * slot + w);
    uint4 sd = make_uint4(0u, 0u, 0u, 0u);
    if (SOLID) sd = ld4(s0 + 7 * slot + w);
    uint4 n0, n1, n2, n3, n4, n5;
    if ((y & 1) == 0) {
        // Even row: E, NE, SE come from x-1; W from x+1; NW, SW from x.
        n2 = pull_left(i2, s0[2 * slot + wl]);
        n3 = pull_left(i3, s0[3 * slot + wl]);
        n1 = pull_left(i1, s0[1 * slot + wl]);
        n5 = pull_right<RAGGED>(i5, s0[5 * slot + wr], m);
        n4 = i4;
        n0 = i0;
    } else {
        // Odd row: E from x-1; W, NW, SW from x+1; NE, SE from x.
        n2 = pull_left(i2, s0[2 * slot + wl]);
        n5 = pull_right<RAGGED>(i5, s0[5 * slot + wr], m);
        n4 = pull_right<RAGGED>(i4, s0[4 * slot + wr], m);
        n0 = pull_right<RAGGED>(i0, s0[0 * slot + wr], m);
        n3 = i3;
        n1 = i1;
    }
    finish_quad<SOLID, FORCE, RAGGED, SAT>(a, v, q, y, m, n0, n1, n2, n3, n4, n5, i6, sd, true);
}

// SAT selects the FHP-III rule set (collision-saturated scattering).
template <bool SOLID, bool FORCE, bool RAGGED, bool SAT = false>
__device__ __forceinline__ void compute_tile(const StepArgs& a, const StepVar& v, const TileArgs& ta, int tile,
                                             const uint32_t* stage, int tid, int nthreads) {
    const int y0 = tile * ta.R;
    const int rows = min(ta.R, a.H - y0);
    // Items ordered even local rows first, then odd ones, so that the row
    // parity (which selects the shift pattern) is uniform within a warp.
    const int even_rows = (rows + 1) >> 1;
    const int even_items = even_rows * a.nq;
    const int items = rows * a.nq;
    for (int it = tid; it < items; it += nthreads) {
        const int h = it >= even_items;
        const uint32_t j = (uint32_t)(h ? it - even_items : it);
        const int k = (int)(((unsigned long long)j * ta.nq_magic) >> 32);  // j / nq
        const int q = (int)j - k * a.nq;
        const int r = 2 * k + h;
        quad_from_stage<SOLID, FORCE, RAGGED, SAT>(a, v, ta, stage, r, y0 + r, q);
    }
}

// Cross-CTA completion counters of the multi-step kernels (a tile's counter
// counts the consumer warps that finished it, summed over steps).
__device__ __forceinline__ unsigned int ld_relaxed_gpu(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until the counters of tiles a, b (and c if check_c) reach `target`.
// The loads are relaxed so that they are in flight together; one acquire
// fence after they all pass orders the later reads of the tiles' rows.
// Gives up (false) after kWaitLimitNs.
__device__ __noinline__ bool wait_tiles(const unsigned int* done, int ta_, int tb, int tc, bool check_c,
                                        unsigned int target) {
    unsigned long long start = 0;
    for (;;) {
        const unsigned int va = ld_relaxed_gpu(done + ta_);
        const unsigned int vb = ld_relaxed_gpu(done + tb);
        const unsigned int vc = check_c ? ld_relaxed_gpu(done + tc) : target;
        if (va >= target && vb >= target && vc >= target) {
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            return true;
        }
        const unsigned long long now = global_ns();
        if (start == 0) start = now;
        else if (now - start > kWaitLimitNs) return false;
        __nanosleep(32);
    }
}

__device__ __forceinline__ void st_release_cta_shared(unsigned int* p, unsigned int v) {
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int ld_acquire_cta_shared(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

}  // namespace
}  // namespace fhp
