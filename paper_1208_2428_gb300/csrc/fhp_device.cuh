// fhp_device.cuh -- device building blocks of the FHP step on bit-planes.
//
// A lattice row is stored as words of 32 nodes: bit (x mod 32) of word x/32
// of plane i holds occupation bit i of node x (i = 0..5 movers along c_i at
// (i-2)*60 degrees, 6 rest particle; a separate plane holds the solid flag).
// Every function here works on whole words, so one instruction updates 32
// nodes (multi-spin coding of the node byte of arXiv:1208.2428, Section 2).
#pragma once

#include <cstdint>

#include "fhp_internal.h"

namespace fhp {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two 32x32
// -> 64-bit products whose halves are swapped and xored with the other two
// counter words and the round key; the key advances by two Weyl constants.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, Key2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t x0 = c.x, x2 = c.z;
        const uint32_t hi_a = __umulhi(0xD2511F53u, x0);
        const uint32_t lo_a = 0xD2511F53u * x0;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, x2);
        const uint32_t lo_b = 0xCD9E8D57u * x2;
        c = make_uint4(hi_b ^ c.y ^ k.lo, lo_b, hi_a ^ c.w ^ k.hi, lo_a);
        k.lo += 0x9E3779B9u;
        k.hi += 0xBB67AE85u;
    }
    return c;
}

// Random block of the four words 4q..4q+3 of row y at step t for `stream`
// (stream 0: chirality, 1 + d: forcing draw d).  Counter layout:
// (q, y, t mod 2^32, stream + (t div 2^32) * 2^16).
__device__ __forceinline__ uint4 rng_block(uint32_t q, uint32_t y, uint32_t t_lo, uint32_t t_hi,
                                           uint32_t stream, Key2 key) {
    return philox4x32_10(make_uint4(q, y, t_lo, stream | (t_hi << 16)), key);
}

__device__ __forceinline__ uint32_t word_of(const uint4& v, int j) {
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

// ---------------------------------------------------------------------------
// Scattering of 32 nodes at once (FHP-II rule set, or FHP-I when the
// rest-particle rules are masked off, bounce-back on solid).
// Every rule of the set exchanges the particles of a node for another set
// with the same mass and momentum, so the update is a per-bit flip mask:
//   head-on pair {i, i+3} (others empty)  -> turned by +60 deg (chi 0) or -60 deg (chi 1)
//   triple {0,2,4} <-> {1,3,5}            -> all six movers flip
//   rest + {i}  <->  {i-1, i+1}            -> rest bit and movers i-1, i, i+1 flip
// (each with the rest particle as a spectator where it is not involved).
// Solid nodes reverse every mover (i <-> i+3) and keep the rest particle.
// ---------------------------------------------------------------------------
struct Planes7 {
    uint32_t m0, m1, m2, m3, m4, m5, rest;
};

// rest_rules: all ones applies the rest-particle rules (FHP-II), zero skips
// them (FHP-I: head-on and three-body collisions only).
__host__ __device__ __forceinline__ Planes7 scatter(const Planes7 in, uint32_t solid, uint32_t chi,
                                                    uint32_t rest_rules = 0xFFFFFFFFu) {
    const uint32_t a0 = in.m0, a1 = in.m1, a2 = in.m2, a3 = in.m3, a4 = in.m4, a5 = in.m5;
    const uint32_t r = in.rest;

    // Occupation of the three opposite pairs (0,3), (1,4), (2,5).
    const uint32_t full0 = a0 & a3, full1 = a1 & a4, full2 = a2 & a5;
    const uint32_t empty0 = ~(a0 | a3), empty1 = ~(a1 | a4), empty2 = ~(a2 | a5);
    // Direction i present without its opposite.
    const uint32_t lone0 = a0 & ~a3, lone3 = a3 & ~a0;
    const uint32_t lone1 = a1 & ~a4, lone4 = a4 & ~a1;
    const uint32_t lone2 = a2 & ~a5, lone5 = a5 & ~a2;

    // Head-on collisions: exactly one pair occupied, the other two empty.
    const uint32_t head0 = full0 & empty1 & empty2;
    const uint32_t head1 = full1 & empty0 & empty2;
    const uint32_t head2 = full2 & empty0 & empty1;
    // Symmetric triples.
    const uint32_t triple = (lone0 & lone2 & lone4) | (lone1 & lone3 & lone5);

    // Rest-particle rule for direction i: with rest, mover i alone; without
    // rest, exactly the movers i-1 and i+1.
    const uint32_t one0 = lone0 & empty1 & empty2, one3 = lone3 & empty1 & empty2;
    const uint32_t one1 = lone1 & empty0 & empty2, one4 = lone4 & empty0 & empty2;
    const uint32_t one2 = lone2 & empty0 & empty1, one5 = lone5 & empty0 & empty1;
    const uint32_t two0 = lone5 & lone1 & empty0, two3 = lone2 & lone4 & empty0;
    const uint32_t two1 = lone0 & lone2 & empty1, two4 = lone3 & lone5 & empty1;
    const uint32_t two2 = lone1 & lone3 & empty2, two5 = lone4 & lone0 & empty2;
    const uint32_t q0 = ((r & one0) | (~r & two0)) & rest_rules, q1 = ((r & one1) | (~r & two1)) & rest_rules;
    const uint32_t q2 = ((r & one2) | (~r & two2)) & rest_rules, q3 = ((r & one3) | (~r & two3)) & rest_rules;
    const uint32_t q4 = ((r & one4) | (~r & two4)) & rest_rules, q5 = ((r & one5) | (~r & two5)) & rest_rules;

    // Head-on flips of movers j and j+3: pair j%3 itself, and the pair it is
    // turned onto, which depends on the chirality.
    const uint32_t turn0 = head0 | (chi & head1) | (~chi & head2);
    const uint32_t turn1 = head1 | (chi & head2) | (~chi & head0);
    const uint32_t turn2 = head2 | (chi & head0) | (~chi & head1);

    Planes7 out;
    const uint32_t fl = ~solid;
    out.m0 = (solid & a3) | (fl & (a0 ^ (triple | turn0 | q5 | q0 | q1)));
    out.m1 = (solid & a4) | (fl & (a1 ^ (triple | turn1 | q0 | q1 | q2)));
    out.m2 = (solid & a5) | (fl & (a2 ^ (triple | turn2 | q1 | q2 | q3)));
    out.m3 = (solid & a0) | (fl & (a3 ^ (triple | turn0 | q2 | q3 | q4)));
    out.m4 = (solid & a1) | (fl & (a4 ^ (triple | turn1 | q3 | q4 | q5)));
    out.m5 = (solid & a2) | (fl & (a5 ^ (triple | turn2 | q4 | q5 | q0)));
    out.rest = r ^ (fl & (q0 | q1 | q2 | q3 | q4 | q5));
    return out;
}

// ---------------------------------------------------------------------------
// Scattering of 32 nodes at once, FHP-III (collision-saturated): every fluid
// state that shares its mass and momentum with another state changes, as a
// per-bit flip mask over disjoint state classes (k = 0..5 below, indices of
// movers mod 6; "pair p" = movers p and p+3):
//   zero momentum (every pair full or empty, or a triple): the movers turn
//     by +60 deg (chi 0) or -60 deg (chi 1), the rest particle stays;
//   rest + k <-> {k-1, k+1}                    flip rest, k-1, k, k+1
//   all movers but k+3 <-> rest + {k-1,k,k+1,k+3}   flip rest, k+2, k+3, k+4
//   momentum c_k, mass 3, chi 0: A = k + pair k+1 -> B = k + pair k+2
//     -> C = rest + {k-1, k+1} -> A  (chi 1 backwards)
//   momentum c_k, mass 4, chi 0: D = rest + k + pair k+2 -> E = rest + k +
//     pair k+1 -> F = {k-1, k+1} + pair k -> D  (chi 1 backwards)
// Solid nodes reverse every mover (i <-> i+3) and keep the rest particle.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ Planes7 scatter_saturated(const Planes7 in, uint32_t solid, uint32_t chi) {
    const uint32_t a[6] = {in.m0, in.m1, in.m2, in.m3, in.m4, in.m5};
    const uint32_t r = in.rest, nr = ~in.rest, nchi = ~chi;
    uint32_t full[3], empty[3], lone[6];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        full[p] = a[p] & a[p + 3];
        empty[p] = ~(a[p] | a[p + 3]);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) lone[i] = a[i] & ~a[(i + 3) % 6];
    const uint32_t triple = (lone[0] & lone[2] & lone[4]) | (lone[1] & lone[3] & lone[5]);
    const uint32_t zero = ((full[0] | empty[0]) & (full[1] | empty[1]) & (full[2] | empty[2])) | triple;

    uint32_t f[6], fr = 0u;
#pragma unroll
    for (int i = 0; i < 6; ++i)
        f[i] = zero & (a[i] ^ ((chi & a[(i + 1) % 6]) | (nchi & a[(i + 5) % 6])));
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int km2 = (k + 4) % 6, km1 = (k + 5) % 6, kp1 = (k + 1) % 6, kp2 = (k + 2) % 6, kp3 = (k + 3) % 6,
                  kp4 = (k + 4) % 6;
        const uint32_t pk = full[k % 3], p1 = full[(k + 1) % 3], p2 = full[(k + 2) % 3];
        const uint32_t x = p1 & lone[k] & empty[(k + 2) % 3];       // k + pair k+1
        const uint32_t y = p2 & lone[k] & empty[(k + 1) % 3];       // k + pair k+2
        const uint32_t side = lone[km1] & lone[kp1];                // movers k-1 and k+1
        const uint32_t A = x & nr, E = x & r, B = y & nr, D = y & r;
        const uint32_t C = r & side & empty[k % 3], F = nr & side & pk;
        // two-state classes
        const uint32_t q = (r & lone[k] & empty[(k + 1) % 3] & empty[(k + 2) % 3]) | (nr & side & empty[k % 3]);
        const uint32_t s5 = (nr & p1 & p2 & lone[k]) | (r & pk & side);
        // three-state cycles
        const uint32_t ab = (nchi & A) | (chi & B) | (nchi & D) | (chi & E);   // flip k-2, k-1, k+1, k+2
        const uint32_t bc = (nchi & B) | (chi & C);                           // flip k, k+1, k+2, rest
        const uint32_t ca = (nchi & C) | (chi & A);                           // flip k-2, k-1, k, rest
        const uint32_t ef = (nchi & E) | (chi & F);                           // flip k-2, k-1, k+3, rest
        const uint32_t fd = (nchi & F) | (chi & D);                           // flip k+1, k+2, k+3, rest
        f[km1] |= q | ab | ca | ef;
        f[k] |= q | bc | ca;
        f[kp1] |= q | ab | bc | fd;
        f[kp2] |= s5 | ab | bc | fd;
        f[kp3] |= s5 | ef | fd;
        f[kp4] |= s5;
        f[km2] |= ab | ca | ef;
        fr |= q | s5 | bc | ca | ef | fd;
    }
    Planes7 out;
    const uint32_t fl = ~solid;
    out.m0 = (solid & a[3]) | (fl & (a[0] ^ f[0]));
    out.m1 = (solid & a[4]) | (fl & (a[1] ^ f[1]));
    out.m2 = (solid & a[5]) | (fl & (a[2] ^ f[2]));
    out.m3 = (solid & a[0]) | (fl & (a[3] ^ f[3]));
    out.m4 = (solid & a[1]) | (fl & (a[4] ^ f[4]));
    out.m5 = (solid & a[2]) | (fl & (a[5] ^ f[5]));
    out.rest = r ^ (fl & fr);
    return out;
}

// ---------------------------------------------------------------------------
// Forcing (ForcingTable: Q_g, g = 0..32, in units of 2^-32 -- a uniform
// u < Q_g means "one of the next g candidates is forced").
// ---------------------------------------------------------------------------
// Forced-node mask of one word: `cand` holds the candidates (fluid, bit 5
// set, bit 2 clear), `u0` is the word's first forcing draw, `more(d)` returns
// draw d >= 1.  Walk: while candidates remain, the least g with u < Q_g picks
// the g-th remaining candidate; candidates before it are not forced; a fresh
// draw decides the ones after it.
template <class MoreDraws>
__device__ __forceinline__ uint32_t forced_mask(uint32_t cand, uint32_t u0, const ForcingTable& ft,
                                                MoreDraws more) {
    uint32_t forced = 0;
    uint32_t u = u0;
    uint32_t draw = 0;
    while (cand) {
        const int remaining = __popc(cand);
        if ((unsigned long long)u >= ft.q[remaining]) break;
        int lo = 1, hi = remaining;  // least g in [1, remaining] with u < Q_g
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((unsigned long long)u < ft.q[mid]) hi = mid; else lo = mid + 1;
        }
        uint32_t c = cand;
        for (int i = 1; i < lo; ++i) c &= c - 1;   // drop the lo-1 lowest candidates
        const int pos = __ffs(c) - 1;              // the lo-th candidate
        forced |= 1u << pos;
        cand = pos == 31 ? 0u : (cand & (0xFFFFFFFFu << (pos + 1)));
        if (!cand) break;   // no candidate left: the next draw would decide nothing
        ++draw;
        u = more(draw);
    }
    return forced;
}

}  // namespace fhp
