/*
 * fhp_oracle.c -- plain, slow CPU oracle for the FHP lattice-gas step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) links, loads or calls this file.  Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark use it.
 *
 * It shares no code, header or table with the CUDA path.  Every function
 * follows the model of Szkoda, Koza & Tykierko, "Accelerating cellular
 * automata simulations using AVX and CUDA" (arXiv:1208.2428), Section 2:
 *
 *   - a node is one byte: bits 0-5 are particles moving with velocity c_i,
 *     bit 6 is the rest particle, bit 7 marks a boundary (solid) node
 *     (Section 2, Fig. 1);
 *   - one time step is motion (every particle hops to the neighbour along its
 *     velocity, the rest particle stays) followed by scattering through a
 *     256-entry look-up table indexed by the node byte; the same table holds
 *     the bounce-back entries of boundary nodes (Section 2, Fig. 2);
 *   - the triangular lattice is stored as a rectangular array whose odd rows
 *     are shifted by half a lattice constant (Section 2, Fig. 3);
 *   - periodic boundaries in x (Section 2, Fig. 4), walls as solid rows;
 *   - forcing: a node whose bits match (..1..0..) -- bit 5 set, bit 2 clear --
 *     has bits 2 and 5 exchanged with probability p (Section 2, last
 *     paragraph).
 *
 * Where the paper is silent (the picture of the rule set, the direction
 * numbering, the random-number source, the step order) this file follows the
 * readings listed in the design notes of the repository (R-dir, R-map,
 * R-order, R-rules, R-fhp3, R-solid, R-rng, R-force, R-cg).
 *
 * Direction numbering (R-dir): c_i points at angle (i-2)*60 degrees,
 * counter-clockwise from +x; i+3 (mod 6) is opposite to i.
 *     0 = SW, 1 = SE, 2 = E, 3 = NE, 4 = NW, 5 = W, 6 = rest, 7 = solid.
 * Row index y grows upwards; odd rows sit half a lattice constant to the
 * right of even rows (R-map).
 *
 * Parity status: every function here is pinned by the not-gpu tests
 * (closed forms, invariants, brute force, a library generator); none is
 * "parity unpinned".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Each round multiplies two counter words by the */
/* round multipliers, keeps both halves of the 64-bit products, and mixes in */
/* the other two counter words and the round key; the key is bumped by the   */
/* two Weyl constants between rounds.                                        */
/* ------------------------------------------------------------------------ */
ORACLE_EXPORT void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                                        uint32_t out[4]) {
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)mult0 * c0;
        uint64_t prod1 = (uint64_t)mult1 * c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += weyl0;
        k1 += weyl1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One random 32-bit word for (word w of row y, step t, stream s) (R-rng):
 * the Philox block with counter (w/4, y, t mod 2^32, s + (t/2^32)*2^16) and
 * key (seed mod 2^32, seed / 2^32) covers the four words 4*(w/4) .. +3;
 * word w takes output w mod 4.  Bit (x mod 32) of the word belongs to node x. */
static uint32_t rng_word(uint64_t seed, uint64_t t, int y, int w, uint32_t stream) {
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = (uint32_t)(w >> 2);
    ctr[1] = (uint32_t)y;
    ctr[2] = (uint32_t)t;
    ctr[3] = stream | ((uint32_t)(t >> 32) << 16);
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    oracle_philox4x32_10(ctr, key, out);
    return out[w & 3];
}

ORACLE_EXPORT uint32_t oracle_rng_word(uint64_t seed, uint64_t t, int y, int w, uint32_t stream) {
    return rng_word(seed, t, y, w, stream);
}

/* ------------------------------------------------------------------------ */
/* Collision table (Section 2: scattering through a 256-entry table; Fig. 2  */
/* is not legible in the source, so the FHP-II rule set of reading R-rules   */
/* is written out here).                                                     */
/* ------------------------------------------------------------------------ */
#define REST_BIT 6
#define SOLID_BIT 7

static int dir_bit(int i) { return 1 << (((i % 6) + 6) % 6); }

/* FHP-III, the collision-saturated rule set (reading R-fhp3; the paper
 * cites the model family but prints no table).  A fluid state (7 bits) whose
 * mass and momentum are shared by no other state stays; every other state
 * becomes another state of its class:
 *   - zero momentum (head-on pairs, triples, two head-on pairs, each with or
 *     without the rest particle): the moving particles turn by +60 degrees
 *     (chirality 0) or -60 degrees (chirality 1);
 *   - a class of two states (rest + i <-> {i-1, i+1}, and the particle-hole
 *     duals of those pairs): the other state;
 *   - a class of three states (momentum c_k, mass 3 or 4): a cycle, written
 *     out below for momentum c_2 and turned to c_k; chirality 1 runs it
 *     backwards.
 * Momentum is counted in the lattice basis (c_2, c_3): c_0 = (0,-1),
 * c_1 = (1,-1), c_2 = (1,0), c_3 = (0,1), c_4 = (-1,1), c_5 = (-1,0). */
static void node_invariants(int s, int* mass, int* px, int* py) {
    static const int vx[6] = {0, 1, 1, 0, -1, -1}, vy[6] = {-1, -1, 0, 1, 1, 0};
    *mass = (s >> REST_BIT) & 1;
    *px = *py = 0;
    for (int i = 0; i < 6; ++i)
        if (s & dir_bit(i)) {
            ++*mass;
            *px += vx[i];
            *py += vy[i];
        }
}

/* Moving particle i becomes i + by (mod 6); the rest bit is kept. */
static int turn_movers(int s, int by) {
    int out = s & (1 << REST_BIT);
    for (int i = 0; i < 6; ++i)
        if (s & dir_bit(i)) out |= dir_bit(i + by);
    return out;
}

static int fhp3_scatter(int s, int chirality) {
    int mass, px, py;
    node_invariants(s, &mass, &px, &py);
    int cls[128], n = 0;
    for (int t = 0; t < 128; ++t) {
        int m2, x2, y2;
        node_invariants(t, &m2, &x2, &y2);
        if (m2 == mass && x2 == px && y2 == py) cls[n++] = t;
    }
    if (n == 1) return s;
    if (px == 0 && py == 0) return turn_movers(s, chirality == 0 ? 1 : 5);
    if (n == 2) return cls[0] == s ? cls[1] : cls[0];
    /* Three states with momentum c_k.  For k = 2 (E), chirality 0:
     *   mass 3: E + pair {0,3} -> E + pair {1,4} -> rest + {1,3} -> back;
     *   mass 4: rest + E + pair {1,4} -> rest + E + pair {0,3}
     *           -> {1,3} + pair {2,5} -> back
     * (the mass-4 cycle is the particle-hole dual of the mass-3 one). */
    static const int cyc3[3] = {0x0D, 0x16, 0x4A}, cyc4[3] = {0x56, 0x4D, 0x2E};
    static const int vx[6] = {0, 1, 1, 0, -1, -1}, vy[6] = {-1, -1, 0, 1, 1, 0};
    int k = 0;
    while (vx[k] != px || vy[k] != py) ++k;
    const int* cyc = mass == 3 ? cyc3 : cyc4;
    const int e = turn_movers(s, 2 - k + 6);
    int j = 0;
    while (cyc[j] != e) ++j;
    return turn_movers(cyc[(j + (chirality == 0 ? 1 : 2)) % 3], k - 2 + 6);
}

/* Rule sets: 2 = FHP-II (reading R-rules), 1 = FHP-I (the original model of
 * Frisch, Hasslacher and Pomeau: head-on and symmetric three-body collisions
 * only; a rest particle, if present, is a spectator that never changes),
 * 3 = FHP-III (above). */
ORACLE_EXPORT void oracle_build_table_rules(int rules, int chirality, uint8_t table[256]) {
    for (int b = 0; b < 256; ++b) {
        int moving = b & 0x3F;
        int rest = (b >> REST_BIT) & 1;
        int out = b;
        if (b & (1 << SOLID_BIT)) {
            /* Boundary node (R-solid): every moving particle reverses,
             * i <-> i+3; the rest bit and the solid flag are kept. */
            int reflected = 0;
            for (int i = 0; i < 6; ++i)
                if (moving & dir_bit(i)) reflected |= dir_bit(i + 3);
            out = (b & 0xC0) | reflected;
        } else if (rules == 3) {
            out = fhp3_scatter(b, chirality);
        } else {
            int done = 0;
            /* Two-body head-on: exactly the pair {i, i+3} moving (rest
             * particle, if any, is a spectator).  Chirality 0 rotates the
             * pair by +60 degrees, chirality 1 by -60 degrees. */
            for (int i = 0; i < 3 && !done; ++i) {
                if (moving == (dir_bit(i) | dir_bit(i + 3))) {
                    int turned = chirality == 0 ? (dir_bit(i + 1) | dir_bit(i + 4))
                                                : (dir_bit(i - 1) | dir_bit(i + 2));
                    out = (b & 0xC0) | turned;
                    done = 1;
                }
            }
            /* Three-body symmetric: {0,2,4} <-> {1,3,5}, spectator rest kept. */
            if (!done) {
                int even = dir_bit(0) | dir_bit(2) | dir_bit(4);
                int odd = dir_bit(1) | dir_bit(3) | dir_bit(5);
                if (moving == even) { out = (b & 0xC0) | odd; done = 1; }
                else if (moving == odd) { out = (b & 0xC0) | even; done = 1; }
            }
            /* Rest-particle collisions (FHP-II only): a rest particle plus
             * one moving particle i become two moving particles i-1 and i+1,
             * and back. */
            for (int i = 0; i < 6 && !done && rules == 2; ++i) {
                int pair = dir_bit(i - 1) | dir_bit(i + 1);
                if (rest && moving == dir_bit(i)) {
                    out = pair;                       /* rest bit cleared */
                    done = 1;
                } else if (!rest && moving == pair) {
                    out = (1 << REST_BIT) | dir_bit(i);
                    done = 1;
                }
            }
        }
        table[b] = (uint8_t)out;
    }
}

ORACLE_EXPORT void oracle_build_table(int chirality, uint8_t table[256]) {
    oracle_build_table_rules(2, chirality, table);
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry (R-map).                                                 */
/* ------------------------------------------------------------------------ */
/* Neighbour of (x, y) along c_i on the W x H periodic array whose odd rows
 * are shifted right by half a lattice constant. */
static void neighbour(int W, int H, int x, int y, int i, int* nx, int* ny) {
    int odd = y & 1;
    int dx = 0, dy = 0;
    switch (i) {
        case 0: dx = odd - 1; dy = -1; break;  /* SW */
        case 1: dx = odd;     dy = -1; break;  /* SE */
        case 2: dx = 1;       dy = 0;  break;  /* E  */
        case 3: dx = odd;     dy = 1;  break;  /* NE */
        case 4: dx = odd - 1; dy = 1;  break;  /* NW */
        case 5: dx = -1;      dy = 0;  break;  /* W  */
    }
    *nx = ((x + dx) % W + W) % W;
    *ny = ((y + dy) % H + H) % H;
}

ORACLE_EXPORT void oracle_neighbour(int W, int H, int x, int y, int i, int* nx, int* ny) {
    neighbour(W, H, x, y, i, nx, ny);
}

/* ------------------------------------------------------------------------ */
/* Forcing thresholds (R-force).                                             */
/* p is quantised to P = round(p * 2^32).  S_0 = 2^32 and                    */
/* S_g = floor(S_{g-1} * (2^32 - P) / 2^32) approximate 2^32 (1-p)^g, the    */
/* chance, in units of 2^-32, that none of g candidates is forced;           */
/* Q_g = 2^32 - S_g.                                                         */
/* ------------------------------------------------------------------------ */
ORACLE_EXPORT void oracle_forcing_thresholds(double p, uint64_t q[33]) {
    const uint64_t one = (uint64_t)1 << 32;
    double scaled = p * 4294967296.0;
    uint64_t P;
    if (!(scaled > 0.0)) P = 0;                 /* also catches NaN */
    else if (scaled >= 4294967296.0) P = one;
    else {
        /* round half to even, written out with integer parts */
        uint64_t fl = (uint64_t)scaled;
        double frac = scaled - (double)fl;
        if (frac > 0.5 || (frac == 0.5 && (fl & 1))) fl += 1;
        P = fl;
    }
    uint64_t S = one;
    q[0] = 0;
    for (int g = 1; g <= 32; ++g) {
        S = (uint64_t)(((unsigned __int128)S * (one - P)) >> 32);
        q[g] = one - S;
    }
}

/* Forcing on one word of one row after scattering (R-force).  The
 * candidates are the fluid nodes of the word with bit 5 set and bit 2 clear,
 * taken in increasing x.  Each candidate is forced independently with
 * probability p, realised by geometric skipping: a uniform u picks the first
 * forced candidate among the remaining ones (G = least g with u < Q_g), a new
 * uniform is drawn after every forced candidate.  Draw d of the word comes
 * from stream 1 + d.  Returns the number of forced nodes. */
static int force_word(uint8_t* row, int w, uint64_t seed, uint64_t t, int y,
                      const uint64_t q[33]) {
    int cand[32];
    int K = 0;
    for (int b = 0; b < 32; ++b) {
        uint8_t v = row[32 * w + b];
        int fluid = !(v & (1 << SOLID_BIT));
        if (fluid && (v & dir_bit(5)) && !(v & dir_bit(2))) cand[K++] = 32 * w + b;
    }
    int next = 0;  /* index of the first candidate not yet decided */
    int forced = 0;
    uint32_t draw = 0;
    while (next < K) {
        uint32_t u = rng_word(seed, t, y, w, 1u + draw);
        int remaining = K - next;
        if ((uint64_t)u >= q[remaining]) break;  /* none of the rest forced */
        int g = 1;
        while (!((uint64_t)u < q[g])) ++g;
        int x = cand[next + g - 1];
        row[x] = (uint8_t)((row[x] & ~dir_bit(5)) | dir_bit(2));
        ++forced;
        next += g;
        ++draw;
    }
    return forced;
}

/* ------------------------------------------------------------------------ */
/* One time step (R-order): S_{t+1} = Force_t(Scatter_t(Move(S_t))).         */
/* in and out are H x W bytes, row-major; they must not overlap.             */
/* ------------------------------------------------------------------------ */
/* Row y of the array is row (row_base + y) mod Hg of the lattice: that row
 * keys the random words (for a whole lattice row_base = 0 and Hg = H).       */
static int64_t step_once(int W, int H, const uint8_t* in, uint8_t* out, uint64_t seed,
                         uint64_t t, const uint64_t q[33], int force_on,
                         const uint8_t table[2][256], int64_t row_base, int Hg) {
    int64_t events = 0;
#pragma omp parallel for schedule(static) reduction(+ : events)
    for (int y = 0; y < H; ++y) {
        uint8_t* orow = out + (size_t)y * W;
        const int gy = (int)((((row_base + y) % Hg) + Hg) % Hg);
        uint32_t chi_word = 0;
        for (int x = 0; x < W; ++x) {
            /* Motion: the particle moving along c_i that arrives at (x, y)
             * left the neighbour in direction c_{i+3} one step earlier. */
            uint8_t here = in[(size_t)y * W + x];
            int b = here & ((1 << REST_BIT) | (1 << SOLID_BIT));
            for (int i = 0; i < 6; ++i) {
                int sx, sy;
                neighbour(W, H, x, y, (i + 3) % 6, &sx, &sy);
                b |= in[(size_t)sy * W + sx] & dir_bit(i);
            }
            /* Scattering with this node's chirality bit (stream 0). */
            if ((x & 31) == 0) chi_word = rng_word(seed, t, gy, x >> 5, 0u);
            int chi = (chi_word >> (x & 31)) & 1;
            orow[x] = table[chi][b];
        }
        if (force_on)
            for (int w = 0; w < W / 32; ++w) events += force_word(orow, w, seed, t, gy, q);
    }
    return events;
}

static int64_t run_rows(int W, int H, uint8_t* state, uint8_t* scratch, uint64_t seed, uint64_t t0, int64_t n,
                        double p, int64_t row_base, int Hg, int rules);

/* Advance `state` (H x W bytes) by n steps starting at step t0.  `scratch`
 * must hold H x W bytes.  Returns the total number of forcing events. */
ORACLE_EXPORT int64_t oracle_run(int W, int H, uint8_t* state, uint8_t* scratch, uint64_t seed,
                                 uint64_t t0, int64_t n, double p) {
    return run_rows(W, H, state, scratch, seed, t0, n, p, 0, H, 2);
}

/* oracle_run with the rule set chosen (1 = FHP-I, 2 = FHP-II). */
ORACLE_EXPORT int64_t oracle_run_rules(int W, int H, uint8_t* state, uint8_t* scratch, uint64_t seed, uint64_t t0,
                                       int64_t n, double p, int rules) {
    if (rules < 1 || rules > 3) return -1;
    return run_rows(W, H, state, scratch, seed, t0, n, p, 0, H, rules);
}

/* A strip of a larger lattice, for the row-strip decomposition across
 * devices (the paper's multi-GPU runs, Table 1): `state` holds H rows, row y
 * being row (row_base + y) mod Hg of a W x Hg lattice, and is advanced n steps
 * as if periodic in its own H rows.  Rows within n rows of either edge of
 * the array are therefore not those of the lattice; the others are exact when
 * the array's edge rows held the lattice's rows at the start.  row_base must
 * be even (so that the half-cell shift of odd rows is the lattice's), H even. */
ORACLE_EXPORT int64_t oracle_run_rows(int W, int H, uint8_t* state, uint8_t* scratch, uint64_t seed, uint64_t t0,
                                      int64_t n, double p, int64_t row_base, int Hg) {
    if ((row_base & 1) || (H & 1) || Hg < 2) return -1;
    return run_rows(W, H, state, scratch, seed, t0, n, p, row_base, Hg, 2);
}

static int64_t run_rows(int W, int H, uint8_t* state, uint8_t* scratch, uint64_t seed, uint64_t t0, int64_t n,
                        double p, int64_t row_base, int Hg, int rules) {
    uint8_t table[2][256];
    oracle_build_table_rules(rules, 0, table[0]);
    oracle_build_table_rules(rules, 1, table[1]);
    uint64_t q[33];
    oracle_forcing_thresholds(p, q);
    int force_on = q[32] != 0;
    int64_t events = 0;
    uint8_t* a = state;
    uint8_t* b = scratch;
    for (int64_t k = 0; k < n; ++k) {
        events += step_once(W, H, a, b, seed, t0 + (uint64_t)k, q, force_on, table, row_base, Hg);
        uint8_t* tmp = a; a = b; b = tmp;
    }
    if (a != state) memcpy(state, a, (size_t)W * H);
    return events;
}

/* ------------------------------------------------------------------------ */
/* Coarse-graining over B x B blocks (R-cg).                                 */
/* counts[(by * (W/B) + bx) * 9 + k]: k = 0..6 number of fluid nodes of the  */
/* block with bit k set, k = 7 number of fluid nodes, k = 8 particle mass.   */
/* rho = mass / fluid; ux = jx2 / (2 mass); uy = (sqrt(3)/2) jy / mass with  */
/* jx2 = sum n_i 2cos(theta_i), jy = sum n_i sgn(sin(theta_i)).              */
/* ------------------------------------------------------------------------ */
ORACLE_EXPORT void oracle_coarse_grain(int W, int H, const uint8_t* state, int B,
                                       int32_t* counts, double* rho, double* ux,
                                       double* uy) {
    int nbx = W / B, nby = H / B;
    /* 2 cos(theta_i) and the sign of sin(theta_i) for theta_i = (i-2)*60 deg. */
    const int two_cos[6] = {-1, 1, 2, 1, -1, -2};
    const int sgn_sin[6] = {-1, -1, 0, 1, 1, 0};
    for (int by = 0; by < nby; ++by) {
        for (int bx = 0; bx < nbx; ++bx) {
            int64_t n[7] = {0, 0, 0, 0, 0, 0, 0};
            int64_t fluid = 0;
            for (int y = by * B; y < (by + 1) * B; ++y) {
                for (int x = bx * B; x < (bx + 1) * B; ++x) {
                    uint8_t v = state[(size_t)y * W + x];
                    if (v & (1 << SOLID_BIT)) continue;
                    ++fluid;
                    for (int k = 0; k < 7; ++k) n[k] += (v >> k) & 1;
                }
            }
            int64_t mass = 0, jx2 = 0, jy = 0;
            for (int k = 0; k < 7; ++k) mass += n[k];
            for (int i = 0; i < 6; ++i) { jx2 += two_cos[i] * n[i]; jy += sgn_sin[i] * n[i]; }
            size_t cell = (size_t)by * nbx + bx;
            for (int k = 0; k < 7; ++k) counts[cell * 9 + k] = (int32_t)n[k];
            counts[cell * 9 + 7] = (int32_t)fluid;
            counts[cell * 9 + 8] = (int32_t)mass;
            double half_sqrt3 = 0.8660254037844386;  /* sqrt(3)/2 rounded to double */
            rho[cell] = fluid ? (double)mass / (double)fluid : 0.0;
            ux[cell] = mass ? (double)jx2 / (2.0 * (double)mass) : 0.0;
            uy[cell] = mass ? half_sqrt3 * (double)jy / (double)mass : 0.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Random initial state (reading R-init2, used when the state is generated  */
/* rather than uploaded): bit b (0..6) of fluid node x in row y is set iff  */
/* its 16-bit uniform is below P = round-half-even(rho * 2^16).  The        */
/* uniforms of word w = x / 32 and bit b come from the Philox blocks with    */
/* counter (w, y, b, j), j = 0..3, under the key (seed_lo ^ 0x9E3779B9,      */
/* seed_hi ^ 0x7F4A7C15) -- a key of its own, so these draws never meet the  */
/* step's.  Node i = x mod 32 of the word takes block j = i / 8, output      */
/* word (i mod 8) / 2, half i mod 2 (low 16 bits for even i).  Solid nodes   */
/* (mask nonzero) get bit 7 only.                                            */
/* ------------------------------------------------------------------------ */
ORACLE_EXPORT void oracle_init_random(int W, int H, uint64_t seed, double rho, const uint8_t* solid_mask,
                                      uint8_t* state) {
    double scaled = rho * 65536.0;
    uint32_t P;
    if (!(scaled > 0.0)) P = 0;
    else if (scaled >= 65536.0) P = 65536;
    else {
        uint32_t fl = (uint32_t)scaled;
        double frac = scaled - (double)fl;
        if (frac > 0.5 || (frac == 0.5 && (fl & 1))) fl += 1;
        P = fl;
    }
    const uint32_t key[2] = {(uint32_t)seed ^ 0x9E3779B9u, (uint32_t)(seed >> 32) ^ 0x7F4A7C15u};
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            uint8_t v = 0;
            if (solid_mask && solid_mask[(size_t)y * W + x]) {
                v = 0x80;
            } else {
                int i = x & 31;
                for (int b = 0; b < 7; ++b) {
                    uint32_t ctr[4] = {(uint32_t)(x >> 5), (uint32_t)y, (uint32_t)b, (uint32_t)(i >> 3)};
                    uint32_t out[4];
                    oracle_philox4x32_10(ctr, key, out);
                    uint32_t word = out[(i & 7) >> 1];
                    uint32_t u = (i & 1) ? (word >> 16) : (word & 0xFFFFu);
                    if (u < P) v |= (uint8_t)(1u << b);
                }
            }
            state[(size_t)y * W + x] = v;
        }
    }
}

ORACLE_EXPORT void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

ORACLE_EXPORT int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
