"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test states what fixes the expected value: a worked example of the paper
(tests/golden), a closed form, a conservation law, a lattice symmetry, a
library generator, or a brute-force model written from geometry
(tests/naive_fhp.py).
"""
from __future__ import annotations

import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

import naive_fhp as naive

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.txt")

# Geometry written independently of the oracle: unit velocities at (i-2)*60 deg.
VEL = [(math.cos((i - 2) * math.pi / 3), math.sin((i - 2) * math.pi / 3)) for i in range(6)]


def mass(b: int) -> int:
    return bin(b & 0x7F).count("1")


def mom(b: int):
    return (sum(VEL[i][0] for i in range(6) if b >> i & 1),
            sum(VEL[i][1] for i in range(6) if b >> i & 1))


def golden_lines():
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


# --------------------------------------------------------------------------
# Paper's worked examples (Section 2)
# --------------------------------------------------------------------------

def test_golden_decode():
    """Section 2, Fig. 1 and the 00100100 example: bit meaning of a node byte."""
    seen = 0
    for parts in golden_lines():
        if parts[0] != "decode":
            continue
        b = int(parts[1], 2)
        fields = dict(kv.split("=") for kv in parts[2:])
        moving = [int(v) for v in fields["moving"].split(",") if v]
        assert [i for i in range(6) if b >> i & 1] == moving
        assert (b >> 6 & 1) == int(fields["rest"])
        assert (b >> 7 & 1) == int(fields["solid"])
        seen += 1
    assert seen == 4
    # bits 2 and 5 are a horizontal opposite pair (forcing reverses a horizontal mover)
    assert VEL[2][1] == pytest.approx(0.0, abs=1e-12) and VEL[5][1] == pytest.approx(0.0, abs=1e-12)
    assert VEL[2][0] == pytest.approx(-VEL[5][0])


def _single_node_step(oracle_mod, byte_after_motion: int, p: float):
    """Place particles so that after the motion step node (40, 2) of a 64 x 6
    lattice holds `byte_after_motion` and no other node holds anything that
    collides; return that node after one step with forcing probability p."""
    W, H, x, y = 64, 6, 40, 2
    s = np.zeros((H, W), dtype=np.uint8)
    s[y, x] = byte_after_motion & 0x40          # rest particle stays put
    for i in range(6):
        if byte_after_motion >> i & 1:
            # the particle that arrives along c_i starts one hop behind it
            sx, sy = naive.push_target(W, H, x, y, (i + 3) % 6)
            s[sy, sx] |= 1 << i
    out, events = oracle_mod.run(s, seed=99, t0=0, n=1, p=p)
    return int(out[y, x]), events


def test_golden_forcing(oracle_mod):
    """Section 2, forcing paragraph: (..1..0..) -> (..0..1..) when it fires."""
    for parts in golden_lines():
        if parts[0] == "force":
            b, expect = int(parts[1], 2), int(parts[2], 2)
            got, ev = _single_node_step(oracle_mod, b, p=1.0)
            assert got == expect and ev == 1, (parts, got)
            got0, ev0 = _single_node_step(oracle_mod, b, p=0.0)
            assert got0 == b and ev0 == 0
        elif parts[0] == "noforce":
            b = int(parts[1], 2)
            got, ev = _single_node_step(oracle_mod, b, p=1.0)
            assert got == b and ev == 0, (parts, got)


# --------------------------------------------------------------------------
# Scattering table (Section 2, Fig. 2; reading R-rules, R-solid)
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def tables(oracle_mod):
    return [oracle_mod.table(0), oracle_mod.table(1)]


def test_table_conserves_mass_and_momentum(tables):
    for chi in (0, 1):
        t = tables[chi]
        for b in range(128):
            o = int(t[b])
            assert o < 128, "fluid node must stay fluid"
            assert mass(o) == mass(b)
            mb, mo = mom(b), mom(o)
            assert mo[0] == pytest.approx(mb[0], abs=1e-9)
            assert mo[1] == pytest.approx(mb[1], abs=1e-9)


def test_table_solid_bounce_back(tables):
    for chi in (0, 1):
        t = tables[chi]
        for b in range(128, 256):
            o = int(t[b])
            assert o & 0x80 and (o & 0x40) == (b & 0x40)
            assert mass(o) == mass(b)
            mb, mo = mom(b), mom(o)
            assert mo[0] == pytest.approx(-mb[0], abs=1e-9)
            assert mo[1] == pytest.approx(-mb[1], abs=1e-9)
            # bounce-back is an involution
            assert int(t[o]) == b


def _rot(b: int, k: int) -> int:
    """Rotate the moving bits of b by k * 60 degrees (geometry: c_i -> c_{i+k})."""
    out = b & 0xC0
    for i in range(6):
        if b >> i & 1:
            out |= 1 << ((i + k) % 6)
    return out


def _reflect(b: int) -> int:
    """Mirror in the x axis: angle theta -> -theta, i.e. (i-2) -> -(i-2)."""
    out = b & 0xC0
    for i in range(6):
        if b >> i & 1:
            out |= 1 << ((4 - i) % 6)
    return out


def test_table_rotation_covariance(tables):
    for chi in (0, 1):
        t = tables[chi]
        for b in range(256):
            for k in range(6):
                assert int(t[_rot(b, k)]) == _rot(int(t[b]), k)


def test_table_reflection_swaps_chirality(tables):
    # check the reflection is the geometric mirror first
    for i in range(6):
        j = [k for k in range(6) if _reflect(1 << i) == 1 << k][0]
        assert VEL[j][0] == pytest.approx(VEL[i][0]) and VEL[j][1] == pytest.approx(-VEL[i][1])
    for b in range(256):
        assert int(tables[1][_reflect(b)]) == _reflect(int(tables[0][b]))


def test_table_chiralities_are_inverse(tables):
    """Turning a head-on pair by +60 then by -60 degrees gives it back; the
    other rules are involutions, so T_1(T_0(s)) = s for every fluid state."""
    for b in range(128):
        assert int(tables[1][int(tables[0][b])]) == b


def test_table_rule_examples(tables):
    t0, t1 = tables
    # head-on SW+NE -> SE+NW (chi 0, +60 deg) or E+W (chi 1, -60 deg)
    assert t0[0b0001001] == 0b0010010 and t1[0b0001001] == 0b0100100
    # with a spectator rest particle (FHP-II)
    assert t0[0b1001001] == 0b1010010
    # symmetric triples swap
    assert t0[0b0010101] == 0b0101010 and t1[0b0101010] == 0b0010101
    # rest + E  <->  SE + NE (the two movers whose velocities add up to c_E)
    assert t0[0b1000100] == 0b0001010 and t0[0b0001010] == 0b1000100
    # everything else that is not in a rule class is left alone
    assert t0[0b0000100] == 0b0000100 and t0[0b0110000] == 0b0110000
    assert t0[0] == 0 and t0[0x7F] == 0x7F
    # 3 head-on pairs x (rest or not) + 2 triples x 2 + 6 x 2 rest rules
    for t in tables:
        assert sum(int(t[b]) != b for b in range(128)) == 6 + 4 + 12


def test_table_matches_geometric_rules(tables):
    """Brute force over all 256 bytes x 2 chiralities against the rules
    phrased as rotations of the velocity set (tests/naive_fhp.py)."""
    for chi in (0, 1):
        for b in range(256):
            assert int(tables[chi][b]) == naive.scatter(b, chi), (chi, bin(b))


# --------------------------------------------------------------------------
# Motion (Section 2, Fig. 3; reading R-map)
# --------------------------------------------------------------------------

def test_neighbours_are_unit_hops(oracle_mod):
    W, H = 64, 8
    for y in range(H):
        for x in (0, 1, 31, 32, 63):
            for i in range(6):
                nx, ny = oracle_mod.neighbour(W, H, x, y, i)
                assert (nx, ny) == naive.push_target(W, H, x, y, i)


@pytest.mark.parametrize("W,H", [(64, 8), (96, 6), (32, 2)])
def test_free_streaming_closed_form(oracle_mod, W, H):
    """A lone particle moves one lattice vector per step; its physical
    displacement after n steps is n * c_i (mod the periodic box)."""
    for i in range(6):
        for y0 in (0, 1):
            x0 = 5
            s = np.zeros((H, W), dtype=np.uint8)
            s[y0, x0] = 1 << i
            n = 7
            out, _ = oracle_mod.run(s, seed=1, t0=0, n=n, p=0.0)
            ys, xs = np.nonzero(out)
            assert len(xs) == 1 and out[ys[0], xs[0]] == 1 << i
            px0, py0 = naive.position(x0, y0)
            px, py = naive.position(int(xs[0]), int(ys[0]))
            dx = px - px0 - n * naive.VEL[i][0]
            dy = py - py0 - n * naive.VEL[i][1]
            # displacement must equal n c_i up to whole periods of the box
            ry = dy / (math.sqrt(3) / 2)
            assert abs(ry - round(ry)) < 1e-9 and round(ry) % H == 0
            # a vertical period of H rows (H even) keeps the row parity
            assert abs(dx - round(dx)) < 1e-9 and round(dx) % W == 0


@pytest.mark.parametrize("W,H", [(64, 8), (96, 6)])
def test_free_streaming_period(oracle_mod, W, H):
    """Horizontal movers return after W steps; diagonal movers climb one row
    and half a column per step, so they return after H*W/gcd(W, H/2) steps."""
    for i in range(6):
        s = np.zeros((H, W), dtype=np.uint8)
        s[1, 3] = 1 << i
        period = W if i in (2, 5) else H * W // math.gcd(W, H // 2)
        out, _ = oracle_mod.run(s, seed=3, t0=0, n=period, p=0.0)
        assert np.array_equal(out, s)
        out2, _ = oracle_mod.run(s, seed=3, t0=0, n=period - 1, p=0.0)
        assert not np.array_equal(out2, s)


# --------------------------------------------------------------------------
# Random numbers (reading R-rng): Philox4x32-10 against cuRAND's host generator
# --------------------------------------------------------------------------

def _curand():
    for name in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def _curand_philox_host(lib, seed: int, n: int, offset: int = 0) -> np.ndarray:
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        if offset:
            assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
        return out
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 0x0123456789ABCDEF, 0xFFFFFFFF00000001])
def test_philox_matches_curand_host(oracle_mod, seed):
    """cuRAND's host Philox4_32_10 generator emits block i = Philox(counter
    (i >> 16, 0, i & 0xffff, 0), key = seed); compare a spread of blocks."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    nblocks = 65536 + 64
    ref = _curand_philox_host(lib, seed, 4 * nblocks)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in list(range(0, 64)) + list(range(65536 - 8, nblocks)) + [12345, 40000]:
        ctr = [i >> 16, 0, i & 0xFFFF, 0]
        assert np.array_equal(oracle_mod.philox4x32_10(ctr, key), ref[4 * i:4 * i + 4]), i
    # a large first counter word through the generator offset
    off_blocks = (1234 << 16)
    ref2 = _curand_philox_host(lib, seed, 8, offset=4 * off_blocks)
    assert np.array_equal(oracle_mod.philox4x32_10([1234, 0, 0, 0], key), ref2[:4])


def test_rng_word_layout_and_balance(oracle_mod):
    seed = 0xDEADBEEFCAFEF00D
    key = [seed & 0xFFFFFFFF, seed >> 32]
    t = (5 << 32) + 77
    blk = oracle_mod.philox4x32_10([9, 3, t & 0xFFFFFFFF, 2 | (5 << 16)], key)
    for j in range(4):
        assert oracle_mod.rng_word(seed, t, 3, 36 + j, 2) == int(blk[j])
    # bit balance over many words: each bit position near 1/2
    words = np.array([oracle_mod.rng_word(seed, 11, y, w, 0) for y in range(64) for w in range(64)],
                     dtype=np.uint64)
    bits = ((words[:, None] >> np.arange(32, dtype=np.uint64)) & 1).astype(np.float64)
    n = len(words)
    per_bit = bits.mean(axis=0)
    assert np.all(np.abs(per_bit - 0.5) < 5 * 0.5 / math.sqrt(n))


# --------------------------------------------------------------------------
# Forcing sampler (reading R-force)
# --------------------------------------------------------------------------

def test_forcing_thresholds_closed_form(oracle_mod):
    for p in (0.0, 1e-3, 5e-4, 0.25, 0.5, 1.0):
        q = oracle_mod.forcing_thresholds(p)
        assert [int(v) for v in q] == naive.thresholds(p)
        for g in range(1, 33):
            exact = (1 << 32) * (1 - (1 - p) ** g)
            assert abs(int(q[g]) - exact) <= g + 1
    assert int(oracle_mod.forcing_thresholds(1.0)[1]) == 1 << 32
    assert int(oracle_mod.forcing_thresholds(0.0)[32]) == 0


def test_forcing_threshold_growth_bound():
    """Q_K <= K (P + 1) for the integer recurrence (P = round(p 2^32)): each
    floor step loses less than one unit, so Q_g - Q_{g-1} <= P + 1.  The GPU's
    per-word pre-check rejects a word when u >= K (P + 1) on this bound, so a
    violation would drop forcing events; checked here on the recurrence
    itself for many p, including the rounding edges and p = 1."""
    rng = np.random.Generator(np.random.PCG64(77))
    ps = [0.0, 1.0, 1e-3, 5e-4, 0.5, 2.0 ** -32, 0.5 * 2.0 ** -32, 1.5 * 2.0 ** -32, 1 - 2.0 ** -32]
    ps += list(rng.uniform(0, 1, 200)) + list(10.0 ** rng.uniform(-9, -1, 200))
    for p in ps:
        q = naive.thresholds(p)
        P = q[1]            # Q_1 = 2^32 - floor(2^32 (2^32 - P) / 2^32) = P
        for K in range(33):
            assert q[K] <= K * (P + 1), (p, K)


def test_forcing_p1_forces_every_candidate(oracle_mod):
    """With p = 1 no fluid node is left with bit 5 set and bit 2 clear."""
    import workloads
    s = workloads.bernoulli_lattice(128, 16, 0.4, 5, workloads.channel_walls(128, 16))
    out, ev = oracle_mod.run(s, seed=5, t0=0, n=1, p=1.0)
    fluid = (out & 0x80) == 0
    assert not np.any(fluid & ((out & 0x20) != 0) & ((out & 0x04) == 0))
    out0, ev0 = oracle_mod.run(s, seed=5, t0=0, n=1, p=0.0)
    cand = ((out0 & 0x80) == 0) & ((out0 & 0x20) != 0) & ((out0 & 0x04) == 0)
    assert ev == int(cand.sum())
    assert np.array_equal(out0 ^ out, np.where(cand, 0x24, 0).astype(np.uint8))


def test_forcing_binomial_statistics(oracle_mod):
    """Forced nodes among the candidates of one word are Binomial(K, p):
    check the mean rate, and that position within the word does not matter."""
    import workloads
    p = 0.2
    W, H = 1024, 64
    s = workloads.bernoulli_lattice(W, H, 0.3, 17)
    tot_c = tot_f = 0
    first_half = second_half = 0
    for t in range(4):
        out0, _ = oracle_mod.run(s, seed=8, t0=t, n=1, p=0.0)
        out1, ev = oracle_mod.run(s, seed=8, t0=t, n=1, p=p)
        cand = ((out0 & 0x80) == 0) & ((out0 & 0x20) != 0) & ((out0 & 0x04) == 0)
        forced = (out0 != out1)
        assert not np.any(forced & ~cand)
        tot_c += int(cand.sum())
        tot_f += int(forced.sum())
        assert int(forced.sum()) == ev
        xs = np.arange(W) % 32
        first_half += int((forced & (xs < 16)[None, :]).sum())
        second_half += int((forced & (xs >= 16)[None, :]).sum())
    rate = tot_f / tot_c
    sd = math.sqrt(p * (1 - p) / tot_c)
    assert abs(rate - p) < 5 * sd
    # candidates are spread evenly over the word, so forced nodes must be too
    n = first_half + second_half
    assert abs(first_half - n / 2) < 5 * math.sqrt(n / 4)


# --------------------------------------------------------------------------
# Whole-step invariants and brute force
# --------------------------------------------------------------------------

def _totals(s: np.ndarray):
    m = int(sum(np.count_nonzero(s >> k & 1) for k in range(7)))
    # integer momenta: 2 cos and sign(sin) components
    two_cos = [-1, 1, 2, 1, -1, -2]
    sgn_sin = [-1, -1, 0, 1, 1, 0]
    n = [int(np.count_nonzero(s >> k & 1)) for k in range(6)]
    # these integer weights are the geometry: check them against VEL once
    for i in range(6):
        assert two_cos[i] == round(2 * VEL[i][0]) and sgn_sin[i] == int(np.sign(round(VEL[i][1], 9)))
    return m, sum(a * b for a, b in zip(two_cos, n)), sum(a * b for a, b in zip(sgn_sin, n))


def test_invariants_periodic(oracle_mod):
    import workloads
    s = workloads.bernoulli_lattice(256, 64, 0.3, 1)
    m0, jx0, jy0 = _totals(s)
    out, ev = oracle_mod.run(s, seed=1, t0=0, n=20, p=0.0)
    assert ev == 0
    assert _totals(out) == (m0, jx0, jy0)


def test_forcing_momentum_balance(oracle_mod):
    """Each forcing event turns a W mover into an E mover: jx2 grows by 4."""
    import workloads
    s = workloads.bernoulli_lattice(256, 32, 0.25, 2)
    m0, jx0, jy0 = _totals(s)
    out, ev = oracle_mod.run(s, seed=2, t0=0, n=10, p=0.01)
    assert ev > 0
    m1, jx1, jy1 = _totals(out)
    assert m1 == m0 and jy1 == jy0 and jx1 - jx0 == 4 * ev


def test_mass_conserved_with_obstacles_and_forcing(oracle_mod):
    import workloads
    W, H = 512, 128
    s = workloads.bernoulli_lattice(W, H, 0.25, 3, workloads.cylinder_mask(W, H))
    m0 = _totals(s)[0]
    out, ev = oracle_mod.run(s, seed=3, t0=0, n=30, p=5e-3)
    assert ev > 0 and _totals(out)[0] == m0
    # solid flags never change
    assert np.array_equal(out & 0x80, s & 0x80)


def test_resume_and_thread_independence(oracle_mod):
    import workloads
    W, H = 256, 32
    s = workloads.bernoulli_lattice(W, H, 0.3, 4, workloads.channel_walls(W, H))
    full, e_full = oracle_mod.run(s, seed=4, t0=10, n=12, p=0.02)
    half, e1 = oracle_mod.run(s, seed=4, t0=10, n=5, p=0.02)
    rest, e2 = oracle_mod.run(half, seed=4, t0=15, n=7, p=0.02)
    assert np.array_equal(full, rest) and e_full == e1 + e2
    nthr = oracle_mod.max_threads()
    try:
        oracle_mod.set_threads(1)
        one, _ = oracle_mod.run(s, seed=4, t0=10, n=12, p=0.02)
    finally:
        oracle_mod.set_threads(nthr)
    assert np.array_equal(one, full)


@pytest.mark.parametrize("W,H,p,obst", [(32, 2, 0.0, None), (32, 4, 0.3, "walls"),
                                         (64, 6, 0.2, "points"), (32, 8, 0.5, "points")])
def test_brute_force_naive_model(oracle_mod, W, H, p, obst):
    """Tiny lattices, several steps: the oracle equals the geometric model."""
    import workloads
    rng = np.random.Generator(np.random.PCG64(W * 1000 + H))
    solid = None
    if obst == "walls":
        solid = workloads.channel_walls(W, H)
    elif obst == "points":
        solid = workloads.random_points(W, H, 0.1, rng)
    s = workloads.bernoulli_lattice(W, H, 0.35, W + H, solid)
    seed = 777
    cur = s.copy()
    for t in range(5):
        ref = naive.step(cur, seed, t, p, oracle_mod.rng_word)
        got, _ = oracle_mod.run(cur, seed=seed, t0=t, n=1, p=p)
        assert np.array_equal(got, ref), (W, H, t)
        cur = ref


# --------------------------------------------------------------------------
# Coarse-graining (reading R-cg)
# --------------------------------------------------------------------------

def test_coarse_grain_closed_forms(oracle_mod):
    B = 32
    W, H = 96, 64
    s = np.zeros((H, W), dtype=np.uint8)
    s[0:32, 0:32] = 0x7F                 # block (0,0): all seven bits everywhere
    s[0:32, 32:64] = 1 << 3              # block (0,1): everything moving NE
    s[0:32, 64:96] = 0x80                # block (0,2): solid
    s[32:64, 0:32] = 1 << 2              # block (1,0): everything moving E
    s[32:64, 32:64] = (1 << 5) | (1 << 6)  # W mover plus rest particle
    s[40, 70] = 0x80 | 0x3F              # a solid node inside block (1,2) holding movers
    counts, rho, ux, uy = oracle_mod.coarse_grain(s, B)
    assert counts.shape == (2, 3, 9)
    assert list(counts[0, 0]) == [B * B] * 7 + [B * B, 7 * B * B]
    assert rho[0, 0] == 7.0 and ux[0, 0] == 0.0 and uy[0, 0] == 0.0
    assert counts[0, 1, 3] == B * B and counts[0, 1, 8] == B * B
    assert ux[0, 1] == pytest.approx(VEL[3][0], abs=1e-12)
    assert uy[0, 1] == pytest.approx(VEL[3][1], abs=1e-12)
    assert counts[0, 2, 7] == 0 and rho[0, 2] == 0.0 and ux[0, 2] == 0.0
    assert ux[1, 0] == pytest.approx(1.0) and uy[1, 0] == 0.0
    assert ux[1, 1] == pytest.approx(-0.5) and rho[1, 1] == 2.0
    # the solid node is not counted: block (1,2) has one fluid node fewer and no particles
    assert counts[1, 2, 7] == B * B - 1 and counts[1, 2, 8] == 0


# --------------------------------------------------------------------------
# Generated initial state (reading R-init2)
# --------------------------------------------------------------------------

def test_init_random_closed_forms_and_statistics(oracle_mod):
    W, H = 512, 64
    empty = oracle_mod.init_random(W, H, 5, 0.0)
    assert not empty.any()
    full = oracle_mod.init_random(W, H, 5, 1.0)
    assert np.all(full == 0x7F)
    mask = np.zeros((H, W), dtype=bool)
    mask[3, :] = True
    mask[10:20, 100:140] = True
    s = oracle_mod.init_random(W, H, 7, 0.3, mask)
    assert np.all(s[mask] == 0x80) and not np.any(s[~mask] & 0x80)
    # each bit set with probability round(0.3 * 65536) / 65536, independently
    fluid = s[~mask]
    p = round(0.3 * 65536) / 65536
    n = fluid.size
    sd = math.sqrt(p * (1 - p) / n)
    for b in range(7):
        assert abs(float(np.mean(fluid >> b & 1)) - p) < 5 * sd
    # pairs of bits of one node are independent: P(both) = p^2
    both = float(np.mean((fluid & 1) & (fluid >> 1 & 1)))
    assert abs(both - p * p) < 5 * math.sqrt(p * p * (1 - p * p) / n)
    # neighbouring nodes of a word are independent too
    adj = float(np.mean((s[:, 0:W:2] & 1) & (s[:, 1:W:2] & 1)))
    assert abs(adj - p * p) < 0.01
    # the uniforms are the documented Philox outputs (key transform, counter, halves)
    seed = 0x1234_5678_9ABC_DEF0
    key = [(seed & 0xFFFFFFFF) ^ 0x9E3779B9, (seed >> 32) ^ 0x7F4A7C15]
    x, y, b = 45, 6, 3
    i = x % 32
    blk = oracle_mod.philox4x32_10([x // 32, y, b, i // 8], key)
    word = int(blk[(i % 8) // 2])
    u = (word >> 16) if i % 2 else (word & 0xFFFF)
    s2 = oracle_mod.init_random(W, H, seed, 0.5)
    assert (int(s2[y, x]) >> b & 1) == (1 if u < 32768 else 0)


# ---------------------------------------------------------------------------
# FHP-I rule set (head-on and three-body collisions only; the rest particle,
# if any, is a spectator).
# ---------------------------------------------------------------------------
def test_fhp1_table_against_geometric_rules_and_invariants(oracle_mod):
    for chi in (0, 1):
        t1 = oracle_mod.table(chi, rules=1)
        t2 = oracle_mod.table(chi, rules=2)
        for b in range(256):
            out = int(t1[b])
            assert out == naive.scatter(b, chi, rules=1), (chi, bin(b))
            assert (out ^ b) & 0xC0 == 0                       # rest bit and solid flag never change
            assert bin(out).count("1") == bin(b).count("1")    # mass
            if not b & 0x80:
                assert naive.momentum([i for i in range(6) if out >> i & 1]) == pytest.approx(
                    naive.momentum([i for i in range(6) if b >> i & 1]), abs=1e-9)
        # differs from FHP-II exactly on the twelve rest-particle patterns
        diff = [b for b in range(256) if t1[b] != t2[b]]
        assert len(diff) == 12 and all(b & 0x80 == 0 for b in diff)
        assert sorted(diff) == sorted([0x40 | (1 << i) for i in range(6)]
                                      + [(1 << ((i + 5) % 6)) | (1 << ((i + 1) % 6)) for i in range(6)])
    # the two chiralities are inverse permutations
    t0, t1_ = oracle_mod.table(0, rules=1), oracle_mod.table(1, rules=1)
    assert all(int(t1_[int(t0[b])]) == b for b in range(256))


@pytest.mark.parametrize("W,H,p", [(32, 4, 0.0), (64, 6, 0.2)])
def test_fhp1_brute_force_naive_model(oracle_mod, W, H, p):
    rng = np.random.Generator(np.random.PCG64(17))
    s = rng.integers(0, 128, size=(H, W), dtype=np.uint8)
    s[0, :5] |= 0x80
    seed, cur = 5, s.copy()
    orig_scatter = naive.scatter
    try:
        naive.scatter = lambda b, c, rules=1: orig_scatter(b, c, rules=1)
        for t in range(4):
            cur = naive.step(cur, seed, t, p, oracle_mod.rng_word)
    finally:
        naive.scatter = orig_scatter
    got, _ = oracle_mod.run(s, seed, 0, 4, p, rules=1)
    assert np.array_equal(got, cur)
    assert int(np.count_nonzero(got & 0x40)) == int(np.count_nonzero(s & 0x40))  # rest particles never move or change


# ---------------------------------------------------------------------------
# FHP-III rule set (reading R-fhp3: collision-saturated; every fluid state
# that shares its mass and momentum with another state changes).
# ---------------------------------------------------------------------------
def _turn(b, by):
    out = b & 0xC0
    for i in range(6):
        if b >> i & 1:
            out |= 1 << ((i + by) % 6)
    return out


def test_fhp3_table_invariants_and_symmetries(oracle_mod):
    t3 = [oracle_mod.table(c, rules=3) for c in (0, 1)]
    t2 = [oracle_mod.table(c, rules=2) for c in (0, 1)]
    for chi in (0, 1):
        t = t3[chi]
        assert sorted(int(v) for v in t) == list(range(256))             # a permutation
        for b in range(256):
            o = int(t[b])
            assert o == naive.scatter(b, chi, rules=3), (chi, b)         # the geometric model
            assert int(t3[1 - chi][o]) == b                              # chiralities are inverse
            if b & 0x80:
                assert o == int(t2[chi][b])                               # bounce-back unchanged
                continue
            assert o < 128 and mass(o) == mass(b)
            assert mom(o) == pytest.approx(mom(b), abs=1e-9)
            assert int(t[127 - b]) == 127 - o                            # particle-hole duality
            for by in range(6):                                           # rotation covariance
                assert int(t[_turn(b, by)]) == _turn(o, by)
            if t2[chi][b] != b:                                           # every FHP-II collision kept
                assert o == int(t2[chi][b]), (chi, b)
        # saturation: a state changes iff another state has its mass and momentum
        for b in range(128):
            shared = any(mass(c) == mass(b) and mom(c) == pytest.approx(mom(b), abs=1e-9)
                         for c in range(128) if c != b)
            assert (int(t[b]) != b) == shared, b
        assert sum(int(t[b]) != b for b in range(128)) == 76


def test_fhp3_rule_examples(oracle_mod):
    t0, t1 = oracle_mod.table(0, rules=3), oracle_mod.table(1, rules=3)
    E, NE, NW, W, SW, SE, R = 1 << 2, 1 << 3, 1 << 4, 1 << 5, 1 << 0, 1 << 1, 1 << 6
    # two head-on pairs turn like one (FHP-II leaves them alone)
    assert t0[SW | NE | SE | NW] == SE | NW | E | W
    assert t1[SW | NE | SE | NW] == SW | NE | E | W
    # five movers <-> rest + four movers of the same momentum
    assert t0[SW | SE | E | NE | NW] == R | SE | E | NE | W
    assert t1[R | SE | E | NE | W] == SW | SE | E | NE | NW
    # mover E with a spectator pair: the pair turns, then the rest particle appears
    assert t0[E | SW | NE] == E | SE | NW
    assert t0[E | SE | NW] == R | SE | NE
    assert t0[R | SE | NE] == E | SW | NE
    assert t1[E | SW | NE] == R | SE | NE
    # states without a partner stay (rest + E is not one: it pairs with SE + NE)
    assert t0[R | E] == SE | NE and t1[R | E] == SE | NE
    for b in (0, R, E, SW | SE | E | NE | NW | W, 0x7F, E | NE):
        assert t0[b] == b and t1[b] == b


@pytest.mark.parametrize("W,H,p", [(32, 4, 0.0), (64, 6, 0.2)])
def test_fhp3_brute_force_naive_model(oracle_mod, W, H, p):
    rng = np.random.Generator(np.random.PCG64(23))
    s = rng.integers(0, 128, size=(H, W), dtype=np.uint8)
    s[1, 3:9] |= 0x80
    seed, cur = 8, s.copy()
    orig_scatter = naive.scatter
    try:
        naive.scatter = lambda b, c, rules=3: orig_scatter(b, c, rules=3)
        for t in range(4):
            cur = naive.step(cur, seed, t, p, oracle_mod.rng_word)
    finally:
        naive.scatter = orig_scatter
    got, _ = oracle_mod.run(s, seed, 0, 4, p, rules=3)
    assert np.array_equal(got, cur)
