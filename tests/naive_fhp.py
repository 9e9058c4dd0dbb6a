"""A second, deliberately naive FHP model used only to pin the C oracle.

It is written from the geometry of the triangular lattice rather than from
bit indices, so that a wrong index, sign or offset in the oracle shows up as a
disagreement:

* node positions are physical points (x + (y odd)/2, y * sqrt(3)/2)
  (arXiv:1208.2428, Section 2, Fig. 3: odd rows shifted by half a cell);
* velocities are unit vectors at angle (i-2)*60 degrees (reading R-dir);
* motion PUSHES each particle to the node nearest to position + c_i
  (the oracle pulls from the opposite neighbour);
* scattering is phrased as rotations of the velocity set: a head-on pair turns
  by +-60 degrees (sign from the chirality bit), a symmetric triple turns by
  60 degrees, a rest particle plus one mover splits into the two movers whose
  velocities sum to the mover's, and back (reading R-rules);
* forcing walks the candidates one by one (the oracle jumps to the next forced
  candidate) with the same uniforms, thresholds written as exact fractions.

Pure Python loops; only for lattices of a few hundred nodes.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

ANGLES = [(i - 2) * math.pi / 3 for i in range(6)]
VEL = [(math.cos(a), math.sin(a)) for a in ANGLES]


def direction_of(vx: float, vy: float) -> int:
    """Index of the lattice velocity equal to (vx, vy)."""
    for i, (cx, cy) in enumerate(VEL):
        if abs(cx - vx) < 1e-9 and abs(cy - vy) < 1e-9:
            return i
    raise ValueError("not a lattice velocity")


def rotate(i: int, turns: int) -> int:
    """Direction obtained by rotating c_i by turns * 60 degrees (geometrically)."""
    a = ANGLES[i] + turns * math.pi / 3
    return direction_of(math.cos(a), math.sin(a))


def position(x: int, y: int):
    return x + 0.5 * (y & 1), y * math.sqrt(3) / 2


def push_target(W: int, H: int, x: int, y: int, i: int):
    px, py = position(x, y)
    qx, qy = px + VEL[i][0], py + VEL[i][1]
    ty = round(qy / (math.sqrt(3) / 2))
    tx = round(qx - 0.5 * (ty & 1))
    return tx % W, ty % H


def momentum(dirs) -> tuple[float, float]:
    return (sum(VEL[i][0] for i in dirs), sum(VEL[i][1] for i in dirs))


def _byte(dirs, rest) -> int:
    return (0x40 if rest else 0) | sum(1 << i for i in set(dirs))


def _same_invariants(dirs, rest):
    """Every 7-bit fluid state with the mass and (vector) momentum of this one."""
    mass = len(dirs) + rest
    px, py = momentum(dirs)
    out = []
    for b in range(128):
        d = [i for i in range(6) if b >> i & 1]
        qx, qy = momentum(d)
        if len(d) + (b >> 6) == mass and abs(qx - px) < 1e-9 and abs(qy - py) < 1e-9:
            out.append(b)
    return out


def scatter_saturated(dirs, rest: bool, chirality: int) -> int:
    """FHP-III (reading R-fhp3), phrased with velocities: a state with zero
    momentum turns its whole velocity set by 60 degrees; one that shares its
    mass and momentum with exactly one other state becomes that state; the
    three states of momentum c_k and mass 3 (mover k plus a head-on pair along
    c_{k+1}, the same with the pair along c_{k+2}, rest plus movers k-1, k+1)
    and of mass 4 (rest + mover k + pair along c_{k+2}, rest + mover k + pair
    along c_{k+1}, movers k-1, k+1 + pair along c_k) are visited in that
    order for chirality 0 and backwards for chirality 1."""
    turn = 1 if chirality == 0 else -1
    same = _same_invariants(dirs, rest)
    if len(same) == 1:
        return _byte(dirs, rest)
    px, py = momentum(dirs)
    if abs(px) < 1e-9 and abs(py) < 1e-9:
        return _byte([rotate(i, turn) for i in dirs], rest)
    if len(same) == 2:
        me = _byte(dirs, rest)
        return same[1] if same[0] == me else same[0]
    k = direction_of(px, py)
    def pair(j):
        return [j, rotate(j, 3)]
    if len(dirs) + rest == 3:
        cycle = [_byte([k] + pair(rotate(k, 1)), False), _byte([k] + pair(rotate(k, 2)), False),
                 _byte([rotate(k, -1), rotate(k, 1)], True)]
    else:
        cycle = [_byte([k] + pair(rotate(k, 2)), True), _byte([k] + pair(rotate(k, 1)), True),
                 _byte([rotate(k, -1), rotate(k, 1)] + pair(k), False)]
    j = cycle.index(_byte(dirs, rest))
    return cycle[(j + turn) % 3]


def scatter(byte: int, chirality: int, rules: int = 2) -> int:
    """rules 2: FHP-II; rules 1: FHP-I (no rest-particle collisions); rules 3:
    FHP-III (collision-saturated)."""
    solid = bool(byte & 0x80)
    rest = bool(byte & 0x40)
    dirs = [i for i in range(6) if byte >> i & 1]
    if solid:
        # bounce-back: every velocity reversed
        new = [rotate(i, 3) for i in dirs]
        return 0x80 | (0x40 if rest else 0) | sum(1 << i for i in new)
    if rules == 3:
        return scatter_saturated(dirs, rest, chirality)
    px, py = momentum(dirs)
    zero = abs(px) < 1e-9 and abs(py) < 1e-9
    new_rest = rest
    new = dirs
    if len(dirs) == 2 and zero:
        turn = 1 if chirality == 0 else -1
        new = [rotate(i, turn) for i in dirs]
    elif len(dirs) == 3 and zero and all(rotate(i, 3) not in dirs for i in dirs):
        new = [rotate(i, 1) for i in dirs]
    elif rules == 1:
        pass
    elif rest and len(dirs) == 1:
        i = dirs[0]
        new = [rotate(i, 1), rotate(i, -1)]
        new_rest = False
    elif (not rest) and len(dirs) == 2:
        # two movers 120 degrees apart whose sum is a lattice velocity
        for k in range(6):
            if abs(VEL[k][0] - px) < 1e-9 and abs(VEL[k][1] - py) < 1e-9:
                new = [k]
                new_rest = True
                break
    return (0x40 if new_rest else 0) | sum(1 << i for i in new)


def thresholds(p: float) -> list[int]:
    """Q_0..Q_32 as exact integers (units of 2^-32)."""
    one = 1 << 32
    P = int(round(Fraction(p) * one))  # round half to even on the exact value
    P = max(0, min(one, P))
    q = [0]
    S = one
    for _ in range(32):
        S = (S * (one - P)) >> 32
        q.append(one - S)
    return q


def step(state: np.ndarray, seed: int, t: int, p: float, rng_word) -> np.ndarray:
    H, W = state.shape
    moved = np.zeros_like(state)
    for y in range(H):
        for x in range(W):
            v = int(state[y, x])
            moved[y, x] |= v & 0xC0
            for i in range(6):
                if v >> i & 1:
                    tx, ty = push_target(W, H, x, y, i)
                    moved[ty, tx] |= 1 << i
    out = np.zeros_like(state)
    for y in range(H):
        for x in range(W):
            chi = rng_word(seed, t, y, x // 32, 0) >> (x % 32) & 1
            out[y, x] = scatter(int(moved[y, x]), chi)
    if p > 0:
        q = thresholds(p)
        for y in range(H):
            for w in range(W // 32):
                cands = [x for x in range(32 * w, 32 * w + 32)
                         if not out[y, x] & 0x80 and out[y, x] >> 5 & 1 and not out[y, x] >> 2 & 1]
                draw = 0
                u = rng_word(seed, t, y, w, 1)
                offset = 0  # candidates seen since the last forced one
                for x in cands:
                    offset += 1
                    if q[offset - 1] <= u < q[offset]:
                        out[y, x] = (int(out[y, x]) & 0xDF) | 0x04
                        draw += 1
                        offset = 0
                        u = rng_word(seed, t, y, w, 1 + draw)
    return out
