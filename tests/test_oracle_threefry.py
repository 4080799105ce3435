"""Pin of the oracle's Threefry-4x64-12 (Sec. "Computation with stochastic
differential equations" names the generator; Salmon et al., SC'11, define it):
no published known-answer vectors are available offline, so the oracle's
block function is pinned by its structure instead.  Threefry is a key-
alternating cipher -- for a fixed key a bijection of the 256-bit counter -- so
its inverse is a separate computation: undo each key injection (after every
fourth round, with the injection counter s, and the key-schedule word that
XORs the key with the parity constant 0x1BD11BDAA9FC1A22), then each round in
reverse (XOR, rotate right by the round's constants (14,16), (52,57), (23,40),
(5,37), (25,33), (46,12), (58,22), (32,32), subtract; the word pairs swap
between even and odd rounds), then the initial key addition.  Running that
inverse on the oracle's outputs must give back the counters; a dropped
injection, a wrong rotation, a swapped pair or a wrong round count in the
oracle's forward function does not round-trip."""
import ctypes as C

import numpy as np

import oracle as O

M64 = (1 << 64) - 1
ROT = ((14, 16), (52, 57), (23, 40), (5, 37), (25, 33), (46, 12), (58, 22), (32, 32))
PARITY = 0x1BD11BDAA9FC1A22


def rotr(x, r):
    return ((x >> r) | (x << (64 - r))) & M64


def inverse(out, key, rounds=12):
    ks = list(key) + [PARITY ^ key[0] ^ key[1] ^ key[2] ^ key[3]]
    x0, x1, x2, x3 = out
    for r in reversed(range(rounds)):
        if r % 4 == 3:
            s = r // 4 + 1
            x0 = (x0 - ks[s % 5]) & M64
            x1 = (x1 - ks[(s + 1) % 5]) & M64
            x2 = (x2 - ks[(s + 2) % 5]) & M64
            x3 = (x3 - ks[(s + 3) % 5] - s) & M64
        ra, rb = ROT[r % 8]
        if r % 2 == 0:      # forward: (x0, x1) with ra, (x2, x3) with rb
            x1 = rotr(x1 ^ x0, ra)
            x0 = (x0 - x1) & M64
            x3 = rotr(x3 ^ x2, rb)
            x2 = (x2 - x3) & M64
        else:               # forward: (x0, x3) with ra, (x2, x1) with rb
            x3 = rotr(x3 ^ x0, ra)
            x0 = (x0 - x3) & M64
            x1 = rotr(x1 ^ x2, rb)
            x2 = (x2 - x1) & M64
    return [(x0 - ks[0]) & M64, (x1 - ks[1]) & M64, (x2 - ks[2]) & M64, (x3 - ks[3]) & M64]


def oracle_block(ctr, key):
    L = O.lib()
    c = (C.c_uint64 * 4)(*ctr)
    k = (C.c_uint64 * 4)(*key)
    o = (C.c_uint64 * 4)()
    L.orc_threefry4x64_12(c, k, o)
    return [int(v) for v in o]


def test_threefry_inverts_to_its_counter():
    rng = np.random.default_rng(2411)
    cases = [([0, 0, 0, 0], [0, 0, 0, 0]), ([M64] * 4, [M64] * 4),
             ([1, 0, 0, 0], [0, 0, 0, 0]), ([0, 0, 0, 1], [20241125, 0, 0, 0])]
    for _ in range(300):
        cases.append(([int(v) for v in rng.integers(0, 2**63, 4, dtype=np.uint64) * 2 + 1],
                      [int(v) for v in rng.integers(0, 2**63, 4, dtype=np.uint64)]))
    for ctr, key in cases:
        out = oracle_block(ctr, key)
        assert out != ctr
        assert inverse(out, key) == ctr, (ctr, key)


def test_round_count_and_injections_matter():
    """Inverting with one round fewer or more, or a key with one bit flipped,
    does not give the counter back: the pin is sensitive to each."""
    ctr, key = [5, 6, 7, 8], [20241125, 0, 0, 0]
    out = oracle_block(ctr, key)
    assert inverse(out, key, rounds=11) != ctr
    assert inverse(out, key, rounds=13) != ctr
    assert inverse(out, [20241125 ^ 1, 0, 0, 0]) != ctr
