"""Search the shared-memory placement of the 16 x 16 block layout (kPhys16, kAssign16 in
csrc/lrh_block.cuh).

A region's matrix is stored as 72 units of 16 bytes: unit u < 36 holds entries (0, 1) of block u,
unit 36 + u entries (2, 3), blocks being the upper-triangle 2 x 2 blocks (k <= l) of the 8 x 8
block grid in row order.  A buffer offers 144 unit slots.  Each round, every off-diagonal block
is read (two 16-byte loads) by its (j, lane) position and its four entries are written (8-byte
stores) to their positions after the tournament permutation; the diagonal blocks are read by
lanes pair mod 8 and three of their entries written by lanes 0..7.  The model counts shared-memory
wavefronts as the hardware serves them: 8-byte stores per 16 lanes (32 banks x 4 bytes = 16 slots
of 8 bytes), 16-byte loads per 8 lanes (8 slots of 16 bytes); lanes reading the same address
share a wavefront, lanes hitting one slot class at different addresses need one each.
Simulated annealing over the placement and the block-to-position assignment minimises the
count; the kernel's tables are the result.

    python -m paper_2609_40336_b300.blk16_layout [iterations] [seed]
"""
from __future__ import annotations

import math
import random
import sys

D, N, NB, NOFF, PER, SLOTS = 16, 8, 36, 28, 2, 144


def rr_dst(o: int) -> int:
    """Next slot of the entries in slot o under the round-robin tournament."""
    return 0 if o == 0 else (2 if o == 1 else (o - 2 if o % 2 else (D - 1 if o == D - 2 else o + 2)))


def bidx(k: int, l: int) -> int:
    return k * N - (k * (k - 1)) // 2 + (l - k)


def unit_of(i: int, j: int):
    e = ((i & 1) << 1) | (j & 1)
    return (e >> 1) * NB + bidx(i >> 1, j >> 1), e & 1


def dest(i: int, j: int):
    a, b = rr_dst(i), rr_dst(j)
    return unit_of(a, b) if a <= b else unit_of(b, a)


OFF = [(k, l) for k in range(N) for l in range(k + 1, N)]


def wavefronts_load(slots):
    w = 0
    for q in range(0, len(slots), 8):
        cls = {}
        for x in slots[q:q + 8]:
            cls.setdefault(x % 8, set()).add(x)
        w += max(len(v) for v in cls.values())
    return w


def wavefronts_store(f2):
    cls = {}
    for x in f2:
        cls.setdefault(x % 16, set()).add(x)
    return max(len(v) for v in cls.values())


def cost(phys, assign):
    total = 0
    for j in range(PER):
        blocks = [assign[j * 16 + s] if assign[j * 16 + s] >= 0 else NOFF - 1 for s in range(16)]
        total += wavefronts_load([phys[bidx(*OFF[b])] for b in blocks])
        total += wavefronts_load([phys[NB + bidx(*OFF[b])] for b in blocks])
        for e in range(4):
            f2 = []
            for b in blocks:
                k, l = OFF[b]
                u, h = dest(2 * k + (e >> 1), 2 * l + (e & 1))
                f2.append(phys[u] * 2 + h)
            total += wavefronts_store(f2)
    diag = [bidx(s & 7, s & 7) for s in range(16)]
    total += wavefronts_load([phys[u] for u in diag]) + wavefronts_load([phys[NB + u] for u in diag])
    for a, b in ((0, 0), (0, 1), (1, 1)):
        f2 = []
        for s in range(8):
            u, h = dest(2 * s + a, 2 * s + b)
            f2.append(phys[u] * 2 + h)
        total += wavefronts_store(f2)
    return total


def search(iters: int = 200000, seed: int = 0):
    rnd = random.Random(seed)
    phys = list(range(2 * NB))
    free = list(range(2 * NB, SLOTS))
    assign = [m if m < NOFF else -1 for m in [s + 16 * j for j in range(PER) for s in range(16)]]
    cur = cost(phys, assign)
    best = (cur, list(phys), list(assign))
    start = cur
    for it in range(iters):
        temp = 1.5 * (1 - it / iters) + 0.02
        r = rnd.random()
        if r < 0.4:
            a, fi = rnd.randrange(2 * NB), rnd.randrange(len(free))
            phys[a], free[fi] = free[fi], phys[a]
            c = cost(phys, assign)
            if c <= cur or rnd.random() < math.exp((cur - c) / temp):
                cur = c
            else:
                phys[a], free[fi] = free[fi], phys[a]
        elif r < 0.7:
            a, b = rnd.randrange(2 * NB), rnd.randrange(2 * NB)
            phys[a], phys[b] = phys[b], phys[a]
            c = cost(phys, assign)
            if c <= cur or rnd.random() < math.exp((cur - c) / temp):
                cur = c
            else:
                phys[a], phys[b] = phys[b], phys[a]
        else:
            a, b = rnd.randrange(32), rnd.randrange(32)
            assign[a], assign[b] = assign[b], assign[a]
            c = cost(phys, assign)
            if c <= cur or rnd.random() < math.exp((cur - c) / temp):
                cur = c
            else:
                assign[a], assign[b] = assign[b], assign[a]
        if cur < best[0]:
            best = (cur, list(phys), list(assign))
    return start, best


if __name__ == "__main__":
    iters = int(sys.argv[1]) if len(sys.argv) > 1 else 200000
    seed = int(sys.argv[2]) if len(sys.argv) > 2 else 0
    start, (c, phys, assign) = search(iters, seed)
    print(f"modelled wavefronts per round and region: {start} (identity) -> {c}")
    print("kPhys16 =", ", ".join(map(str, phys)))
    print("kAssign16 =", ", ".join(map(str, assign)))
