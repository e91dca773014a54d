"""Offline search for the shared-memory row swizzles of the warp-local line
transforms (RowSwz in paper_2506_23712_gb300/csrc/ens_kernels.cuh).

A warp-local line of N complex values (float2) lives in one shared-memory
row; the z-direction passes touch it with a few fixed access patterns: the
pass exchanges of the radix plan (write in butterfly order, read in the next
pass's order), the store of the transform output, and the Hermitian
unpacking reads of positions k and N - k.  An 8-byte request of a warp is
served per half-warp: 16 lanes, 16 bank pairs, so a request costs as many
wavefronts as the most-used bank pair has distinct words.  The swizzle maps
position pos to slot pos ^ mask[pos >> 4] (a permutation inside every
16-aligned block, no padding); this script scores every pattern of one row
(five line transforms, two output stores, the unpacking reads) and searches
the masks:

  N = 128, 256: masks that are GF(2)-linear in the block index (exhaustive)
  N = 384, 512: one free mask per block (seeded local search)

The persistent z pass uses, for the power-of-two plans, one additive
layout per pass exchange instead (WPad in paper_2506_23712_gb300/csrc/ens_fft.cuh): exchange s puts
position pos at slot pos + (pos >> A_s) * D_s, and `pad_search` picks A_s,
D_s and a common row stride with the fewest wavefronts over that exchange's
store and load patterns (exhaustive over small A, D).

Run: python tests/swizzle_search.py   (prints the packed
64-bit tables and the wavefront counts: ideal, additive padding, swizzle;
then the per-exchange pad table).
"""
from __future__ import annotations

import itertools
import random

# warp-local plans of csrc/ens_fft.cuh: (threads per line P, passes, radices)
PLANS = {16: (4, (4, 4)), 32: (8, (4, 2, 4)), 64: (8, (8, 8)), 128: (16, (8, 2, 8)), 256: (32, (8, 4, 8)),
         384: (32, (4, 4, 6, 4)), 512: (32, (16, 2, 16))}


def wavefronts(words):
    """8-byte words requested by one warp (lane order) -> wavefronts."""
    total = 0
    for half in (words[:16], words[16:]):
        if not half:
            continue
        pairs = {}
        for w in set(half):
            pairs.setdefault(w % 16, set()).add(w)
        total += max(len(v) for v in pairs.values())
    return total


def patterns(N):
    """(weight, [(line, pos) per lane]) for every shared-memory request of one row."""
    P, radices = PLANS[N]
    lpw = 32 // P
    V = N // P
    out = []
    ns = 1
    for s in range(len(radices) - 1):
        R, Rn = radices[s], radices[s + 1]
        for b in range(N // (R * P)):
            for t in range(R):
                lanes = []
                for line in range(lpw):
                    for p in range(P):
                        j = p + b * P
                        lanes.append((line, (j // ns) * ns * R + (j % ns) + t * ns))
                out.append((5, lanes))
        for b in range(N // (Rn * P)):
            for t in range(Rn):
                out.append((5, [(line, p + b * P + t * (N // Rn)) for line in range(lpw) for p in range(P)]))
        ns *= R
    RL = radices[-1]
    for i in range(V):
        out.append((2, [(line, p + (i // RL) * P + (i % RL) * (N // RL)) for line in range(lpw) for p in range(P)]))
    nz = (N + 2) // 3
    for j in range((nz + P - 1) // P):
        ks = [(line, p + j * P) for line in range(lpw) for p in range(P)]
        out.append((2, [(l, k) for l, k in ks if k < nz]))
        out.append((2, [(l, (N - k) % N) for l, k in ks if k < nz]))
    return out


def cost(pats, slot, srow):
    return sum(w * wavefronts([line * srow + slot(pos) for line, pos in lanes]) for w, lanes in pats)


def ideal(pats):
    return sum(w * ((len(lanes) + 15) // 16) for w, lanes in pats)


def padded(N):
    """the additive padding the small sizes keep"""
    if len(PLANS[N][1]) == 2:
        return (lambda pos: pos + (pos >> 4)), N + N // 16 + N // 32 + 1
    return (lambda pos: pos + (pos >> 4) + (pos >> 5)), N + N // 16 + N // 32 + 1


def search(N, iters=20000, seed=1):
    pats = patterns(N)
    nblk = N // 16
    if N in (128, 256):
        bits = (nblk - 1).bit_length()
        best = None
        for cols in itertools.product(range(16), repeat=bits):
            masks = []
            for blk in range(nblk):
                m = 0
                for k, c in enumerate(cols):
                    if (blk >> k) & 1:
                        m ^= c
                masks.append(m)
            c = cost(pats, lambda pos, ms=masks: pos ^ ms[pos >> 4], N)
            if best is None or c < best[0]:
                best = (c, masks)
        return best
    rng = random.Random(seed)
    masks = [0] * nblk
    c = cost(pats, lambda pos: pos ^ masks[pos >> 4], N)
    for _ in range(iters):
        k = rng.randrange(nblk)
        old = masks[k]
        masks[k] = rng.randrange(16)
        c2 = cost(pats, lambda pos: pos ^ masks[pos >> 4], N)
        if c2 <= c:
            c = c2
        else:
            masks[k] = old
    return c, masks


def pack(masks):
    lo = sum(m << (4 * i) for i, m in enumerate(masks[:16]))
    hi = sum(m << (4 * i) for i, m in enumerate(masks[16:]))
    return lo, hi


# second warp plans of the z pass (WPlanV<N, VAR> in csrc/ens_fft.cuh)
PLAN_VARIANTS = {(256, 1): (16, (16, 16))}


def plan_of(N, var=0):
    return PLANS[N] if var == 0 else PLAN_VARIANTS[(N, var)]


def exchange_patterns(N, var=0):
    """[[per-lane (line, pos)] for every request of exchange s] for each s"""
    P, radices = plan_of(N, var)
    lpw = 32 // P
    res = []
    ns = 1
    for s in range(len(radices) - 1):
        R, Rn = radices[s], radices[s + 1]
        pats = []
        for b in range(N // (R * P)):
            for t in range(R):
                pats.append([(line, ((p + b * P) // ns) * ns * R + ((p + b * P) % ns) + t * ns)
                             for line in range(lpw) for p in range(P)])
        for b in range(N // (Rn * P)):
            for t in range(Rn):
                pats.append([(line, p + b * P + t * (N // Rn)) for line in range(lpw) for p in range(P)])
        res.append(pats)
        ns *= R
    return res


def pad_search(N, var=0):
    """(wavefronts, row stride, [(A_s, D_s)]) of the best per-exchange pads"""
    ex = exchange_patterns(N, var)
    best = None
    for srow in range(N, N + N // 2 + 1):
        tot, choice = 0, []
        for pats in ex:
            bb = None
            for A in range(1, 10):
                for D in range(0, 33):
                    f = lambda pos, A=A, D=D: pos + (pos >> A) * D
                    if f(N - 1) + 1 > srow:
                        continue
                    c = sum(wavefronts([line * srow + f(pos) for line, pos in lanes]) for lanes in pats)
                    if bb is None or (c, D, A) < bb[0]:
                        bb = ((c, D, A), A, D)
            if bb is None:
                tot = None
                break
            tot += bb[0][0]
            choice.append((bb[1], bb[2]))
        if tot is not None and (best is None or tot < best[0]):
            best = (tot, srow, choice)
    return best


if __name__ == "__main__":
    for N in (128, 256, 384, 512):
        pats = patterns(N)
        f, srow = padded(N)
        c, masks = search(N)
        lo, hi = pack(masks)
        print("N=%d ideal %d padded %d swizzled %d  lo=0x%016x hi=0x%x" % (N, ideal(pats), cost(pats, f, srow), c,
                                                                         lo, hi))
    for N in (16, 32, 64, 128, 256, 512):
        tot, srow, choice = pad_search(N)
        print("WPad<%d>: SROW %d, (A, D) per exchange %s, %d wavefronts" % (N, srow, choice, tot))
    for (N, var) in PLAN_VARIANTS:
        tot, srow, choice = pad_search(N, var)
        print("WPadV<%d, %d>: SROW %d, (A, D) per exchange %s, %d wavefronts" % (N, var, srow, choice, tot))
