"""Exhaustive enumerators used to pin the oracle (tests only).

1. exact_win_probs: the exact winner distribution of a random playout from a
   tiny endgame, by walking every random branch (draw, joker position, guess,
   continue coin) with rational weights.  It is a third, independent statement
   of the rules of Sec. II-A (explicit Python lists, recursion with memo); the
   oracle's Monte Carlo estimate must fall within a binomial bound of it.

2. consistent_deals: every assignment of the tiles an observer cannot see to
   the opponents' face-down slots that keeps numbered tiles ascending (jokers
   free), by plain enumeration of permutations.  Pins the determinizer's count
   and, through a chi-square test, its uniformity.
"""
from fractions import Fraction
from functools import lru_cache
from itertools import permutations


def exact_win_probs(hands, revealed, cur, drawn, ntiles, p_cont, ordered=False, may_stop=False):
    """hands: list of left-to-right tile lists; revealed: set.  The player to
    move is about to guess.  ordered: guesses restricted to identities that
    fit between the slot's nearest face-up numbered neighbours (jokers fit
    anywhere).  may_stop: the player to move has just guessed correctly, so
    with probability p_cont it guesses again and otherwise the turn passes.
    Returns {player: Fraction}."""
    P = len(hands)
    p_cont = Fraction(p_cont)
    init = (tuple(tuple(h) for h in hands), frozenset(revealed),
            tuple(any(t not in revealed for t in h) for h in hands), cur, drawn)

    def pool_of(hs):
        held = {t for h in hs for t in h}
        return [t for t in range(ntiles) if t not in held]

    def insert_positions(h, t):
        if t < 24:
            for i, u in enumerate(h):
                if u < 24 and u > t:
                    return [i]
            return [len(h)]
        return list(range(len(h) + 1))

    def merge(acc, dist, w):
        for k, v in dist.items():
            acc[k] = acc.get(k, Fraction(0)) + v * w

    @lru_cache(maxsize=None)
    def new_turn(hs, rv, alive, c):
        p = c
        while True:
            p = (p + 1) % P
            if alive[p]:
                break
        pool = pool_of(hs)
        if not pool:
            return guess(hs, rv, alive, p, None)
        acc = {}
        for t in pool:
            opts = insert_positions(hs[p], t)
            for pos in opts:
                h = list(hs[p])
                h.insert(pos, t)
                hs2 = tuple(tuple(h) if q == p else hs[q] for q in range(P))
                merge(acc, guess(hs2, rv, alive, p, t), Fraction(1, len(pool) * len(opts)))
        return acc

    @lru_cache(maxsize=None)
    def guess(hs, rv, alive, c, dr):
        own = set(hs[c])
        legal = []
        for off in range(1, P):
            q = (c + off) % P
            if not alive[q]:
                continue
            for i, t in enumerate(hs[q]):
                if t in rv:
                    continue
                left = [u for u in hs[q][:i] if u in rv and u < 24]
                right = [u for u in hs[q][i + 1:] if u in rv and u < 24]
                lo = left[-1] if left else -1
                hi = right[0] if right else 24
                for x in range(ntiles):
                    if x in own or x in rv:
                        continue
                    if ordered and x < 24 and not lo < x < hi:
                        continue
                    legal.append((q, i, x))
        acc = {}
        w = Fraction(1, len(legal))
        for q, i, x in legal:
            t = hs[q][i]
            if t == x:
                rv2 = rv | {t}
                al = list(alive)
                if all(u in rv2 for u in hs[q]):
                    al[q] = False
                al = tuple(al)
                if sum(al) == 1:
                    merge(acc, {c: Fraction(1)}, w)
                    continue
                if p_cont > 0:
                    merge(acc, guess(hs, rv2, al, c, dr), w * p_cont)
                    merge(acc, new_turn(hs, rv2, al, c), w * (1 - p_cont))
                else:
                    merge(acc, new_turn(hs, rv2, al, c), w)
            else:
                if dr is not None:
                    rv2 = rv | {dr}
                else:
                    first = next(u for u in hs[c] if u not in rv)
                    rv2 = rv | {first}
                al = list(alive)
                if all(u in rv2 for u in hs[c]):
                    al[c] = False
                al = tuple(al)
                if sum(al) == 1:
                    merge(acc, {al.index(True): Fraction(1)}, w)
                    continue
                merge(acc, new_turn(hs, rv2, al, c), w)
        return acc

    hs, rv, alive, c, dr = init
    if may_stop:
        acc = {}
        if p_cont > 0:
            merge(acc, guess(hs, rv, alive, c, dr), p_cont)
        if p_cont < 1:
            merge(acc, new_turn(hs, rv, alive, c), 1 - p_cont)
        return acc
    return guess(hs, rv, alive, c, dr)


def consistent_deals(hands, revealed, observer, ntiles):
    """All full assignments consistent with the observer's view.  Returns a
    list of tuples: for each opponent (seat order from observer+1) the tuple of
    tiles in its face-down slots, left to right."""
    P = len(hands)
    opps = [(observer + k) % P for k in range(1, P)]
    own = set(hands[observer])
    unknown = [t for t in range(ntiles) if t not in own and t not in revealed]
    slots = []
    for q in opps:
        for i, t in enumerate(hands[q]):
            if t not in revealed:
                slots.append((q, i))
    out = []
    for perm in permutations(unknown, len(slots)):
        new = {q: list(hands[q]) for q in opps}
        for (q, i), t in zip(slots, perm):
            new[q][i] = t
        ok = True
        for q in opps:
            nums = [t for t in new[q] if t < 24]
            if any(a > b for a, b in zip(nums, nums[1:])):
                ok = False
                break
        if ok:
            out.append(tuple(tuple(new[q][i] for i, t in enumerate(hands[q]) if t not in revealed) for q in opps))
    return out
