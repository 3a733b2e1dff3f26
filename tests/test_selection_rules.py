"""Two rules of the device selection, checked on the host against their plain definitions.

1. Scans keep the two largest stale keys.  Each block reports its top two keys (m1 >= m2) as
   old = atomicMax(stale_max, m1) and then atomicMax(stale_2nd, max(m2, min(old, m1))).  For
   any split of the keys into blocks, and any order of the blocks, stale_2nd must end as the
   second largest key.
2. Pair steps.  After a round won by its only evaluated candidate, the next round's top stale
   key y and the next one z are evaluated together, z as if y had won.  This must give the same
   seeds, gains and per-round evaluation counts as lazy greedy with Alg. 4's doubling batches
   (Alg. 2) run one step at a time.

The model set function is a weighted coverage function: monotone and submodular, like the
spread estimate of Alg. 1.  The keys pack (gain, smallest id first), as the device's do.
"""
import random

import pytest

BITS = 12
MASK = (1 << BITS) - 1


def _key(gain, v):
    return (gain << BITS) | (MASK - v)


def _vertex(key):
    return MASK - (key & MASK)


def test_two_largest_keys_survive_any_block_order():
    rng = random.Random(5)
    for _ in range(2000):
        keys = rng.sample(range(1, 10_000), rng.randint(2, 40))
        rng.shuffle(keys)
        cuts = sorted(rng.sample(range(1, len(keys)), rng.randint(0, min(8, len(keys) - 1))))
        blocks = [keys[a:b] for a, b in zip([0] + cuts, cuts + [len(keys)])]
        rng.shuffle(blocks)
        stale_max = stale_2nd = 0
        for blk in blocks:
            top = sorted(blk, reverse=True) + [0]
            m1, m2 = top[0], top[1]
            old = stale_max
            stale_max = max(stale_max, m1)
            stale_2nd = max(stale_2nd, max(m2, min(old, m1)))
        want = sorted(keys, reverse=True)
        assert (stale_max, stale_2nd) == (want[0], want[1])


class Coverage:
    def __init__(self, n, elems, rng):
        self.w = [rng.randint(1, 9) for _ in range(elems)]
        self.sets = [set(rng.sample(range(elems), rng.randint(0, 6))) for _ in range(n)]
        self.covered = set()

    def gain(self, v, extra=()):
        cov = self.covered.union(*[self.sets[u] for u in extra]) if extra else self.covered
        return sum(self.w[e] for e in self.sets[v] - cov)

    def add(self, v):
        self.covered |= self.sets[v]


def _lazy_greedy(n, k, f, pairs):
    """Rounds of doubling batches over the largest stale keys (Alg. 2 with Alg. 4's batches).

    With `pairs`, a round won by its only evaluation is followed by a pair step.
    """
    key = {v: _key(f.gain(v), v) for v in range(n)}
    seeds, gains, evals = [], [], []
    pending = None   # (z, fresh key of z) evaluated ahead for the round that opens
    last_single = False
    while len(seeds) < k:
        fresh = {}
        if pending is not None:
            z, fz = pending
            fresh[z] = fz
            pending = None
        nev = len(fresh)
        rnd = len(seeds)
        j = 1 if fresh else 0
        while True:
            unev = sorted((key[v] for v in key if v not in fresh), reverse=True)
            best = max(fresh.values(), default=0)
            if fresh and (not unev or best > unev[0]):
                break
            take = unev if len(unev) <= 2 * (1 << j) else unev[:1 << j]
            pair_ok = (pairs and last_single and j == 0 and not fresh and len(unev) > 3
                       and rnd + 1 < k)
            if pair_ok:
                y, z = _vertex(unev[0]), _vertex(unev[1])
                fy = _key(f.gain(y), y)
                nev += 1
                if fy > unev[1]:   # y beats every other stale key: it wins its round
                    fz = _key(f.gain(z, extra=(y,)), z)
                    fresh[y] = fy
                    pending = (z, fz)
                    break
                fresh[y] = fy      # y lost: z's value is dropped
                j += 1
                continue
            for kk in take:
                v = _vertex(kk)
                fresh[v] = _key(f.gain(v), v)
            nev += len(take)
            j += 1
        sd = max(fresh, key=fresh.get)
        seeds.append(sd)
        gains.append(fresh[sd] >> BITS)
        evals.append(nev)
        last_single = nev == 1
        f.add(sd)
        for v, kv in fresh.items():
            key[v] = kv
        del key[sd]
        if pending is not None:
            z, _ = pending
            if len(seeds) >= k:
                pending = None
    return seeds, gains, evals


@pytest.mark.parametrize("seed", range(40))
def test_pair_steps_keep_lazy_greedy(seed):
    rng = random.Random(seed)
    n = rng.randint(6, 60)
    elems = rng.randint(5, 80)
    k = rng.randint(1, n)
    base = Coverage(n, elems, random.Random(seed))
    with_pairs = Coverage(n, elems, random.Random(seed))
    a = _lazy_greedy(n, k, base, pairs=False)
    b = _lazy_greedy(n, k, with_pairs, pairs=True)
    assert a == b
    # and the seeds are those of plain greedy (largest marginal gain, smallest id on ties)
    plain = Coverage(n, elems, random.Random(seed))
    want = []
    for _ in range(k):
        v = max((u for u in range(n) if u not in want), key=lambda u: (plain.gain(u), -u))
        want.append(v)
        plain.add(v)
    assert a[0] == want
