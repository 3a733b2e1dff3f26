"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* published splitmix64 output; exact rational thresholds (Python fractions);
* the IC model's exact expectation from the cascade process (tests/ic_exact.py) and
  hand-derived closed forms (tests/golden/ic_closed_forms.txt), against the oracle run on
  every live-edge world (sampler "worlds": sketch r = world with live set = bits of r);
* scipy's connected components for the per-sketch labels;
* exhaustive search for the greedy choice and the (1 - 1/e) guarantee (Sec. 2);
* invariants: histogram sums, label idempotence, telescoping spread, submodularity,
  CELF (Alg. 2) = plain greedy, compact sketches (Alg. 3) = memoised components.
"""
from fractions import Fraction
from itertools import combinations
from pathlib import Path

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import graphgen
import oracle
from ic_exact import best_k_subset, sigma_ic, sigma_worlds, world_components, world_spread

GOLDEN = Path(__file__).resolve().parent / "golden" / "ic_closed_forms.txt"


def _golden():
    rows = []
    for line in GOLDEN.read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        name, n, edges, p, seeds, sigma, _ = [x.strip() for x in line.split("|")]
        E = [tuple(int(t) for t in e.split("-")) for e in edges.split(",") if e]
        S = [int(s) for s in seeds.split(",")]
        rows.append((name, int(n), E, Fraction(p), S, Fraction(sigma)))
    return rows


def _edge_arrays(edges):
    E = sorted((min(a, b), max(a, b)) for a, b in edges)
    u = np.array([a for a, _ in E], np.uint32)
    v = np.array([b for _, b in E], np.uint32)
    return E, u, v


# ---------------------------------------------------------------- hash + threshold
def test_mix_matches_published_splitmix64_vector():
    # splitmix64 seeded with 0 yields 0xE220A8397B1DCDAF as its first output
    # (the generator of Steele, Lea and Flood; also java.util.SplittableRandom(0)).
    assert oracle.mix(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF


def test_mix_is_a_bijection_on_a_sample():
    xs = np.random.default_rng(0).integers(0, 2**63, 5000, dtype=np.uint64)
    ys = {oracle.mix(int(x)) for x in xs}
    assert len(ys) == len(set(int(x) for x in xs))


@pytest.mark.parametrize("p", [0.0, 1e-9, 0.01, 0.02, 0.05, 0.1, 1 / 3, 0.5, 0.999999, 1.0, 1.5, -0.1])
def test_threshold_is_exact_floor(p):
    T, all_live = oracle.threshold(p)
    if p >= 1.0:
        assert all_live
    elif p <= 0.0:
        assert (T, all_live) == (0, False)
    else:
        assert not all_live
        assert T == int(Fraction(p) * 2**64)   # exact rational floor


def test_hash_live_fraction_is_binomial():
    seed, p, m, R = 42, 0.05, 4000, 64
    T, _ = oracle.threshold(p)
    hits = sum(oracle.edge_hash(seed, e, r) < T for e in range(m) for r in range(R))
    N = m * R
    assert abs(hits - N * p) < 5 * (N * p * (1 - p)) ** 0.5


def test_hash_per_sketch_and_per_edge_independence():
    seed = 42
    # same edge, different sketches / seeds, and different edges give different words
    a = [oracle.edge_hash(seed, 7, r) for r in range(200)]
    assert len(set(a)) == 200
    assert oracle.edge_hash(seed, 7, 0) != oracle.edge_hash(seed + 1, 7, 0)
    assert oracle.edge_hash(seed, 7, 0) != oracle.edge_hash(seed, 8, 0)


# ------------------------------------------------ exact IC model (worlds enumeration)
@pytest.mark.parametrize("row", _golden(), ids=lambda r: r[0])
def test_golden_closed_forms_cascade_and_worlds(row):
    name, n, edges, p, S, sigma = row
    assert sigma_ic(n, edges, S, p) == sigma          # cascade process (Sec. 2)
    if edges:
        assert sigma_worlds(n, edges, S, p) == sigma  # live-edge worlds via scipy


@pytest.mark.parametrize("row", [r for r in _golden() if r[1] >= 2], ids=lambda r: r[0])
def test_oracle_worlds_spread_equals_golden(row):
    name, n, edges, p, S, sigma = row
    E, u, v = _edge_arrays(edges)
    m = len(E)
    G = oracle.Graph(n, u, v)
    R = 1 << m
    L = G.labels(0, 0.0, R, mode=oracle.MODE_WORLDS)
    tot = Fraction(0)
    for r in range(R):
        k = bin(r).count("1")
        tot += p**k * (1 - p) ** (m - k) * oracle.spread(L[r:r + 1], S)
    assert tot == sigma
    if p == Fraction(1, 2):   # unweighted: sum over all 2^m sketches / 2^m
        assert Fraction(oracle.spread(L, S), R) == sigma


def _random_small_graph(rng, n, m):
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    idx = rng.choice(len(pairs), size=m, replace=False)
    return sorted(pairs[i] for i in idx)


@pytest.mark.parametrize("trial", range(6))
def test_oracle_gains_equal_exact_ic_spread_on_all_worlds(trial):
    rng = np.random.default_rng(100 + trial)
    n = int(rng.integers(3, 7))
    m = int(rng.integers(1, min(9, n * (n - 1) // 2) + 1))
    E = _random_small_graph(rng, n, m)
    _, u, v = _edge_arrays(E)
    G = oracle.Graph(n, u, v)
    R = 1 << m
    L = G.labels(0, 0.0, R, mode=oracle.MODE_WORLDS)
    g = oracle.gains(L)
    for x in range(n):
        assert Fraction(int(g[x]), R) == sigma_ic(n, E, [x], Fraction(1, 2))
    # labels of every world against scipy's components
    for r in range(R):
        comp = world_components(n, E, r)
        for a in range(n):
            for b in range(n):
                assert (L[r, a] == L[r, b]) == (comp[a] == comp[b])


@pytest.mark.parametrize("trial", range(4))
def test_greedy_is_stepwise_argmax_and_within_1_minus_1_over_e(trial):
    rng = np.random.default_rng(200 + trial)
    n = int(rng.integers(4, 7))
    m = int(rng.integers(2, min(8, n * (n - 1) // 2) + 1))
    E = _random_small_graph(rng, n, m)
    _, u, v = _edge_arrays(E)
    G = oracle.Graph(n, u, v)
    R = 1 << m
    L = G.labels(0, 0.0, R, mode=oracle.MODE_WORLDS)

    def spread_bf(S):  # brute force over worlds with library components
        return sum(world_spread(n, E, r, S) for r in range(R)) if S else 0

    k = 3
    seeds, gains = oracle.greedy(L, k, variant=0)
    S = []
    for i in range(k):
        base = spread_bf(S)
        marg = [(spread_bf(S + [x]) - base if x not in S else -1) for x in range(n)]
        best = max(marg)
        expect = min(x for x in range(n) if marg[x] == best)   # ties -> smallest id
        assert seeds[i] == expect and gains[i] == best
        S.append(expect)
    opt, _ = best_k_subset(n, spread_bf, k)
    assert spread_bf(S) >= (1 - 1 / np.e) * opt


# ----------------------------------------------------------------- closed forms
def test_p_zero_every_vertex_alone():
    n, u, v = graphgen.erdos_renyi(300, 1000, 5)
    G = oracle.Graph(n, u, v)
    R, k = 16, 7
    L = G.labels(42, 0.0, R)
    assert np.array_equal(L, np.tile(np.arange(n, dtype=np.uint32), (R, 1)))
    assert np.all(oracle.gains(L) == R)
    seeds, gains = oracle.greedy(L, k)
    assert list(seeds) == list(range(k)) and np.all(gains == R)
    assert oracle.spread(L, seeds) == k * R


def test_p_one_labels_are_graph_components():
    n, u, v = graphgen.erdos_renyi(500, 300, 6)
    G = oracle.Graph(n, u, v)
    R = 4
    L = G.labels(42, 1.0, R)
    A = coo_matrix((np.ones(len(u)), (u, v)), shape=(n, n))
    nc, comp = connected_components(A, directed=False)
    minid = np.full(nc, n, np.int64)
    np.minimum.at(minid, comp, np.arange(n))
    for r in range(R):
        assert np.array_equal(L[r], minid[comp])
    sizes = np.bincount(comp)
    assert np.array_equal(oracle.gains(L), (R * sizes[comp]).astype(np.uint64))


def test_hash_mode_labels_match_scipy_on_live_subgraph():
    n, u, v = graphgen.erdos_renyi(400, 1500, 7)
    seed, p, R = 42, 0.3, 5
    G = oracle.Graph(n, u, v)
    L = G.labels(seed, p, R)
    T, _ = oracle.threshold(p)
    for r in range(R):
        live = np.array([oracle.edge_hash(seed, e, r) < T for e in range(len(u))])
        A = coo_matrix((np.ones(live.sum()), (u[live], v[live])), shape=(n, n))
        nc, comp = connected_components(A, directed=False)
        minid = np.full(nc, n, np.int64)
        np.minimum.at(minid, comp, np.arange(n))
        assert np.array_equal(L[r], minid[comp])


# ------------------------------------------------------------------ invariants
@pytest.fixture(scope="module")
def er_c1():
    n, u, v, prm = graphgen.workload("er_n2000_m10000")
    G = oracle.Graph(n, u, v)
    L = G.labels(prm["seed"], prm["p"], prm["R"])
    return n, u, v, prm, G, L


def test_label_invariants(er_c1):
    n, u, v, prm, G, L = er_c1
    idx = np.arange(n)
    for r in range(0, prm["R"], 37):
        Lr = L[r].astype(np.int64)
        assert np.all(Lr <= idx) and np.array_equal(Lr[Lr], Lr)
        assert np.bincount(Lr, minlength=n).sum() == n


def test_gain_sum_is_sum_of_squared_sizes(er_c1):
    n, u, v, prm, G, L = er_c1
    g = oracle.gains(L)
    sq = sum(int((np.bincount(L[r], minlength=n).astype(np.int64) ** 2).sum()) for r in range(L.shape[0]))
    assert int(g.sum()) == sq


def test_greedy_variants_and_celf_agree(er_c1):
    n, u, v, prm, G, L = er_c1
    k = 25
    s0, g0 = oracle.greedy(L, k, variant=0)
    s1, g1 = oracle.greedy(L, k, variant=1)
    s2, g2, ev = oracle.celf(L, k)
    assert np.array_equal(s0, s1) and np.array_equal(s0, s2)
    assert np.array_equal(g0, g1) and np.array_equal(g0, g2)
    assert np.all(np.diff(g0.astype(np.int64)) <= 0)            # non-increasing
    assert oracle.spread(L, s0) == int(g0.sum())                 # telescoping
    assert np.all(ev <= n)


def test_celf_evaluation_counts_counted_by_hand():
    """Alg. 2 (CELF) on memoised components given directly, every step counted by hand.

    n = 5, R = 2.  Sketch 0: components {0, 1, 2}, {3}, {4}; sketch 1: {0}, {1, 3}, {2, 4}.
    Initial gains 4, 5, 5, 3, 3.  Round 0 takes vertex 1 (5, smaller id than 2) without an
    evaluation.  Round 1 pops 2 (fresh 2 < 4, back), 0 (fresh 1 < 3, back), 3 (fresh 1 < 3,
    back), 4 (fresh 3 > 2): 4 evaluations.  Round 2 pops 2 (fresh 0), then 0 (fresh 1, beats 3's
    stale 1 on the id): 2.  Round 3: 3 (fresh 1 > 0): 1.  Round 4: 2, the last entry: 1."""
    L = np.array([[0, 0, 0, 3, 4], [0, 1, 2, 1, 2]], np.uint32)
    seeds, gains, ev = oracle.celf(L, 5)
    assert seeds.tolist() == [1, 4, 0, 3, 2]
    assert gains.tolist() == [5, 3, 1, 1, 0]
    assert ev.tolist() == [0, 4, 2, 1, 1]
    g_seeds, g_gains = oracle.greedy(L, 5)
    assert g_seeds.tolist() == seeds.tolist() and g_gains.tolist() == gains.tolist()
    assert oracle.gains(L).tolist() == [4, 5, 5, 3, 3]


def test_submodularity_along_the_seed_sequence(er_c1):
    n, u, v, prm, G, L = er_c1
    k = 6
    seeds, _ = oracle.greedy(L, k)
    rng = np.random.default_rng(3)
    probe = rng.choice(n, 40, replace=False)
    prev = None
    for i in range(k + 1):
        S = list(seeds[:i])
        base = oracle.spread(L, S) if S else 0
        d = np.array([oracle.spread(L, S + [int(x)]) - base for x in probe])
        if prev is not None:
            assert np.all(d <= prev)
        prev = d


# ------------------------------------------------------------- compact sketches
@pytest.mark.parametrize("alpha", [1.0, 0.5, 0.1, 0.013])
def test_centers_rule(alpha):
    n, seed = 1234, 42
    c = oracle.centers(n, seed, alpha)
    rho = oracle.num_centers(n, alpha)
    assert rho == min(n, int(np.ceil(alpha * n)))
    assert len(c) == rho and np.all(np.diff(c.astype(np.int64)) > 0)
    keys = np.array([oracle.center_key(seed, x) for x in range(n)], dtype=np.uint64)
    expect = np.sort(np.argsort(keys, kind="stable")[:rho])
    assert np.array_equal(c, expect)


@pytest.mark.parametrize("alpha", [1.0, 0.3, 0.05])
def test_compact_arrays_invariants(er_c1, alpha):
    n, u, v, prm, G, L = er_c1
    R = 32
    Lr = L[:R]
    ctr = oracle.centers(n, prm["seed"], alpha)
    lab, sz = oracle.compact(Lr, ctr)
    rho = len(ctr)
    i = np.arange(rho)
    for r in range(R):
        l = lab[:, r].astype(np.int64)
        assert np.all(l <= i) and np.array_equal(l[l], l)
        root = Lr[r][ctr]
        # same label <=> same component
        for a in range(0, rho, max(1, rho // 50)):
            assert np.array_equal(l == l[a], root == root[a])
        hist = np.bincount(Lr[r], minlength=n)
        assert np.array_equal(sz[:, r], np.where(l == i, hist[root], 0))
    if alpha == 1.0:
        assert np.array_equal(lab.T, Lr)


@pytest.mark.parametrize("alpha", [1.0, 0.25, 0.02, 0.002])
def test_compact_greedy_equals_memoised_greedy(alpha):
    # Sec. 3: alpha = 1 is full memoisation, alpha -> 0 is simulation; the seeds agree.
    n, u, v = graphgen.erdos_renyi(600, 1500, 11)
    seed, p, R, k = 42, 0.15, 24, 6
    G = oracle.Graph(n, u, v)
    L = G.labels(seed, p, R)
    ctr = oracle.centers(n, seed, alpha)
    lab, sz = oracle.compact(L, ctr)
    s_c, g_c = G.compact_greedy(seed, p, R, ctr, lab, sz, k)
    s_m, g_m = oracle.greedy(L, k, variant=0)
    assert np.array_equal(s_c, s_m) and np.array_equal(g_c, g_m)


def test_compact_marginal_matches_definition_for_random_seed_sets():
    n, u, v = graphgen.erdos_renyi(400, 900, 12)
    seed, p, R, alpha = 42, 0.2, 16, 0.1
    G = oracle.Graph(n, u, v)
    L = G.labels(seed, p, R)
    ctr = oracle.centers(n, seed, alpha)
    lab, sz = oracle.compact(L, ctr)
    ci = oracle.cidx_of(n, ctr)
    rng = np.random.default_rng(5)
    for _ in range(4):
        S = sorted(rng.choice(n, 5, replace=False).tolist())
        in_s = np.zeros(n, np.uint8)
        in_s[S] = 1
        size = sz.copy()
        for r in range(R):   # MarkSeed for every seed (Alg. 3)
            for s in S:
                roots = L[r][ctr]
                hit = np.nonzero(roots == L[r][s])[0]
                if len(hit):
                    size[lab[hit[0], r], r] = 0
        base = oracle.spread(L, S)
        for x in rng.choice(n, 25, replace=False):
            want = 0 if x in S else oracle.spread(L, S + [int(x)]) - base
            assert G.compact_marginal(seed, p, R, ci, lab, size, in_s, int(x)) == want


def test_worlds_mode_compact_greedy_on_tiny_graph():
    E = [(0, 1), (1, 2), (2, 3), (3, 4), (1, 4), (5, 6)]
    E, u, v = _edge_arrays(E)
    n, R = 7, 1 << len(E)
    G = oracle.Graph(n, u, v)
    L = G.labels(0, 0.0, R, mode=oracle.MODE_WORLDS)
    for alpha in (1.0, 0.3):
        ctr = oracle.centers(n, 9, alpha)
        lab, sz = oracle.compact(L, ctr)
        s_c, g_c = G.compact_greedy(0, 0.0, R, ctr, lab, sz, 3, mode=oracle.MODE_WORLDS)
        s_m, g_m = oracle.greedy(L, 3, variant=0)
        assert np.array_equal(s_c, s_m) and np.array_equal(g_c, g_m)
    # first seed's gain / 2^m is the exact IC spread of that vertex
    assert Fraction(int(g_m[0]), R) == sigma_ic(n, E, [int(s_m[0])], Fraction(1, 2))


def test_oracle_rejects_bad_edges():
    with pytest.raises(ValueError):
        oracle.Graph(3, np.array([0], np.uint32), np.array([3], np.uint32))
    with pytest.raises(ValueError):
        oracle.Graph(3, np.array([1], np.uint32), np.array([1], np.uint32))


# ---- per-edge probabilities (Sec. 2: the IC model gives every edge its own p_e) --------

@pytest.mark.parametrize("p", [0.0, 0.05, 0.37, 1.0])
def test_per_edge_mode_with_equal_probabilities_is_the_uniform_mode(p):
    n, u, v = graphgen.erdos_renyi(400, 1500, 11)
    G = oracle.Graph(n, u, v)
    G.set_probs(np.full(len(u), p))
    assert np.array_equal(G.labels(7, -1.0, 12, mode=oracle.MODE_EDGE), G.labels(7, p, 12))


def test_per_edge_zero_one_probabilities_give_components_of_the_always_live_edges():
    n, u, v = graphgen.erdos_renyi(500, 1400, 12)
    rng = np.random.default_rng(3)
    p = rng.integers(0, 2, len(u)).astype(np.float64)
    G = oracle.Graph(n, u, v)
    G.set_probs(p)
    keep = p == 1.0
    A = coo_matrix((np.ones(keep.sum()), (u[keep], v[keep])), shape=(n, n))
    _, comp = connected_components(A, directed=False)
    first = {}
    for x in range(n):
        first.setdefault(comp[x], x)
    want = np.array([first[comp[x]] for x in range(n)], np.uint32)
    L = G.labels(5, -1.0, 6, mode=oracle.MODE_EDGE)
    for r in range(6):
        assert np.array_equal(L[r], want)


def test_per_edge_live_frequencies_follow_each_probability():
    # a perfect matching: u and its partner share a component in sketch r iff the edge is
    # live there, so (gain(u) - R) / R is the edge's live fraction
    m, R = 64, 4096
    u = np.arange(0, 2 * m, 2, dtype=np.uint32)
    v = u + 1
    p = np.linspace(0.01, 0.99, m)
    G = oracle.Graph(2 * m, u, v)
    G.set_probs(p)
    gain = oracle.gains(G.labels(21, -1.0, R, mode=oracle.MODE_EDGE)).astype(np.int64)
    frac = (gain[u] - R) / R
    sd = np.sqrt(p * (1 - p) / R)
    assert np.all(np.abs(frac - p) <= 5 * sd + 1e-12)
    assert np.array_equal(gain[u], gain[v])


def test_wic_probabilities_closed_forms():
    # star K_{1,d}: every edge joins a vertex of degree d and one of degree 1
    d = 9
    G = oracle.Graph(d + 1, np.zeros(d, np.uint32), np.arange(1, d + 1, dtype=np.uint32))
    assert np.allclose(G.set_wic(), 2.0 / (d + 1))
    # path 0-1-2-3-4: end edges 2/3, inner edges 2/4
    G = oracle.Graph(5, np.array([0, 1, 2, 3], np.uint32), np.array([1, 2, 3, 4], np.uint32))
    assert np.array_equal(G.set_wic(), np.array([2 / 3, 0.5, 0.5, 2 / 3]))
    # a single edge: p = 1, always live
    G = oracle.Graph(2, np.array([0], np.uint32), np.array([1], np.uint32))
    assert np.array_equal(G.set_wic(), [1.0])
    assert np.all(G.labels(3, -1.0, 4, mode=oracle.MODE_EDGE) == 0)


def test_per_edge_mode_compact_greedy_equals_memoised_greedy():
    n, u, v = graphgen.erdos_renyi(600, 2400, 13)
    G = oracle.Graph(n, u, v)
    G.set_probs(np.random.default_rng(8).uniform(0.1, 0.3, len(u)))
    R, k = 24, 6
    L = G.labels(42, -1.0, R, mode=oracle.MODE_EDGE)
    ctr = oracle.centers(n, 42, 0.2)
    lab, sz = oracle.compact(L, ctr)
    s1, g1 = oracle.greedy(L, k)
    s2, g2 = G.compact_greedy(42, -1.0, R, ctr, lab, sz, k, mode=oracle.MODE_EDGE)
    assert np.array_equal(s1, s2) and np.array_equal(g1, g2)
