"""GPU path (through the C ABI) against the CPU oracle, element by element.

Everything is integer, so every comparison is exact: labels, component sizes, initial gains,
centers, compact label/size arrays, the seed sequence, the gains along it and the spread.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_07554_gb300 as im  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    im.lib()


def _run(n, u, v, seed, p, R, alpha, k, batch=0, spread_sets=(), lanes=1, spec=None):
    with im.IMContext(n, u, v) as ctx:
        if batch:
            im.im_set_sketch_batch(ctx.h, batch)
        if spec is not None:
            im.im_set_seed_speculation(ctx.h, spec)
        im.im_set_pipeline(ctx.h, lanes)
        ctx.build_sketches(R, seed, p, alpha)
        out = dict(gains=ctx.gains(), centers=ctx.centers())
        out["label"], out["size"] = ctx.compact()
        if k:
            out["seeds"], out["seed_gains"] = ctx.select_seeds(k)
            out["spread"] = ctx.spread(out["seeds"])
            out["round_evals"] = ctx.round_evals()
        out["spreads"] = [ctx.spread(s) for s in spread_sets]
        out["stats"] = ctx.stats()
        out["labels"] = {r: ctx.labels(r) for r in range(min(R, 8))}
    return out


def _oracle(n, u, v, seed, p, R, alpha, k):
    G = oracle.Graph(n, u, v)
    L = G.labels(seed, p, R)
    ctr = oracle.centers(n, seed, alpha)
    lab, sz = oracle.compact(L, ctr)
    o = dict(L=L, gains=oracle.gains(L), centers=ctr, label=lab, size=sz)
    if k:
        o["seeds"], o["seed_gains"] = oracle.greedy(L, k)
        o["spread"] = oracle.spread(L, o["seeds"])
    return o


def _compare(g, o, k):
    for r, lab in g["labels"].items():
        assert np.array_equal(lab, o["L"][r]), f"labels of sketch {r}"
    assert np.array_equal(g["gains"], o["gains"]), "initial gains"
    assert np.array_equal(g["centers"], o["centers"]), "centers"
    assert np.array_equal(g["label"], o["label"]), "compact labels"
    assert np.array_equal(g["size"], o["size"]), "compact sizes"
    if k:
        assert np.array_equal(g["seeds"], o["seeds"]), (g["seeds"], o["seeds"])
        assert np.array_equal(g["seed_gains"], o["seed_gains"])
        assert g["spread"] == o["spread"] == int(o["seed_gains"].sum())


def test_er_full_labels_workload():
    """n=2000, m=10^4 Erdos-Renyi, p=0.05, R=256, full labels, k=10 (all sketches checked)."""
    n, u, v, prm = graphgen.workload("er_n2000_m10000")
    g = _run(n, u, v, prm["seed"], prm["p"], prm["R"], prm["alpha"], prm["k"])
    o = _oracle(n, u, v, prm["seed"], prm["p"], prm["R"], prm["alpha"], prm["k"])
    _compare(g, o, prm["k"])
    with im.IMContext(n, u, v) as ctx:
        ctx.build_sketches(prm["R"], prm["seed"], prm["p"], prm["alpha"])
        for r in range(prm["R"]):
            assert np.array_equal(ctx.labels(r), o["L"][r]), r


@pytest.mark.parametrize("alpha", [0.5, 0.1, 0.01])
@pytest.mark.parametrize("p", [0.05, 0.2])
def test_compact_sketches(alpha, p):
    n, u, v = graphgen.erdos_renyi(3001, 9007, 4)
    g = _run(n, u, v, 42, p, 77, alpha, 12)
    o = _oracle(n, u, v, 42, p, 77, alpha, 12)
    _compare(g, o, 12)


def test_small_alpha_forces_global_fallback_search():
    # p well above the percolation threshold: a giant component with very few centers, so
    # many searches exceed the shared-memory queue and spill to the global one
    n, u, v = graphgen.erdos_renyi(4000, 12000, 9)
    g = _run(n, u, v, 7, 0.4, 40, 0.001, 6, spec=0)   # round 1 by searches, not overlap sums
    o = _oracle(n, u, v, 7, 0.4, 40, 0.001, 6)
    _compare(g, o, 6)
    assert g["stats"]["bfs_fallbacks"] > 0


@pytest.mark.parametrize("lanes", [1, 2])
@pytest.mark.parametrize("batch", [1, 2, 4, 8, 16, 32])
def test_sketch_batch_sizes_agree(batch, lanes):
    n, u, v = graphgen.erdos_renyi(1500, 6001, 3)
    g = _run(n, u, v, 42, 0.1, 45, 0.2, 5, batch=batch, lanes=lanes)
    o = _oracle(n, u, v, 42, 0.1, 45, 0.2, 5)
    _compare(g, o, 5)


@pytest.mark.parametrize("path", [0, 1, 2])
@pytest.mark.parametrize("alpha", [1.0, 0.2])
@pytest.mark.parametrize("R", [40, 77])
def test_union_paths_agree(path, alpha, R):
    # IM_UNION_FUSED (hashing and unions in one kernel), IM_UNION_RECORDS (live-pair records and
    # a union kernel with several unions in flight per thread) and IM_UNION_BUCKETS (records
    # grouped by sketch, united sketch by sketch): all equal the oracle (R = 77: a ragged batch)
    n, u, v = graphgen.erdos_renyi(2500, 9000, 17)
    with im.IMContext(n, u, v) as ctx:
        im.im_set_union_path(ctx.h, path)
        ctx.build_sketches(R, 42, 0.15, alpha)
        g = dict(gains=ctx.gains(), centers=ctx.centers())
        g["label"], g["size"] = ctx.compact()
        g["seeds"], g["seed_gains"] = ctx.select_seeds(6)
        g["spread"] = ctx.spread(g["seeds"])
        g["labels"] = {r: ctx.labels(r) for r in (0, R - 1)}
    o = _oracle(n, u, v, 42, 0.15, R, alpha, 6)
    _compare(g, o, 6)


@pytest.mark.parametrize("path", [1, 2])
def test_record_overflow_falls_back_to_the_fused_loop(path):
    # the record capacity capped far below the live pairs of a batch: the union kernel redoes
    # every batch with the fused sampling+union loop (decided on the device); same results
    n, u, v = graphgen.erdos_renyi(3000, 12000, 18)
    im.im_debug_record_cap(100)
    try:
        g = _run_path(n, u, v, 42, 0.2, 40, 0.3, 6, path)
    finally:
        im.im_debug_record_cap(-1)
    _compare(g, _oracle(n, u, v, 42, 0.2, 40, 0.3, 6), 6)


def _run_path(n, u, v, seed, p, R, alpha, k, path):
    with im.IMContext(n, u, v) as ctx:
        im.im_set_union_path(ctx.h, path)
        ctx.build_sketches(R, seed, p, alpha)
        out = dict(gains=ctx.gains(), centers=ctx.centers())
        out["label"], out["size"] = ctx.compact()
        out["seeds"], out["seed_gains"] = ctx.select_seeds(k)
        out["spread"] = ctx.spread(out["seeds"])
        out["labels"] = {r: ctx.labels(r) for r in (0, R - 1)}
    return out


@pytest.mark.parametrize("R", [40, 64])
def test_bucketed_unions_over_many_regions(R):
    # a graph large enough that the bucketed sampling writes one region per (sketch, sampling
    # block) for thousands of blocks and each union block takes several regions of one sketch
    # (R = 40: a ragged second batch); equal to the oracle and to the record path
    n, u, v = graphgen.chung_lu(200000, 2000000, 2.1, 2000.0, 19)
    g = _run_path(n, u, v, 42, 0.1, R, 0.1, 5, im.IM_UNION_BUCKETS)
    o = _oracle(n, u, v, 42, 0.1, R, 0.1, 5)
    _compare(g, o, 5)
    r = _run_path(n, u, v, 42, 0.1, R, 0.1, 5, im.IM_UNION_RECORDS)
    for key in ("gains", "label", "size", "seeds", "seed_gains"):
        assert np.array_equal(g[key], r[key]), key


def test_large_graph_adjacency_built_in_source_ranges():
    # from 2^24 edges the static adjacency is built in two passes (arcs binned by source range,
    # then placed range by range); the searches of the selection walk it: seeds, gains, spread,
    # compact sketches and labels equal the oracle's
    n, u, v = graphgen.erdos_renyi(1 << 20, (1 << 24) + 4097, 7)
    g = _run(n, u, v, 42, 0.05, 8, 0.1, 5)
    o = _oracle(n, u, v, 42, 0.05, 8, 0.1, 5)
    _compare(g, o, 5)


def test_automatic_union_path():
    # IM_UNION_AUTO (the default) takes the record path while a batch's parent arrays fit in
    # 256 MiB and the bucketed path beyond
    n, u, v = graphgen.erdos_renyi(3000, 9000, 21)
    with im.IMContext(n, u, v) as ctx:
        ctx.build_sketches(32, 42, 0.1, 1.0)
        assert ctx.stats()["union_path"] == im.IM_UNION_RECORDS
    n2 = 2200000                        # 4 n B = 282 MB with 32 sketches per batch
    u2 = np.arange(0, 200000, dtype=np.uint32)
    v2 = (u2 * 7 + 1) % n2
    with im.IMContext(n2, u2, v2.astype(np.uint32)) as ctx:
        im.im_set_sketch_batch(ctx.h, 32)
        ctx.build_sketches(32, 42, 0.5, 1.0)
        assert ctx.stats()["union_path"] == im.IM_UNION_BUCKETS
        im.im_set_union_path(ctx.h, im.IM_UNION_RECORDS)
        ctx.build_sketches(32, 42, 0.5, 1.0)
        assert ctx.stats()["union_path"] == im.IM_UNION_RECORDS


@pytest.mark.parametrize("R", [1, 31, 33, 64])
def test_ragged_sketch_counts(R):
    n, u, v = graphgen.erdos_renyi(777, 3333, 5)
    g = _run(n, u, v, 11, 0.1, R, 0.3, 7)
    o = _oracle(n, u, v, 11, 0.1, R, 0.3, 7)
    _compare(g, o, 7)


def test_p_zero_and_p_one():
    n, u, v = graphgen.erdos_renyi(500, 700, 2)
    for p in (0.0, 1.0):
        for alpha in (1.0, 0.25):
            g = _run(n, u, v, 42, p, 16, alpha, 5)
            o = _oracle(n, u, v, 42, p, 16, alpha, 5)
            _compare(g, o, 5)
    g = _run(n, u, v, 42, 0.0, 16, 1.0, 5)
    assert list(g["seeds"]) == [0, 1, 2, 3, 4] and g["spread"] == 5 * 16


def test_no_edges_and_single_vertex():
    e = np.zeros(0, np.uint32)
    g = _run(5, e, e, 42, 0.5, 8, 1.0, 5)
    assert list(g["seeds"]) == [0, 1, 2, 3, 4] and np.all(g["gains"] == 8)
    g = _run(1, e, e, 42, 0.5, 3, 1.0, 1)
    assert list(g["seeds"]) == [0] and g["spread"] == 3


def test_select_every_vertex():
    n, u, v = graphgen.erdos_renyi(60, 150, 8)
    g = _run(n, u, v, 42, 0.3, 20, 0.5, n)
    o = _oracle(n, u, v, 42, 0.3, 20, 0.5, n)
    _compare(g, o, n)
    assert sorted(g["seeds"].tolist()) == list(range(n))


def test_parallel_edges_are_sampled_independently():
    # a multigraph: every edge twice, each copy with its own edge id
    n, u, v = graphgen.erdos_renyi(400, 900, 12)
    uu, vv = np.concatenate([u, u]), np.concatenate([v, v])
    g = _run(n, uu, vv, 42, 0.2, 32, 0.2, 6)
    o = _oracle(n, uu, vv, 42, 0.2, 32, 0.2, 6)
    _compare(g, o, 6)


def test_prefix_consistency_and_reset():
    n, u, v = graphgen.erdos_renyi(2000, 8000, 6)
    with im.IMContext(n, u, v) as ctx:
        ctx.build_sketches(64, 42, 0.08, 0.2)
        s5, g5 = ctx.select_seeds(5)
        s12, g12 = ctx.select_seeds(12)
        s3, _ = ctx.select_seeds(3)
        assert np.array_equal(s12[:5], s5) and np.array_equal(g12[:5], g5)
        assert np.array_equal(s3, s5[:3])
        ctx.reset_selection()
        s12b, g12b = ctx.select_seeds(12)
        assert np.array_equal(s12, s12b) and np.array_equal(g12, g12b)


def test_spread_of_arbitrary_seed_sets():
    n, u, v = graphgen.erdos_renyi(2500, 9000, 13)
    rng = np.random.default_rng(1)
    sets = [rng.choice(n, k, replace=True).astype(np.uint32) for k in (1, 7, 50, 333)]
    sets.append(np.array([5, 5, 5], np.uint32))
    sets.append(np.zeros(0, np.uint32))
    for alpha in (1.0, 0.05):
        g = _run(n, u, v, 42, 0.15, 48, alpha, 0, spread_sets=sets)
        L = oracle.Graph(n, u, v).labels(42, 0.15, 48)
        for s, got in zip(sets, g["spreads"]):
            assert got == (oracle.spread(L, s) if len(s) else 0)


def test_device_pointer_input_and_torch_stream():
    n, u, v = graphgen.erdos_renyi(1000, 4000, 14)
    du = torch.from_numpy(u.view(np.int32)).cuda()
    dv = torch.from_numpy(v.view(np.int32)).cuda()
    stream = torch.cuda.Stream()
    with im.IMContext(n, du, dv, stream=stream.cuda_stream) as ctx:
        ctx.build_sketches(32, 42, 0.1, 0.3)
        seeds, gains = ctx.select_seeds(6)
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.labels(3, out)
        torch.cuda.synchronize()
    o = _oracle(n, u, v, 42, 0.1, 32, 0.3, 6)
    assert np.array_equal(seeds, o["seeds"]) and np.array_equal(gains, o["seed_gains"])
    assert np.array_equal(out.cpu().numpy().view(np.uint32), o["L"][3])


def test_argument_errors():
    n, u, v = graphgen.erdos_renyi(100, 200, 1)
    with im.IMContext(n, u, v) as ctx:
        with pytest.raises(im.IMError) as e:
            ctx.select_seeds(1)
        assert e.value.code == im.IM_ESTATE
        for bad in [dict(R=0, alpha=1.0), dict(R=4, alpha=0.0), dict(R=4, alpha=1.5)]:
            with pytest.raises(im.IMError) as e:
                ctx.build_sketches(bad["R"], 42, 0.1, bad["alpha"])
            assert e.value.code == im.IM_EINVAL
        ctx.build_sketches(4, 42, 0.1, 1.0)
        with pytest.raises(im.IMError):
            ctx.select_seeds(101)
        with pytest.raises(im.IMError):
            ctx.spread(np.array([100], np.uint32))
        with pytest.raises(im.IMError):
            ctx.labels(4)
    for bad_u, bad_v in [([0, 3], [1, 3]),            # self-loop
                         ([0, 7], [1, 2]),            # id >= n (skipped by the degree count)
                         ([0, 1], [0x80000000, 2])]:  # id >= 2^31
        with pytest.raises(im.IMError) as e:
            im.IMContext(4, np.array(bad_u, np.uint32), np.array(bad_v, np.uint32))
        assert e.value.code == im.IM_EINVAL


def test_lazy_evaluation_counts_are_bounded():
    # Sec. 4: batched lazy evaluation does at most twice the work of CELF
    n, u, v, prm = graphgen.workload("er_n2000_m10000")
    G = oracle.Graph(n, u, v)
    L = G.labels(prm["seed"], prm["p"], prm["R"])
    k = 30
    _, _, ev_celf = oracle.celf(L, k)
    with im.IMContext(n, u, v) as ctx:
        ctx.build_sketches(prm["R"], prm["seed"], prm["p"], 1.0)
        ctx.select_seeds(k)
        ev = ctx.round_evals()
    assert ev[0] == 0
    # Sec. 4.1: prefix doubling re-evaluates the candidates in CELF's order and stops at the
    # end of the first batch that holds CELF's stopping point, so a round costs at most 2 c - 1
    # evaluations where CELF costs c; a pair step (one round's candidate evaluated with the
    # next round's) adds at most one evaluation to a round
    assert np.all(ev <= 2 * ev_celf + 1)
    assert int(ev.sum()) <= 2 * int(ev_celf.sum())


@pytest.mark.parametrize("threshold", [1, 2**64 - 1])
@pytest.mark.parametrize("alpha", [1.0, 0.1])
def test_both_batch_evaluators_give_identical_seeds(threshold, alpha):
    # threshold 1: every re-evaluation batch recomputes the sketches; 2^64-1: every batch
    # runs one GetCenter search per (candidate, sketch).  Both must equal plain greedy.
    n, u, v = graphgen.chung_lu(20000, 120000, 2.1, 2000.0, 5)
    seed, p, R, k = 42, 0.05, 64, 25
    with im.IMContext(n, u, v) as ctx:
        im.im_set_refresh_threshold(ctx.h, threshold)
        im.im_set_seed_speculation(ctx.h, 0)   # round 1 by the evaluator under test too
        ctx.build_sketches(R, seed, p, alpha)
        seeds, gains = ctx.select_seeds(k)
        st = ctx.stats()
    o = _oracle(n, u, v, seed, p, R, alpha, k)
    assert np.array_equal(seeds, o["seeds"]) and np.array_equal(gains, o["seed_gains"])
    if threshold == 1:
        assert st["refresh_batches"] > 0
    else:
        assert st["refresh_batches"] == 0


@pytest.mark.parametrize("threshold", [1, 64, 2**64 - 1])
def test_graph_and_host_driven_selection_agree(threshold):
    """The selection loop as one CUDA graph (while / switch nodes set by k_plan and
    k_mark_seed) and the same kernels launched batch by batch from the host: identical seeds,
    gains, per-round evaluation counts and batch counts, equal to the oracle's greedy.
    threshold 1 evaluates every batch by refresh, 2^64-1 every batch by searches, 64 mixes."""
    n, u, v = graphgen.erdos_renyi(3001, 9007, 4)
    k = 40
    G = oracle.Graph(n, u, v)
    L = G.labels(42, 0.2, 77)
    o_seeds, o_gains = oracle.greedy(L, k)
    got = []
    for graph in (True, False):
        with im.IMContext(n, u, v) as ctx:
            im.im_set_graph(ctx.h, graph)
            im.im_set_refresh_threshold(ctx.h, threshold)
            ctx.build_sketches(77, 42, 0.2, 0.1)
            s1, _ = ctx.select_seeds(7)            # a prefix, then the rest
            seeds, gains = ctx.select_seeds(k)
            st = ctx.stats()
            got.append((seeds, gains, ctx.round_evals(), st["batches"], st["refresh_batches"],
                        st["spec_batches"]))
            assert np.array_equal(s1, seeds[:7])
    (sg, gg, eg, bg, rg, _), (sh, gh, eh, bh, rh, _) = got
    assert np.array_equal(sg, o_seeds) and np.array_equal(gg, o_gains)
    assert np.array_equal(sh, sg) and np.array_equal(gh, gg)
    assert np.array_equal(eg, eh) and bg == bh and rg == rh
    if threshold == 1:
        assert rg + got[0][5] == bg > 0     # every batch but a speculative round 1 refreshes
    if threshold == 2**64 - 1:
        assert rg == 0


def test_rebuilds_in_one_context_match_fresh_contexts():
    """Builds that reuse the device buffers and the selection graph (same shapes, same
    sampler), re-capture the graph (new seed) or re-allocate (new p, R, alpha) all give the
    results of a fresh context; the last configuration is also checked against the oracle."""
    n, u, v = graphgen.erdos_renyi(2000, 8000, 12)
    cfgs = [(42, 0.1, 50, 0.2), (42, 0.1, 50, 0.2), (7, 0.1, 50, 0.2), (7, 0.3, 50, 0.2),
            (7, 0.3, 64, 0.05)]
    k = 8
    with im.IMContext(n, u, v) as ctx:
        for seed, p, R, alpha in cfgs:
            ctx.build_sketches(R, seed, p, alpha)
            got = ctx.select_seeds(k) + ctx.compact() + (ctx.gains(),)
            with im.IMContext(n, u, v) as fresh:
                fresh.build_sketches(R, seed, p, alpha)
                want = fresh.select_seeds(k) + fresh.compact() + (fresh.gains(),)
            for a, b in zip(got, want):
                assert np.array_equal(a, b), (seed, p, R, alpha)
    o = _oracle(n, u, v, 7, 0.3, 64, 0.05, k)
    assert np.array_equal(got[0], o["seeds"]) and np.array_equal(got[1], o["seed_gains"])
    assert np.array_equal(got[2], o["label"]) and np.array_equal(got[3], o["size"])


@pytest.mark.parametrize("graph", ["chunglu", "er"])
@pytest.mark.parametrize("candidates", [0, 1, 4, 8])
@pytest.mark.parametrize("lanes", [1, 2])
def test_first_seed_speculation_gives_the_same_selection(candidates, graph, lanes):
    """Round 1's batches evaluated from the build's overlap sums of candidate first seeds (the
    vertices with the largest gains over the first batch of 32 sketches) give the plain
    selection, with the same batches and evaluation counts; the speculation is used exactly
    when the first seed is among the candidates (computed here from the oracle's labels).
    On the Chung-Lu graph the hubs tie at the top and the smallest id wins, as in the full
    argmax; on the Erdos-Renyi graph the first seed ranks third, so one candidate misses it.
    With two lanes (R = 128: two batches per lane) lane 1 waits for the candidates and sums its
    overlaps apart."""
    R = 64 if lanes == 1 else 128
    if graph == "chunglu":
        n, u, v = graphgen.chung_lu(20000, 100000, 2.1, 2000.0, 5)
    else:
        n, u, v = graphgen.erdos_renyi(2000, 10000, 7)
    G = oracle.Graph(n, u, v)
    L = G.labels(42, 0.05, R)
    o_seeds, o_gains = oracle.greedy(L, 8)
    g32 = oracle.gains(L[:32]).astype(np.int64)
    cand = np.lexsort((np.arange(n), -g32))[:candidates]
    hit = bool(np.isin(o_seeds[0], cand))
    with im.IMContext(n, u, v) as ctx:
        im.im_set_seed_speculation(ctx.h, candidates)
        im.im_set_pipeline(ctx.h, lanes)
        ctx.build_sketches(R, 42, 0.05, 0.1)
        assert ctx.stats()["sketch_batch"] == 32
        s1, g1 = ctx.select_seeds(2)                 # through round 1, then the rest
        seeds, gains = ctx.select_seeds(8)
        st = ctx.stats()
        ev = ctx.round_evals()
    with im.IMContext(n, u, v) as ref:
        im.im_set_seed_speculation(ref.h, 0)
        ref.build_sketches(R, 42, 0.05, 0.1)
        ref.select_seeds(8)
        assert np.array_equal(ev, ref.round_evals()) and st["batches"] == ref.stats()["batches"]
    assert np.array_equal(s1, seeds[:2])
    assert np.array_equal(seeds, o_seeds) and np.array_equal(gains, o_gains)
    assert (st["spec_batches"] > 0) == hit
    if lanes == 1:
        assert hit == (candidates >= (1 if graph == "chunglu" else 3))
    with pytest.raises(im.IMError) as e:
        with im.IMContext(n, u, v) as ctx:
            im.im_set_seed_speculation(ctx.h, 9)
    assert e.value.code == im.IM_EINVAL


def test_page_locked_host_lists_are_read_in_place():
    """Edge lists in page-locked host memory (torch pin_memory) are read by the packing kernel
    where they are, without a staging copy: the results equal the oracle's, for a new context
    and for a graph loaded into an existing one; a bad id in such a list is still refused."""
    n, u, v = graphgen.erdos_renyi(1500, 6001, 3)
    pu = torch.from_numpy(u.view(np.int32)).pin_memory()
    pv = torch.from_numpy(v.view(np.int32)).pin_memory()
    o = _oracle(n, u, v, 42, 0.1, 45, 0.2, 5)
    with im.IMContext(n, pu, pv) as ctx:
        ctx.build_sketches(45, 42, 0.1, 0.2)
        s1, g1 = ctx.select_seeds(5)
        n2, u2, v2 = graphgen.erdos_renyi(900, 5000, 5)
        ctx.load_graph(n2, torch.from_numpy(u2.view(np.int32)).pin_memory(),
                       torch.from_numpy(v2.view(np.int32)).pin_memory())
        ctx.build_sketches(45, 42, 0.1, 0.2)
        s2, g2 = ctx.select_seeds(5)
        bad = pv.clone().pin_memory()
        bad[17] = n + 3
        with pytest.raises(im.IMError) as e:
            ctx.load_graph(n, pu, bad)
        assert e.value.code == im.IM_EINVAL
    assert np.array_equal(s1, o["seeds"]) and np.array_equal(g1, o["seed_gains"])
    o2 = _oracle(n2, u2, v2, 42, 0.1, 45, 0.2, 5)
    assert np.array_equal(s2, o2["seeds"]) and np.array_equal(g2, o2["seed_gains"])


def test_load_graph_serves_one_graph_after_another():
    """One context, several graphs (same n and m: buffers and selection graph reused; other
    sizes: reallocated; host and device edge lists): each gives the results of a fresh
    context.  A failed load leaves no graph (IM_ESTATE) until a good one is loaded."""
    graphs = [graphgen.erdos_renyi(1500, 6001, 3), graphgen.erdos_renyi(1500, 6001, 4),
              graphgen.erdos_renyi(900, 5000, 5), graphgen.erdos_renyi(1500, 6001, 3)]
    R, seed, p, alpha, k = 45, 42, 0.1, 0.2, 5

    def results(ctx):
        return ctx.select_seeds(k) + ctx.compact() + (ctx.gains(), np.array([ctx.spread(np.arange(3))]))

    n0, u0, v0 = graphs[0]
    with im.IMContext(n0, u0, v0) as ctx:
        for i, (n, u, v) in enumerate(graphs):
            if i % 2:
                ctx.load_graph(n, torch.from_numpy(u.view(np.int32)).cuda(), torch.from_numpy(v.view(np.int32)).cuda())
            else:
                ctx.load_graph(n, u, v)
            with pytest.raises(im.IMError) as e:
                ctx.select_seeds(1)
            assert e.value.code == im.IM_ESTATE
            ctx.build_sketches(R, seed, p, alpha)
            got = results(ctx)
            with im.IMContext(n, u, v) as fresh:
                fresh.build_sketches(R, seed, p, alpha)
                want = results(fresh)
            for a, b in zip(got, want):
                assert np.array_equal(a, b), i
        o = _oracle(*graphs[-1], seed, p, R, alpha, k)
        assert np.array_equal(got[0], o["seeds"]) and np.array_equal(got[1], o["seed_gains"])
        with pytest.raises(im.IMError) as e:
            ctx.load_graph(4, np.array([0, 7], np.uint32), np.array([1, 2], np.uint32))
        assert e.value.code == im.IM_EINVAL
        with pytest.raises(im.IMError) as e:
            ctx.build_sketches(R, seed, p, alpha)
        assert e.value.code == im.IM_ESTATE
        ctx.load_graph(n0, u0, v0)
        ctx.build_sketches(R, seed, p, alpha)
        assert np.array_equal(ctx.select_seeds(k)[0], got[0])


# ---- per-edge IC probabilities (Sec. 2's IC model: each edge its own p_e) -------------------

def _edge_probs(model, G, m):
    if model == "wic":
        return G.set_wic()
    lo, hi = (0.0, 0.1) if model == "u01" else (0.1, 0.3)
    p = np.random.default_rng(17).uniform(lo, hi, m)
    G.set_probs(p)
    return p


@pytest.mark.parametrize("threshold", [0, 1, 2**64 - 1])
@pytest.mark.parametrize("alpha", [1.0, 0.1])
@pytest.mark.parametrize("model", ["u01", "u13", "wic"])
def test_per_edge_probabilities_match_the_oracle(model, alpha, threshold):
    """Uniform U(0,0.1), U(0.1,0.3) (the array passed to both sides) and the weighted cascade
    2/(d_u+d_v) (computed by each side): labels, gains, compact sketches, seeds, gains and
    spread bit for bit; threshold 1 / 2^64-1 force each batch evaluator, 0 is automatic."""
    n, u, v = graphgen.chung_lu(20000, 100000, 2.1, 2000.0, 5)
    G = oracle.Graph(n, u, v)
    p = _edge_probs(model, G, len(u))
    R, seed, k = 64, 42, 10
    L = G.labels(seed, -1.0, R, mode=oracle.MODE_EDGE)
    ctr = oracle.centers(n, seed, alpha)
    lab, sz = oracle.compact(L, ctr)
    o_seeds, o_gains = oracle.greedy(L, k)
    with im.IMContext(n, u, v) as ctx:
        if model == "wic":
            ctx.set_edge_probs(im.IM_PROBS_WIC)
        else:
            ctx.set_edge_probs(im.IM_PROBS_ARRAY, p)
        im.im_set_refresh_threshold(ctx.h, threshold)
        ctx.build_sketches(R, seed, 0.5, alpha)          # p is ignored under per-edge models
        for r in (0, 31, 63):
            assert np.array_equal(ctx.labels(r), L[r]), r
        assert np.array_equal(ctx.gains(), oracle.gains(L))
        g_lab, g_sz = ctx.compact()
        assert np.array_equal(g_lab, lab) and np.array_equal(g_sz, sz)
        seeds, gains = ctx.select_seeds(k)
        assert np.array_equal(seeds, o_seeds) and np.array_equal(gains, o_gains)
        assert ctx.spread(seeds) == oracle.spread(L, seeds) == int(o_gains.sum())


@pytest.mark.parametrize("path", [0, 1, 2])
@pytest.mark.parametrize("model", ["u13", "wic"])
def test_per_edge_probabilities_on_every_union_path(model, path):
    """The per-edge thresholds through each union path (the bucketed sampler reads them in
    pairs with the edges, as the others do): equal to the oracle."""
    n, u, v = graphgen.chung_lu(20000, 100000, 2.1, 2000.0, 6)
    G = oracle.Graph(n, u, v)
    p = _edge_probs(model, G, len(u))
    R, seed, k, alpha = 40, 43, 8, 0.1
    L = G.labels(seed, -1.0, R, mode=oracle.MODE_EDGE)
    ctr = oracle.centers(n, seed, alpha)
    lab, sz = oracle.compact(L, ctr)
    o_seeds, o_gains = oracle.greedy(L, k)
    with im.IMContext(n, u, v) as ctx:
        im.im_set_union_path(ctx.h, path)
        if model == "wic":
            ctx.set_edge_probs(im.IM_PROBS_WIC)
        else:
            ctx.set_edge_probs(im.IM_PROBS_ARRAY, p)
        ctx.build_sketches(R, seed, 0.5, alpha)
        assert ctx.stats()["union_path"] == path
        for r in (0, 39):
            assert np.array_equal(ctx.labels(r), L[r]), r
        assert np.array_equal(ctx.gains(), oracle.gains(L))
        g_lab, g_sz = ctx.compact()
        assert np.array_equal(g_lab, lab) and np.array_equal(g_sz, sz)
        seeds, gains = ctx.select_seeds(k)
        assert np.array_equal(seeds, o_seeds) and np.array_equal(gains, o_gains)


@pytest.mark.parametrize("path", [0, 1, 2])
def test_p_zero_and_p_one_on_every_union_path(path):
    # no live edge, and every edge live (all pairs become records: the record paths' capacity
    # is sized for it), through each union path
    n, u, v = graphgen.erdos_renyi(700, 2100, 8)
    for p in (0.0, 1.0):
        g = _run_path(n, u, v, 42, p, 33, 0.25, 4, path)
        o = _oracle(n, u, v, 42, p, 33, 0.25, 4)
        _compare(g, o, 4)


def test_per_edge_probability_api():
    n, u, v = graphgen.erdos_renyi(2000, 8000, 21)
    R, seed, p0 = 32, 9, 0.15
    with im.IMContext(n, u, v) as ctx:
        ctx.build_sketches(R, seed, p0, 0.2)
        want = (ctx.gains(),) + ctx.compact() + ctx.select_seeds(6)
        # the same probability on every edge, from the host and from the device, is the uniform model
        for arr in (np.full(len(u), p0), torch.full((len(u),), p0, dtype=torch.float64, device="cuda")):
            ctx.set_edge_probs(im.IM_PROBS_ARRAY, arr)
            with pytest.raises(im.IMError) as e:
                ctx.select_seeds(1)
            assert e.value.code == im.IM_ESTATE
            ctx.build_sketches(R, seed, 0.9, 0.2)
            got = (ctx.gains(),) + ctx.compact() + ctx.select_seeds(6)
            for a, b in zip(got, want):
                assert np.array_equal(a, b)
        # back to one p; a new graph also returns to it
        ctx.set_edge_probs(im.IM_PROBS_UNIFORM)
        ctx.build_sketches(R, seed, p0, 0.2)
        assert np.array_equal(ctx.select_seeds(6)[0], want[3])
        ctx.set_edge_probs(im.IM_PROBS_WIC)
        ctx.load_graph(n, u, v)
        ctx.build_sketches(R, seed, p0, 0.2)
        assert np.array_equal(ctx.select_seeds(6)[0], want[3])
        with pytest.raises(im.IMError) as e:
            im.im_set_edge_probs(ctx.h, 7)
        assert e.value.code == im.IM_EINVAL
        with pytest.raises(im.IMError) as e:
            im.im_set_edge_probs(ctx.h, im.IM_PROBS_ARRAY, None)
        assert e.value.code == im.IM_EINVAL


# ---- hubs: high-degree non-centers with label rows of their own (search shortcut) -------------

@pytest.mark.parametrize("threshold", [1, 2**64 - 1])
@pytest.mark.parametrize("model", ["uniform", "wic"])
@pytest.mark.parametrize("hubs", [(0, 32), (im.IM_HUBS_AUTO, 32), (7, 1), (2**31, 1)])
def test_hubs_change_no_value(hubs, model, threshold):
    """Seeds, gains, spread and the compact sketch are the oracle's with no hubs, the automatic
    set, a handful, and every non-center a hub; both batch evaluators; the hub count is
    min(cap, non-centers of degree >= min_degree)."""
    n, u, v = graphgen.chung_lu(20000, 100000, 2.1, 2000.0, 5)
    G = oracle.Graph(n, u, v)
    R, seed, k, alpha, p = 64, 42, 12, 0.05, 0.03
    if model == "wic":
        G.set_wic()
        L = G.labels(seed, -1.0, R, mode=oracle.MODE_EDGE)
    else:
        L = G.labels(seed, p, R)
    ctr = oracle.centers(n, seed, alpha)
    lab, sz = oracle.compact(L, ctr)
    o_seeds, o_gains = oracle.greedy(L, k)
    deg = np.bincount(np.concatenate([u, v]), minlength=n)
    noncenter = np.ones(n, bool)
    noncenter[ctr] = False
    cap = max(1024, n // 64) if hubs[0] == im.IM_HUBS_AUTO else hubs[0]
    want_hubs = min(cap, int((noncenter & (deg >= hubs[1])).sum()))
    sets = [o_seeds[:3], np.argsort(-deg)[:40].astype(np.uint32), np.arange(0, n, 97, dtype=np.uint32)]
    with im.IMContext(n, u, v) as ctx:
        if model == "wic":
            ctx.set_edge_probs(im.IM_PROBS_WIC)
        im.im_set_hubs(ctx.h, *hubs)
        im.im_set_refresh_threshold(ctx.h, threshold)
        ctx.build_sketches(R, seed, p, alpha)
        g_lab, g_sz = ctx.compact()
        assert np.array_equal(g_lab, lab) and np.array_equal(g_sz, sz)
        seeds, gains = ctx.select_seeds(k)
        assert np.array_equal(seeds, o_seeds) and np.array_equal(gains, o_gains)
        for s in sets:
            assert ctx.spread(s) == oracle.spread(L, s)
        assert ctx.stats()["hubs"] == want_hubs
        # the selection again after a reset (hub rows' covered flags are cleared too)
        ctx.reset_selection()
        seeds2, gains2 = ctx.select_seeds(k)
        assert np.array_equal(seeds2, o_seeds) and np.array_equal(gains2, o_gains)


# ---- Monte-Carlo influence evaluator (the paper's quality measure) ---------------------------

@pytest.mark.parametrize("alpha", [1.0, 0.1])
@pytest.mark.parametrize("model", ["uniform", "wic", "u13"])
def test_mc_spread_matches_the_oracle(model, alpha):
    """Sum over simulations of the vertices reachable from the seeds = the oracle's spread over
    the live-edge worlds of the simulation hash seed; ragged simulation counts, duplicates,
    the empty set; the build's own seed gives back the sketches' spread; the sketches are
    untouched (the selection continues as the oracle's)."""
    n, u, v = graphgen.chung_lu(20000, 100000, 2.1, 2000.0, 5)
    G = oracle.Graph(n, u, v)
    R, seed, k, p = 64, 42, 12, 0.03
    mode = oracle.MODE_HASH
    if model == "wic":
        G.set_wic()
        mode = oracle.MODE_EDGE
    elif model == "u13":
        parr = np.random.default_rng(5).uniform(0.1, 0.3, len(u))
        G.set_probs(parr)
        mode = oracle.MODE_EDGE
    L = G.labels(seed, p, R, mode=mode)
    o_seeds, o_gains = oracle.greedy(L, k)
    with im.IMContext(n, u, v) as ctx:
        with pytest.raises(im.IMError) as e:
            ctx.mc_spread([0], 4, 1)
        assert e.value.code == im.IM_ESTATE
        if model == "wic":
            ctx.set_edge_probs(im.IM_PROBS_WIC)
        elif model == "u13":
            ctx.set_edge_probs(im.IM_PROBS_ARRAY, parr)
        ctx.build_sketches(R, seed, p, alpha)
        seeds, gains = ctx.select_seeds(6)
        for sims, mc_seed in ((1, 7), (37, 7), (300, 11)):
            Lm = G.labels(mc_seed, p, sims, mode=mode)
            assert ctx.mc_spread(seeds, sims, mc_seed) == oracle.spread(Lm, seeds), (sims, mc_seed)
        L37 = G.labels(7, p, 37, mode=mode)
        dup = np.concatenate([seeds[:3], seeds[:3], [int(seeds[0])]])
        assert ctx.mc_spread(dup, 37, 7) == oracle.spread(L37, seeds[:3])
        assert ctx.mc_spread(np.array([], np.uint32), 37, 7) == 0
        assert ctx.mc_spread(seeds, 0, 7) == 0
        assert ctx.mc_spread(seeds, R, seed) == ctx.spread(seeds)
        with pytest.raises(im.IMError) as e:
            ctx.mc_spread([n], 4, 1)
        assert e.value.code == im.IM_EINVAL
        seeds, gains = ctx.select_seeds(k)   # continues after the evaluations
        assert np.array_equal(seeds, o_seeds) and np.array_equal(gains, o_gains)


# ---- many instances at once (the batched workload) --------------------------------------------

def _one_by_one(d):
    with im.IMContext(d["n"], d["u"], d["v"]) as ctx:
        ctx.build_sketches(d["R"], d["seed"], d["p"], d["alpha"])
        seeds, gains = ctx.select_seeds(d["k"])
        return seeds, gains, ctx.spread(seeds)


def test_run_batch_matches_one_by_one_and_the_oracle():
    """Instances of the batched workload's recipe (smaller n), run by 3 workers concurrently:
    seeds, gains and spread equal those of separate contexts; the two smallest against the
    oracle."""
    inst = graphgen.c4_instances(8, first_seed=1000, n_range=(2e3, 3e4))
    got = im.im_run_batch(inst, workers=3)
    for d, (s, g, sp) in zip(inst, got):
        s1, g1, sp1 = _one_by_one(d)
        assert np.array_equal(s, s1) and np.array_equal(g, g1) and sp == sp1
    for i in sorted(range(len(inst)), key=lambda i: inst[i]["n"])[:2]:
        d = inst[i]
        L = oracle.Graph(d["n"], d["u"], d["v"]).labels(d["seed"], d["p"], d["R"])
        o_seeds, o_gains = oracle.greedy(L, d["k"])
        assert np.array_equal(got[i][0], o_seeds) and np.array_equal(got[i][1], o_gains)
        assert got[i][2] == oracle.spread(L, o_seeds)
    # errors: a bad instance reports its own status, the others still run
    bad = dict(inst[0])
    bad["k"] = bad["n"] + 1
    with pytest.raises(im.IMError):
        im.im_run_batch([inst[1], bad], workers=2)


def test_one_context_across_graph_sizes():
    """A context that loads larger, smaller and mid-sized graphs in turn (its buffers reused
    while they fit, the selection graph rebuilt) gives what fresh contexts give."""
    graphs = [graphgen.chung_lu(30000, 150000, 2.1, 3000.0, 11), graphgen.erdos_renyi(5000, 20000, 12),
              graphgen.chung_lu(20000, 90000, 2.1, 2000.0, 13), graphgen.chung_lu(30000, 150000, 2.1, 3000.0, 11)]
    params = [(64, 3, 0.04, 0.1, 8), (128, 4, 0.1, 1.0, 5), (32, 5, 0.02, 0.05, 12), (96, 6, 0.03, 0.2, 7)]
    n0, u0, v0 = graphs[0]
    with im.IMContext(n0, u0, v0) as ctx:
        for (n, u, v), (R, seed, p, alpha, k) in zip(graphs, params):
            ctx.load_graph(n, u, v)
            ctx.build_sketches(R, seed, p, alpha)
            s, g = ctx.select_seeds(k)
            sp = ctx.spread(s)
            lab, sz = ctx.compact()
            with im.IMContext(n, u, v) as fresh:
                fresh.build_sketches(R, seed, p, alpha)
                s1, g1 = fresh.select_seeds(k)
                assert np.array_equal(s, s1) and np.array_equal(g, g1) and sp == fresh.spread(s1)
                lab1, sz1 = fresh.compact()
                assert np.array_equal(lab, lab1) and np.array_equal(sz, sz1)


# ---- serving: resident models answering requests for k seeds -----------------------------------

def test_server_answers_are_greedy_prefixes():
    """Requests replayed at their arrival times on three resident models: every answer is the
    first k seeds (and gains) of the model's greedy sequence computed alone, its spread the
    sum of those gains (= the spread of the k seeds); one model against the oracle."""
    graphs = [graphgen.chung_lu(20000, 100000, 2.1, 2000.0, 21), graphgen.erdos_renyi(8000, 30000, 22),
              graphgen.chung_lu(12000, 60000, 2.1, 1500.0, 23)]
    params = [(64, 5, 0.03, 0.1), (32, 6, 0.08, 1.0), (48, 7, 0.05, 0.05)]
    rng = np.random.default_rng(3)
    reqs = [(int(rng.integers(0, 3)), int(rng.integers(1, 40)), int(t)) for t in np.cumsum(rng.exponential(2e6, 80))]
    with im.IMServer() as srv:
        for (n, u, v), (R, seed, p, alpha) in zip(graphs, params):
            mid, fp = srv.add_model(n, u, v, R, seed, p, alpha)
            assert fp > 0
        out = srv.replay(reqs)
        with pytest.raises(im.IMError) as e:
            srv.replay([(3, 5, 0)])
        assert e.value.code == im.IM_EINVAL
    kmax = [max([k for m, k, _ in reqs if m == i] + [1]) for i in range(3)]
    alone = []
    for (n, u, v), (R, seed, p, alpha), k in zip(graphs, params, kmax):
        with im.IMContext(n, u, v) as ctx:
            ctx.build_sketches(R, seed, p, alpha)
            s, g = ctx.select_seeds(k)
            alone.append((s, g, ctx))
            for (m, kk, _), o in zip(reqs, out):
                if m == len(alone) - 1:
                    assert np.array_equal(o["seeds"], s[:kk]) and np.array_equal(o["gains"], g[:kk])
                    assert o["spread"] == int(g[:kk].sum()) == ctx.spread(s[:kk])
                    assert o["done_ns"] >= o["submit_ns"]
    n, u, v = graphs[1]
    L = oracle.Graph(n, u, v).labels(params[1][1], params[1][2], params[1][0])
    o_seeds, o_gains = oracle.greedy(L, kmax[1])
    assert np.array_equal(alone[1][0], o_seeds) and np.array_equal(alone[1][1], o_gains)
