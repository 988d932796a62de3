"""GPU path vs the CPU oracle, element by element, through the C ABI.

All arithmetic is integer, so the bar is bit-exact: same labels after every
label-propagation round, same contracted CSR, same Padberg-Rinaldi and
Nagamochi-Ono-Ibaraki merges, same cut value, same side bitmap and the same trace of
(n, nnz, lambda-hat) after every contraction step.
"""
import random

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1708_06127_gb300 as vc
from tests import helpers as H

pytestmark = pytest.mark.gpu
BIG_N0 = 1 << 40


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    vc.build()
    vc.lib()


def gpu_run(g, seed=1, lp=2, n0=10000, pr=8):
    with vc.MinCut(g.offsets, g.adj, g.w, n0=n0, pr_runs_max=pr, validate=2) as mc:
        cut, bits = mc.run(seed, lp)
        trace = mc.trace()
    return cut, bits, trace


def assert_same(g, seed=1, lp=2, n0=10000, pr=8):
    ref = oracle.viecut(g.offsets, g.adj, g.w, seed=seed, lp_iters=lp, n0=n0, pr_runs_max=pr)
    cut, bits, trace = gpu_run(g, seed, lp, n0, pr)
    assert trace == ref.trace, (g.name, seed, lp, n0)
    assert cut == ref.cut, (g.name, seed, lp, n0)
    assert np.array_equal(bits, ref.side_bits), (g.name, seed, lp, n0)
    return ref


def hub_graph(seed=5):
    """ER background plus vertices of degree 3000 and 1500 (block class: 513 to 4096
    entries, a shared-memory table), 700 (block class) and 200 (warp class); weights in
    [1, 9]."""
    rnd = random.Random(seed)
    n = 6000
    base = gg.er(n, 6, seed, 1, 9)
    E = {}
    for v in range(n):
        for e in range(base.offsets[v], base.offsets[v + 1]):
            u = int(base.adj[e])
            if v < u:
                E[(v, u)] = int(base.w[e])
    for hub, deg in [(0, 3000), (1, 1500), (2, 700), (3, 200)]:
        for u in rnd.sample(range(4, n), deg):
            E[(hub, u)] = rnd.randint(1, 9)
    return gg.from_edges(n, [(a, b, w) for (a, b), w in E.items()], "hubs")


def giant_hub_graph(unit: bool, parallel: bool = False, seed: int = 7):
    """ER background (n = 40000, average degree 6) plus hubs of degree 5000, 12000 and
    20000 -- lists above 4096 entries, the global-table class (a hash table in global
    memory per block) -- and one of 3000 (block class).  Weights in [1, 9], or all 1.
    parallel: every hub edge to an even neighbour is listed twice (parallel entries, so
    the lists are not strictly increasing and the first round cannot take the
    no-aggregation path)."""
    rnd = random.Random(seed)
    n = 40000
    base = gg.er(n, 6, seed, 1, 9)
    E = {}
    for v in range(n):
        for e in range(base.offsets[v], base.offsets[v + 1]):
            u = int(base.adj[e])
            if v < u:
                E[(v, u)] = 1 if unit else int(base.w[e])
    for hub, deg in [(0, 20000), (1, 12000), (2, 5000), (3, 3000)]:
        for u in rnd.sample(range(4, n), deg):
            E[(hub, u)] = 1 if unit else rnd.randint(1, 9)
    edges = [(a, b, w) for (a, b), w in E.items()]
    if parallel:
        edges += [(a, b, w) for (a, b, w) in edges if a < 4 and b % 2 == 0]
    g = gg.core_lcc(gg.from_edges(n, edges), 3)  # 3-core, largest component
    return gg.Graph(g.offsets, g.adj, g.w, f"giant-hubs(unit={unit},parallel={parallel})")


def multi_edge_graph():
    E = [(0, 1, 2), (0, 1, 3), (1, 2, 1), (2, 3, 4), (2, 3, 4), (3, 0, 1), (1, 3, 2), (0, 2, 1), (2, 0, 5)]
    return gg.from_edges(4, E, "parallel-edges")


# ------------------------------------------------------------------ step parity
STEP_GRAPHS = {
    "rhg14": lambda: gg.workload_rhg_small(1),
    "rhg12w": lambda: gg.with_pair_weights(gg.core_lcc(gg.rhg(1 << 12, 20, 7), 0), 7, 1, 50),
    "er_w100": lambda: gg.er(3000, 12, 3, 1, 100),
    "hubs": hub_graph,
}


@pytest.fixture(scope="module")
def step_graphs():
    return {k: f() for k, f in STEP_GRAPHS.items()}


def upload(G):
    return vc.viecut_graph_upload(G.offsets, G.adj, G.w)


@pytest.mark.parametrize("name", list(STEP_GRAPHS))
def test_degrees_parity(step_graphs, name):
    g = step_graphs[name]
    G = oracle.as_csr64(g.offsets, g.adj, g.w)
    d = upload(G)
    try:
        assert np.array_equal(vc.viecut_step_degrees(d), oracle.degrees(G))
    finally:
        vc.viecut_graph_free(d)


@pytest.mark.parametrize("name", list(STEP_GRAPHS))
def test_lp_rounds_parity(step_graphs, name):
    g = step_graphs[name]
    G = oracle.as_csr64(g.offsets, g.adj, g.w)
    d = upload(G)
    try:
        for seed, level in [(1, 0), (77, 3)]:
            key = oracle.level_key(seed, level)
            got = vc.viecut_step_lp(d, None, key, 3)
            lab = np.arange(G.n, dtype=np.int32)
            for r in range(3):
                lab = oracle.lp_round(G, lab, key)
                assert np.array_equal(got[r], lab), (name, seed, r)
        # from arbitrary labels (coarse clusters), as later rounds see them
        rnd = np.random.default_rng(3)
        lab0 = rnd.integers(0, max(2, G.n // 50), G.n).astype(np.int32)
        key = oracle.level_key(5, 1)
        got = vc.viecut_step_lp(d, lab0, key, 2)
        l1 = oracle.lp_round(G, lab0, key)
        assert np.array_equal(got[0], l1)
        assert np.array_equal(got[1], oracle.lp_round(G, l1, key))
    finally:
        vc.viecut_graph_free(d)


def list_shapes_graph():
    """Unit weights, strictly increasing lists of many shapes: a star of 1024 leaves, a
    path (two entries per list), isolated vertices, and a star of 2999 leaves (block
    class) with a few chords between its leaves."""
    n = 6000
    E = {(0, u) for u in range(1, 1025)}
    E |= {(u, u + 1) for u in range(1100, 2100)}
    E |= {(2200, u) for u in range(3001, 6000)}
    rnd = random.Random(11)
    E |= {tuple(sorted(rnd.sample(range(3001, 6000), 2))) for _ in range(400)}
    return gg.from_edges(n, [(a, b, 1) for (a, b) in sorted(E)], "list-shapes")


@pytest.mark.parametrize("name", ["shapes", "er_sparse", "giant_hubs"])
def test_first_round_unit_list_shapes_parity(name):
    """The first round from the identity on unit-weight graphs (the simple-list kernels:
    one vertex per lane group, a block per list above 4096 entries; isolated vertices keep
    their own label), and the second round after it, equal the oracle's rounds."""
    g = {"shapes": list_shapes_graph, "er_sparse": lambda: gg.er(20000, 2.5, 11),
         "giant_hubs": lambda: giant_hub_graph(True)}[name]()
    G = oracle.as_csr64(g.offsets, g.adj, g.w)
    assert (G.w == 1).all()
    d = upload(G)
    try:
        for seed, level in [(1, 0), (9, 2)]:
            key = oracle.level_key(seed, level)
            got = vc.viecut_step_lp(d, None, key, 2)
            l1 = oracle.lp_round(G, np.arange(G.n, dtype=np.int32), key)
            assert np.array_equal(got[0], l1), (name, seed)
            assert np.array_equal(got[1], oracle.lp_round(G, l1, key)), (name, seed)
    finally:
        vc.viecut_graph_free(d)


def test_unaligned_caller_ids():
    """Caller-owned device ids that start 4 bytes past a 16-byte boundary (valid for
    int32): the whole run equals the oracle's."""
    import torch
    g = gg.workload_rhg_small(2)
    dev = torch.device("cuda:0")
    off = torch.from_numpy(g.offsets).to(dev)
    buf = torch.zeros(g.nnz + 1, dtype=torch.int32, device=dev)
    buf[1:] = torch.from_numpy(g.adj).to(dev)
    adj = buf[1:]
    assert adj.data_ptr() % 16 == 4
    w = torch.from_numpy(g.w).to(dev)
    ref = oracle.viecut(g.offsets, g.adj, g.w, seed=3, lp_iters=2, n0=10000)
    with vc.MinCut(off, adj, w, on_device=True) as mc:
        cut, bits = mc.run(3, 2)
    assert cut == ref.cut and np.array_equal(bits, ref.side_bits)


def compare_contract(G, labels):
    d = upload(G)
    out = None
    try:
        out, cid = vc.viecut_step_contract(d, labels)
        off, adj, w = vc.viecut_graph_download(out)
        ref, rcid = oracle.contract(G, labels)
        assert np.array_equal(cid, rcid)
        assert np.array_equal(off, ref.offsets)
        assert np.array_equal(adj, ref.adj)
        assert np.array_equal(w, ref.w)
        return ref
    finally:
        vc.viecut_graph_free(d)
        vc.viecut_graph_free(out)


@pytest.mark.parametrize("name", list(STEP_GRAPHS))
def test_contract_parity(step_graphs, name):
    g = step_graphs[name]
    G = oracle.as_csr64(g.offsets, g.adj, g.w)
    rnd = np.random.default_rng(11)
    # clusterings from label propagation, random with few / many clusters, identity, and
    # the identity with a tenth of the vertices relabelled at random (most vertices alone
    # under their own id: the sparse contraction, with singletons under another id)
    key = oracle.level_key(2, 0)
    lp = oracle.lp_round(G, oracle.lp_round(G, np.arange(G.n, dtype=np.int32), key), key)
    near = np.arange(G.n)
    moved = rnd.choice(G.n, G.n // 10, replace=False)
    near[moved] = rnd.integers(0, G.n, len(moved))
    for labels in [lp, rnd.integers(0, 7, G.n), rnd.integers(0, G.n, G.n), np.arange(G.n),
                   np.zeros(G.n, np.int64), near]:
        compare_contract(G, labels.astype(np.int32))


def test_contract_giant_clusters():
    """A few clusters of more than 4096 pre-merged pairs beside many small ones: the
    small ones take the per-cluster merge, the giant ones one shared radix sort; both
    with mostly singleton clusters and with clusters of four vertices."""
    g = gg.er(30000, 12, 5, 1, 100)
    G = oracle.as_csr64(g.offsets, g.adj, g.w)
    n = G.n
    v = np.arange(n, dtype=np.int64)
    rnd = np.random.default_rng(4)
    perm = rnd.permutation(n)
    giant = np.full(n, -1, np.int64)
    for k, lab in enumerate((perm[0], perm[1], 7)):  # three giant clusters, scattered members
        giant[perm[2 + 800 * k: 2 + 800 * (k + 1)]] = lab
    for rest in (v, v // 4):
        labels = np.where(giant >= 0, giant, rest)
        compare_contract(G, labels.astype(np.int32))


@pytest.mark.parametrize("unit,parallel", [(True, False), (False, False), (True, True)])
def test_global_table_class_parity(unit, parallel):
    """Lists of 5000 to 20000 entries take the global-table kernels: the first round on
    strictly increasing lists (lp_first_simple_block_k), later rounds and first rounds on
    lists with parallel entries (lp_block_k with a global table), and the contraction's
    pre-merge (emit_block_k).  Labels after rounds 1 and 2 (from the identity and from
    arbitrary labels) and the contracted CSR equal the oracle's element by element."""
    g = giant_hub_graph(unit, parallel)
    assert np.diff(g.offsets).max() > 4096 * 4
    G = oracle.as_csr64(g.offsets, g.adj, g.w)
    d = upload(G)
    try:
        for seed, level in [(1, 0), (9, 2)]:
            key = oracle.level_key(seed, level)
            got = vc.viecut_step_lp(d, None, key, 2)
            lab = np.arange(G.n, dtype=np.int32)
            for r in range(2):
                lab = oracle.lp_round(G, lab, key)
                assert np.array_equal(got[r], lab), (g.name, seed, r)
        rnd = np.random.default_rng(5)
        lab0 = rnd.integers(0, 64, G.n).astype(np.int32)
        key = oracle.level_key(4, 1)
        got = vc.viecut_step_lp(d, lab0, key, 2)
        l1 = oracle.lp_round(G, lab0, key)
        assert np.array_equal(got[0], l1) and np.array_equal(got[1], oracle.lp_round(G, l1, key))
    finally:
        vc.viecut_graph_free(d)
    key = oracle.level_key(1, 0)
    lp = oracle.lp_round(G, oracle.lp_round(G, np.arange(G.n, dtype=np.int32), key), key)
    for labels in [lp, np.arange(G.n), rnd.integers(0, 2000, G.n)]:
        compare_contract(G, labels.astype(np.int32))
    assert_same(g, seed=2, lp=2, n0=16)


def test_step_entry_points_refuse_labels_outside_the_vertex_range():
    G = oracle.as_csr64(*(lambda g: (g.offsets, g.adj, g.w))(H.cycle(10)))
    d = upload(G)
    try:
        for bad in (np.full(G.n, G.n, np.int32), np.full(G.n, -1, np.int32)):
            with pytest.raises(vc.ViecutError) as e:
                vc.viecut_step_contract(d, bad)
            assert e.value.code == vc.VIECUT_EINVAL and "outside" in str(e.value)
            with pytest.raises(vc.ViecutError) as e:
                vc.viecut_step_lp(d, bad, 1, 1)
            assert e.value.code == vc.VIECUT_EINVAL
    finally:
        vc.viecut_graph_free(d)


def coarse_graphs():
    out = []
    for seed in range(4):
        g = gg.with_pair_weights(gg.core_lcc(gg.rhg(1 << 11, 16, 40 + seed), 0), seed, 1, 5 + 10 * seed)
        G = oracle.as_csr64(g.offsets, g.adj, g.w)
        key = oracle.level_key(seed, 0)
        lab = oracle.lp_round(G, np.arange(G.n, dtype=np.int32), key)
        if seed % 2:
            lab = oracle.lp_round(G, lab, key)
        h, _ = oracle.contract(G, lab)
        out.append(h)
    for seed in range(6):
        g = H.random_graph(random.Random(seed).randint(5, 40), 0.3, 900 + seed, wmax=6)
        G = oracle.as_csr64(g.offsets, g.adj, g.w)
        h, _ = oracle.contract(G, np.arange(G.n, dtype=np.int32))
        out.append(h)
    return out


@pytest.mark.parametrize("which", ["a", "b", "noi"])
def test_label_steps_parity(which):
    for h in coarse_graphs():
        dmin = int(oracle.degrees(h).min())
        d = upload(h)
        try:
            for lam in [dmin, max(1, dmin // 2), 2 * dmin, 1 << 50]:
                if which == "a":
                    got, ch = vc.viecut_step_pr_a(d, lam)
                    ref, cnt = oracle.pr_pass_a(h, lam)
                elif which == "b":
                    got, ch = vc.viecut_step_pr_b(d, lam)
                    ref, cnt = oracle.pr_pass_b(h, lam)
                else:
                    if lam > dmin:
                        continue  # a round needs lambda-hat <= min degree
                    got, ch = vc.viecut_step_noi_round(d, lam)
                    ref, cnt = oracle.noi_round(h, lam)
                assert np.array_equal(got, ref), (which, h.n, lam)
                assert ch == (1 if cnt > 0 else 0)
        finally:
            vc.viecut_graph_free(d)


def test_exact_round_memory_paths():
    """One exact-step round through each kernel: shared-memory state (up to 16,384
    vertices) and global-memory state (above), for bounds at, below and far below the
    minimum degree, against the oracle's scan with its union-find (labels element by
    element); then the whole exact step on the larger graph."""
    graphs = [gg.with_pair_weights(gg.core_lcc(gg.er(3000, 14, 21), 2), 21, 1, 9),
              gg.with_pair_weights(gg.core_lcc(gg.er(20000, 12, 22), 2), 22, 1, 9),
              gg.core_lcc(gg.rhg(1 << 15, 24, 23), 8)]
    for g in graphs:
        h = oracle.as_csr64(g.offsets, g.adj, g.w)
        dmin = int(oracle.degrees(h).min())
        d = upload(h)
        try:
            for lam in sorted({dmin, max(1, dmin // 2), 1}):
                got, ch = vc.viecut_step_noi_round(d, lam)
                ref, cnt = oracle.noi_round(h, lam)
                assert np.array_equal(got, ref), (g.n, lam)
                assert ch == (1 if cnt > 0 else 0)
        finally:
            vc.viecut_graph_free(d)
    g = graphs[1]
    assert g.n > 16384
    cut, bits = vc.exact_min_cut(g.offsets, g.adj, g.w)
    ref = oracle.viecut(g.offsets, g.adj, g.w, seed=1, lp_iters=0, n0=g.n)
    assert cut == ref.cut and np.array_equal(bits[: len(ref.side_bits)], ref.side_bits)


# ------------------------------------------------------------- whole method
@pytest.mark.parametrize("seed", range(24))
def test_viecut_random_small(seed):
    rnd = random.Random(seed)
    g = H.random_graph(rnd.randint(2, 60), rnd.uniform(0.05, 0.6), 300 + seed, wmax=rnd.choice([1, 4, 30]))
    for lp, n0 in [(0, 1), (1, 2), (2, 1), (3, 8), (2, BIG_N0)]:
        assert_same(g, seed=seed, lp=lp, n0=n0)


@pytest.mark.parametrize("make", [
    H.pr2_counterexample, lambda: H.two_cliques(7, 2), lambda: H.cycle(50), lambda: H.grid(9, 11),
    lambda: H.hypercube(6), lambda: H.complete(20), multi_edge_graph,
    lambda: gg.from_edges(2, [(0, 1, 5)]),
    lambda: gg.from_edges(6, [(0, 1, 2), (1, 2, 2), (3, 4, 1), (4, 5, 1)]),   # disconnected
    lambda: gg.from_edges(5, [(0, 1, 1), (1, 2, 1), (0, 2, 1)]),              # isolated vertices
])
def test_viecut_special_graphs(make):
    g = make()
    for lp, n0 in [(0, 1), (2, 1), (2, 4), (2, BIG_N0)]:
        assert_same(g, lp=lp, n0=n0)


@pytest.mark.parametrize("n0", [10000, 64, 1])
@pytest.mark.parametrize("seed", [1, 2])
def test_viecut_rhg_small_workload(seed, n0):
    """RHG n = 2^14, average degree 32, exponent 5, largest component."""
    g = gg.workload_rhg_small(seed)
    assert_same(g, seed=seed, lp=2, n0=n0)


def test_viecut_weighted_and_hubs():
    assert_same(gg.with_pair_weights(gg.core_lcc(gg.rhg(1 << 13, 24, 9), 0), 9, 1, 10), seed=4, n0=32)
    assert_same(hub_graph(), seed=2, n0=16)
    assert_same(gg.er(3000, 12, 3, 1, 100), seed=3, n0=16)
    assert_same(gg.planted(4, 1 << 10, 16, 8, 5, 1, 100), seed=5, n0=64)
    assert_same(gg.planted(8, 1 << 12, 48, 64, 1, 1, 100), seed=1, n0=10000)


def test_viecut_sparse_exact_step():
    """Kernels above the dense limit take the sparse exact-step rounds first."""
    for seed in range(3):
        g = H.random_graph(700 + 100 * seed, 0.02, 50 + seed, wmax=5)
        assert_same(g, seed=seed, lp=2, n0=BIG_N0)
    g = gg.core_lcc(gg.rhg(3000, 10, 4), 0)
    assert_same(g, seed=1, lp=1, n0=2000)


def test_exact_mode():
    """exact_min_cut (the exact step alone, n0 >= n) equals the oracle's exact run and,
    where label propagation misses it, stays below the method's value."""
    for g in [gg.core_lcc(gg.rhg(1 << 13, 32, 1), 16), H.random_graph(300, 0.05, 8, wmax=9),
              gg.with_pair_weights(gg.core_lcc(gg.er(2000, 10, 4), 3), 4, 1, 20), H.pr2_counterexample()]:
        cut, bits = vc.exact_min_cut(g.offsets, g.adj, g.w)
        ref = oracle.viecut(g.offsets, g.adj, g.w, seed=1, lp_iters=0, n0=g.n)
        assert cut == ref.cut and np.array_equal(bits, ref.side_bits), g.name
        for s in (1, 2, 3):
            assert cut <= oracle.viecut(g.offsets, g.adj, g.w, seed=s, lp_iters=1, n0=64).cut


def test_clustered_er_family():
    """The paper's clustered Erdos-Renyi family (weights inside clusters times n): the
    method equals the oracle, and the exact mode gives the oracle's exact value."""
    for k, d in ((2, 10), (4, 5), (8, 20)):
        g = gg.clustered_er(2000, d, k, 30 + k)
        assert_same(g, seed=k, lp=2, n0=64)
        cut, _ = vc.exact_min_cut(g.offsets, g.adj, g.w)
        assert cut == oracle.viecut(g.offsets, g.adj, g.w, seed=1, lp_iters=0, n0=g.n).cut


def test_correcting_step_parity():
    """The method with the correcting step (Sec. 4.1) equals the oracle's reading of it
    (trace, cut, side); on all but the isolated-vertex graph it changes the run."""
    graphs = [gg.workload_rhg_small(2), gg.with_pair_weights(gg.core_lcc(gg.rhg(1 << 12, 20, 7), 0), 7, 1, 50),
              gg.er(3000, 12, 3, 1, 100), hub_graph(), gg.core_lcc(gg.rhg(1 << 13, 32, 1), 16)]
    changed = 0
    for g in graphs:
        for seed, lp in ((1, 1), (2, 2)):
            ref = oracle.viecut(g.offsets, g.adj, g.w, seed=seed, lp_iters=lp, n0=64, correct=True)
            with vc.MinCut(g.offsets, g.adj, g.w, n0=64, correct=True) as mc:
                cut, bits = mc.run(seed, lp)
                tr = mc.trace()
            assert cut == ref.cut and np.array_equal(bits, ref.side_bits), (g.name, seed, lp)
            assert tr == ref.trace, (g.name, seed, lp)
            changed += ref.trace != oracle.viecut(g.offsets, g.adj, g.w, seed=seed, lp_iters=lp, n0=64).trace
    assert changed >= 8


def test_viecut_repeatable_and_seeded():
    g = gg.workload_rhg_small(3)
    with vc.MinCut(g.offsets, g.adj, g.w, n0=64) as mc:
        a = mc.run(5, 2)
        b = mc.run(5, 2)
        c = mc.run(6, 2)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    ref = oracle.viecut(g.offsets, g.adj, g.w, seed=6, lp_iters=2, n0=64)
    assert c[0] == ref.cut and np.array_equal(c[1], ref.side_bits)


def test_device_resident_inputs_and_errors():
    import torch
    g = gg.workload_rhg_small(1)
    dev = torch.device("cuda:0")
    off = torch.from_numpy(g.offsets).to(dev)
    adj = torch.from_numpy(g.adj).to(dev)
    w = torch.from_numpy(g.w).to(dev)
    ref = oracle.viecut(g.offsets, g.adj, g.w, seed=1, lp_iters=2, n0=10000)
    with vc.MinCut(off, adj, w, on_device=True) as mc:
        cut, bits = mc.run(1, 2)
        d_cut = torch.zeros(1, dtype=torch.int64, device=dev)
        d_bits = torch.zeros((g.n + 63) // 64, dtype=torch.int64, device=dev)
        vc.viecut_run_device(mc.h, 1, 2, d_cut, d_bits)
        torch.cuda.synchronize()
    assert cut == ref.cut and np.array_equal(bits, ref.side_bits)
    assert int(d_cut.item()) == ref.cut
    assert np.array_equal(d_bits.cpu().numpy().view(np.uint64), ref.side_bits)
    # device-side validation catches a self-loop
    bad = adj.clone()
    bad[int(g.offsets[5])] = 5
    with pytest.raises(vc.ViecutError) as e:
        vc.MinCut(off, bad, w, on_device=True)
    assert e.value.code == vc.VIECUT_EINVAL and "self-loop" in str(e.value)
    with pytest.raises(vc.ViecutError):
        with vc.MinCut(g.offsets, g.adj, g.w) as mc:
            mc.run(1, -1)


def test_launches_counted():
    g = gg.workload_rhg_small(1)
    with vc.MinCut(g.offsets, g.adj, g.w, timing=True) as mc:
        before = vc.viecut_launch_count()
        mc.run(1, 2)
        st = mc.stats()
    assert st["kernel_launches"] == vc.viecut_launch_count() - before > 10
    assert st["lp_launches"] == 2 and st["ms_lp_kernel"] > 0


@pytest.mark.parametrize("lp_group,emit_group", [(8, 8), (16, 16), (32, 32), (8, 32), (32, 16)])
def test_group_sizes_give_identical_results(lp_group, emit_group):
    """Lanes per vertex are a launch shape only: every choice gives the oracle's trace,
    cut and side, on unit weights and on stored weights (different kernels)."""
    graphs = [gg.workload_rhg_small(2), gg.with_pair_weights(gg.core_lcc(gg.rhg(1 << 13, 24, 9), 0), 9, 1, 10),
              hub_graph()]
    for g in graphs:
        ref = oracle.viecut(g.offsets, g.adj, g.w, seed=3, lp_iters=2, n0=64)
        with vc.MinCut(g.offsets, g.adj, g.w, n0=64, lp_group=lp_group, emit_group=emit_group) as mc:
            cut, bits = mc.run(3, 2)
            st = mc.stats()
            trace = mc.trace()
        assert (st["first_group"], st["emit_group"]) == (lp_group, emit_group)
        assert trace == ref.trace and cut == ref.cut and np.array_equal(bits, ref.side_bits), g.name


def test_autotuned_groups_on_a_large_graph():
    """Above 2^16 vertices the handle times each choice once and keeps the fastest."""
    g = gg.core_lcc(gg.rhg(1 << 17, 32, 6), 0)
    ref = oracle.viecut(g.offsets, g.adj, g.w, seed=2, lp_iters=2, n0=10000)
    with vc.MinCut(g.offsets, g.adj, g.w) as mc:
        first = mc.run(2, 2)
        st = mc.stats()
        again = mc.run(2, 2)
    assert st["first_group"] in (8, 16, 32) and st["emit_group"] in (8, 16, 32)
    for cut, bits in (first, again):
        assert cut == ref.cut and np.array_equal(bits, ref.side_bits)


def hidden_pair(g, value, stride):
    """A copy of g whose one symmetric entry pair (both positions >= 256 and off the
    multiples of stride) gets weight value."""
    w = g.w.copy()
    for v in range(g.n // 2, g.n):
        for e in range(g.offsets[v], g.offsets[v + 1]):
            u = int(g.adj[e])
            r = [x for x in range(g.offsets[u], g.offsets[u + 1]) if g.adj[x] == v][0]
            if min(e, r) >= 256 and e % stride and r % stride:
                w[e] = w[r] = value
                return gg.Graph(g.offsets, g.adj, w, g.name + f"+pair{value}")
    raise AssertionError("no pair found")


def test_solve_equals_load_and_run():
    """viecut_solve on unit weights runs with unit weights while the weights are checked;
    on weighted graphs it does not speculate; a unit-looking graph with one hidden
    heavier pair is run again with weights; a hidden zero weight is refused and leaves
    the handle without a graph.  Results always equal the oracle's."""
    g_unit = gg.workload_rhg_small(5)
    stride = max(1, g_unit.nnz // 4096)
    cases = [g_unit, gg.with_pair_weights(gg.core_lcc(gg.rhg(1 << 13, 24, 9), 0), 9, 1, 10),
             hidden_pair(g_unit, 3, stride), H.pr2_counterexample()]
    with vc.MinCut(cases[0].offsets, cases[0].adj, cases[0].w, n0=64) as mc:
        for i, g in enumerate(cases + cases[::-1]):
            cut, bits = mc.solve(g.offsets, g.adj, g.w, 11 + i, 2)
            ref = oracle.viecut(g.offsets, g.adj, g.w, seed=11 + i, lp_iters=2, n0=64)
            assert cut == ref.cut and np.array_equal(bits, ref.side_bits), (i, g.name)
            assert mc.trace() == ref.trace, (i, g.name)
        bad = hidden_pair(g_unit, 0, stride)
        with pytest.raises(vc.ViecutError) as e:
            mc.solve(bad.offsets, bad.adj, bad.w, 1, 2)
        assert e.value.code == vc.VIECUT_EINVAL and "weight" in str(e.value)
        with pytest.raises(vc.ViecutError) as e:
            mc.run(1, 2)
        assert e.value.code == vc.VIECUT_EINVAL


def test_lp_converge_parity():
    """The convergence stop (at most lp_iters rounds, ending after a round that changed at
    most 1/10000 of the labels) equals the oracle's; on 4000 K5 plus an edge whose ends
    swap labels every round, the stop fires after the rounds the oracle's level takes."""
    from tests.test_oracle import cliques_and_edge, two_triangles
    graphs = [(gg.workload_rhg_small(3), 64), (cliques_and_edge(), 64), (two_triangles(), 1),
              (gg.planted(4, 1 << 12, 16, 8, 5, 1, 100), 64)]
    for g, n0 in graphs:
        for seed in (1, 2):
            ref = oracle.viecut(g.offsets, g.adj, g.w, seed=seed, lp_iters=25, n0=n0, converge=True)
            with vc.MinCut(g.offsets, g.adj, g.w, n0=n0, lp_converge=True) as mc:
                cut, bits = mc.run(seed, 25)
                tr = mc.trace()
            assert tr == ref.trace and cut == ref.cut and np.array_equal(bits, ref.side_bits), (g.name, seed)
    g = cliques_and_edge()
    G = oracle.as_csr64(g.offsets, g.adj, g.w)
    _, rounds = oracle.lp_level(G, oracle.level_key(1, 0), 25, True)
    with vc.MinCut(g.offsets, g.adj, g.w, n0=g.n - 1, lp_converge=True, timing=True) as mc:
        mc.run(1, 25)
        assert mc.stats()["lp_launches"] == rounds < 25
    with pytest.raises(vc.ViecutError) as e:
        vc.viecut_batch_create([(g.offsets, g.adj, g.w)], vc.viecut_opts_init(lp_converge=1))
    assert e.value.code == vc.VIECUT_EINVAL


@pytest.mark.parametrize("lp_async", [1, 2])
def test_async_lp_parity(lp_async):
    """Asynchronous rounds in shuffled 128-vertex blocks and eight waves (with the first
    round's restriction for lp_async = 2) equal the oracle's reading of them: trace, cut
    and side, with and without the convergence stop."""
    graphs = [(gg.workload_rhg_small(2), 64), (gg.with_pair_weights(gg.core_lcc(gg.rhg(1 << 12, 20, 7), 0), 7, 1, 50), 32),
              (hub_graph(), 16), (gg.planted(4, 1 << 10, 16, 8, 5, 1, 100), 64), (H.two_cliques(7, 2), 1)]
    for g, n0 in graphs:
        for seed, lp, conv in ((1, 2, False), (2, 1, False), (3, 25, True)):
            ref = oracle.viecut(g.offsets, g.adj, g.w, seed=seed, lp_iters=lp, n0=n0, converge=conv,
                                lp_async=lp_async)
            with vc.MinCut(g.offsets, g.adj, g.w, n0=n0, lp_converge=conv, lp_async=lp_async) as mc:
                cut, bits = mc.run(seed, lp)
                tr = mc.trace()
            assert tr == ref.trace and cut == ref.cut and np.array_equal(bits, ref.side_bits), (g.name, seed, lp)
