"""Batched solving: every graph's result in the batch (cut value, side bitmap and
per-step trace) equals the oracle's result for that graph alone, for mixes of
uneven sizes, weights, options and degenerate graphs."""
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


def check_batch(graphs, seed=1, lp=2, n0=10000, pr=8):
    tri = [(g.offsets, g.adj, g.w) for g in graphs]
    with vc.Batch(tri, n0=n0, pr_runs_max=pr) as b:
        cuts, bits = b.run(seed, lp)
        traces = [b.trace(i) for i in range(len(graphs))]
        st = b.stats()
    for i, g in enumerate(graphs):
        ref = oracle.viecut(g.offsets, g.adj, g.w, seed=seed, lp_iters=lp, n0=n0, pr_runs_max=pr)
        assert traces[i] == ref.trace, (i, g.name)
        assert cuts[i] == ref.cut, (i, g.name)
        assert np.array_equal(bits[i], ref.side_bits), (i, g.name)
    return st


def mixed_small(count, seed):
    rnd = random.Random(seed)
    out = []
    for i in range(count):
        r = rnd.random()
        if r < 0.3:
            out.append(H.random_graph(rnd.randint(2, 50), rnd.uniform(0.05, 0.6), 1000 * seed + i, wmax=rnd.choice([1, 5, 40])))
        elif r < 0.6:
            out.append(gg.core_lcc(gg.rhg(rnd.randint(64, 3000), rnd.uniform(6, 24), 77 * seed + i), 0))
        elif r < 0.8:
            out.append(gg.core_lcc(gg.er(rnd.randint(64, 2000), rnd.uniform(4, 16), 31 * seed + i, 1, 10), 0))
        else:
            out.append(rnd.choice([H.pr2_counterexample(), H.cycle(30), H.grid(6, 7), H.two_cliques(8, 2),
                                   gg.from_edges(2, [(0, 1, 3)]),
                                   gg.from_edges(6, [(0, 1, 2), (1, 2, 2), (3, 4, 1), (4, 5, 1)]),
                                   gg.from_edges(5, [(0, 1, 1), (1, 2, 1), (0, 2, 1)])]))
    return out


@pytest.mark.parametrize("n0,lp", [(10000, 2), (16, 2), (1, 1), (BIG_N0, 2), (64, 3)])
def test_batch_mixed_parity(n0, lp):
    check_batch(mixed_small(48, n0 % 97 + lp), seed=3, lp=lp, n0=n0)


def test_batch_single_graph_and_large():
    check_batch([gg.workload_rhg_small(1)], n0=64)
    check_batch([gg.workload_rhg_small(2), gg.planted(8, 1 << 12, 48, 64, 1, 1, 100),
                 gg.with_pair_weights(gg.core_lcc(gg.rhg(1 << 13, 24, 9), 0), 9, 1, 10)], n0=32)
    # kernels above the dense limit take sparse rounds first
    check_batch([H.random_graph(700, 0.02, 50, wmax=5), H.random_graph(40, 0.3, 51)], n0=BIG_N0)


def test_batch_workload_sample():
    """A slice of the batched workload: n log-uniform in [2^6, 2^14], RHG or ER,
    weights [1, 10]."""
    specs = gg.batch_specs(160, seed=11)
    graphs = [gg.batch_graph(s) for s in specs]
    st = check_batch(graphs, seed=2)
    assert st["graphs"] == 160 and st["super_steps"] > 0


def test_batch_equals_single_runs_on_gpu():
    graphs = mixed_small(12, 5)
    tri = [(g.offsets, g.adj, g.w) for g in graphs]
    with vc.Batch(tri, n0=8) as b:
        cuts, bits = b.run(9, 2)
    for i, g in enumerate(graphs):
        with vc.MinCut(g.offsets, g.adj, g.w, n0=8) as mc:
            c, bb = mc.run(9, 2)
        assert c == cuts[i] and np.array_equal(bb, bits[i])


def test_batch_rejects_bad_graph():
    good = gg.from_edges(3, [(0, 1, 1), (1, 2, 1)])
    bad = gg.from_edges(3, [(0, 1, 1), (1, 2, 1)])
    bad.adj[0] = 7
    with pytest.raises(vc.ViecutError) as e:
        vc.Batch([(good.offsets, good.adj, good.w), (bad.offsets, bad.adj, bad.w)])
    assert e.value.code == vc.VIECUT_EINVAL
