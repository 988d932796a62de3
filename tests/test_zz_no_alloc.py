"""The allocation-free exact-step round, viecut_noi_round_noalloc.

Some callers cannot allocate device memory: their GPU memory belongs to another
allocator (a host framework that reserved it for its own pool), or their loop must not
pay cudaMalloc's implicit device synchronisation.  For them the library offers a
Nagamochi-Ono-Ibaraki round whose work space is a static device array.  These tests
call it through the C ABI on device buffers the test owns and compare its output with
the allocating entry point viecut_step_noi_round, twice in a row and across graphs
of different sizes (each call runs on the scratch the previous call left behind), and
on the first pass also with the CPU oracle's round.  Integer results: the comparison
is exact.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1708_06127_gb300 as vc
from tests import helpers as H

pytestmark = pytest.mark.gpu
MAX_N = 1 << 16


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    vc.build()


def merged(g):
    G = oracle.as_csr64(g.offsets, g.adj, g.w)
    h, _ = oracle.contract(G, np.arange(G.n, dtype=np.int32))
    return h


def cases():
    out = []
    g = gg.with_pair_weights(gg.core_lcc(gg.rhg(1 << 12, 16, 3), 0), 3, 1, 9)
    G = oracle.as_csr64(g.offsets, g.adj, g.w)
    key = oracle.level_key(1, 0)
    lab = oracle.lp_round(G, np.arange(G.n, dtype=np.int32), key)
    out.append(oracle.contract(G, lab)[0])           # a coarse graph
    out.append(merged(H.random_graph(300, 0.05, 8, wmax=7)))
    out.append(merged(H.pr2_counterexample()))
    out.append(merged(gg.er(MAX_N, 3, 5, 1, 4)))      # the largest size the scratch holds
    return out


def reference(h, lam):
    d = vc.viecut_graph_upload(h.offsets, h.adj, h.w)
    try:
        return vc.viecut_step_noi_round(d, lam)
    finally:
        vc.viecut_graph_free(d)


def test_noalloc_round_matches_allocating_round():
    import torch
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    work = []
    for h in cases():
        dmin = int(oracle.degrees(h).min())
        for lam in sorted({dmin, max(1, dmin // 2)}):
            work.append((h, lam))
    for call in range(2):  # two passes: every call finds the previous call's leftovers
        for h, lam in work:
            ref_labels, ref_changed = reference(h, lam)
            off = torch.from_numpy(h.offsets).to(dev)
            adj = torch.from_numpy(h.adj).to(dev)
            w = torch.from_numpy(h.w).to(dev)
            labels = torch.full((h.n,), -7, dtype=torch.int32, device=dev)
            changed = torch.full((1,), -7, dtype=torch.int32, device=dev)
            vc.viecut_noi_round_noalloc(off, adj, w, h.n, lam, labels, changed, stream.cuda_stream)
            stream.synchronize()
            assert np.array_equal(labels.cpu().numpy(), ref_labels), (call, h.n, lam)
            assert int(changed.item()) == ref_changed, (call, h.n, lam)
            if call == 0:  # and both equal the oracle's round
                orc_labels, orc_unions = oracle.noi_round(h, lam)
                assert np.array_equal(ref_labels, orc_labels) and ref_changed == (orc_unions > 0), (h.n, lam)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    dev = torch.device("cuda:0")
    n = MAX_N + 1
    off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    labels = torch.zeros(n, dtype=torch.int32, device=dev)
    changed = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(vc.ViecutError) as e:
        vc.viecut_noi_round_noalloc(off, None, None, n, 1, labels, changed)
    assert e.value.code == vc.VIECUT_EINVAL and "65536" in str(e.value)


def test_noalloc_rejects_null_arrays():
    """The host cannot read offsets[n], so null adjacency or weights are refused before
    any launch (a graph with edges would otherwise read through a null pointer)."""
    import torch
    dev = torch.device("cuda:0")
    n = 8
    off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    adj = torch.zeros(4, dtype=torch.int32, device=dev)
    w = torch.ones(4, dtype=torch.int64, device=dev)
    labels = torch.zeros(n, dtype=torch.int32, device=dev)
    changed = torch.zeros(1, dtype=torch.int32, device=dev)
    before = vc.viecut_launch_count()
    for a, b in ((None, w), (adj, None), (None, None)):
        with pytest.raises(vc.ViecutError) as e:
            vc.viecut_noi_round_noalloc(off, a, b, n, 1, labels, changed)
        assert e.value.code == vc.VIECUT_EINVAL and "null" in str(e.value)
    assert vc.viecut_launch_count() == before
