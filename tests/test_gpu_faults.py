"""Failure handling without a GPU fault: device allocations made to fail on the host
(viecut_debug_fail_device_allocs), request cancellation and host-side bounded waits.

Every failure here is made on the host.  The checks: the failing call returns
VIECUT_ENOMEM / VIECUT_ECANCELLED / VIECUT_ETIMEOUT, and the handle, batch or server
that saw it keeps working, with results equal to the CPU oracle's.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1708_06127_gb300 as vc
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    vc.build()


@pytest.fixture(autouse=True)
def _no_injection_left():
    yield
    vc.viecut_debug_fail_device_allocs(0, 0)


def same_as_oracle(g, res, seed=1, n0=10000):
    cut, bits = res[0], res[1]
    ref = oracle.viecut(g.offsets, g.adj, g.w, seed=seed, lp_iters=2, n0=n0)
    assert cut == ref.cut and np.array_equal(bits[: len(ref.side_bits)], ref.side_bits), g.name


def test_handle_survives_failed_allocations():
    g = gg.workload_rhg_small(1)
    big = gg.core_lcc(gg.rhg(1 << 15, 32, 3), 0)
    # creation
    vc.viecut_debug_fail_device_allocs(0, 1)
    with pytest.raises(vc.ViecutError) as e:
        vc.MinCut(g.offsets, g.adj, g.w)
    assert e.value.code == vc.VIECUT_ENOMEM and "injected" in str(e.value)
    with vc.MinCut(g.offsets, g.adj, g.w) as mc:
        # the first run grows the work space: its first allocation fails, the next run works
        vc.viecut_debug_fail_device_allocs(0, 1)
        with pytest.raises(vc.ViecutError) as e:
            mc.run(1, 2)
        assert e.value.code == vc.VIECUT_ENOMEM
        same_as_oracle(g, mc.run(1, 2))
        # a load of a larger graph must grow the handle's buffers: it fails, and the handle
        # holds no graph until the next load
        vc.viecut_debug_fail_device_allocs(0, 1)
        with pytest.raises(vc.ViecutError) as e:
            mc.load(big.offsets, big.adj, big.w)
        assert e.value.code == vc.VIECUT_ENOMEM
        with pytest.raises(vc.ViecutError) as e:
            mc.run(1, 2)
        assert e.value.code == vc.VIECUT_EINVAL
        mc.load(big.offsets, big.adj, big.w)
        same_as_oracle(big, mc.run(1, 2))


def test_batch_survives_failed_allocations():
    graphs = [gg.with_pair_weights(gg.core_lcc(gg.rhg(600 + 50 * i, 16, 70 + i), 0), i, 1, 9) for i in range(12)]
    graphs += [H.pr2_counterexample(), H.two_cliques(8, 2)]
    tri = [(g.offsets, g.adj, g.w) for g in graphs]
    vc.viecut_debug_fail_device_allocs(3, 1)
    with pytest.raises(vc.ViecutError) as e:
        vc.Batch(tri)
    assert e.value.code == vc.VIECUT_ENOMEM
    with vc.Batch(tri) as b:
        vc.viecut_debug_fail_device_allocs(0, 1)
        try:
            b.run(4, 2)
        except vc.ViecutError as e2:
            assert e2.code == vc.VIECUT_ENOMEM
        vc.viecut_debug_fail_device_allocs(0, 0)
        cuts, bits = b.run(4, 2)
    for i, g in enumerate(graphs):
        same_as_oracle(g, (cuts[i], bits[i]), seed=4)


def test_server_answers_failed_admissions_and_goes_on():
    small = gg.core_lcc(gg.rhg(2000, 24, 5), 0)
    large = gg.core_lcc(gg.rhg(1 << 14, 32, 6), 0)
    with vc.Server(max_slots=16, solo_min_n=8000, solo_exact=False, solo_lanes=1) as srv:
        # the union lane: the join's first allocation (its staging buffers) fails
        vc.viecut_debug_fail_device_allocs(0, 1)
        t = srv.submit(small.offsets, small.adj, small.w, 1)
        with pytest.raises(vc.ViecutError) as e:
            srv.wait(t)
        assert e.value.code == vc.VIECUT_ENOMEM
        same_as_oracle(small, srv.wait(srv.submit(small.offsets, small.adj, small.w, 1)))
        # the solo lane: the handle's creation fails
        vc.viecut_debug_fail_device_allocs(0, 1)
        t = srv.submit(large.offsets, large.adj, large.w, 1)
        with pytest.raises(vc.ViecutError) as e:
            srv.wait(t)
        assert e.value.code == vc.VIECUT_ENOMEM
        same_as_oracle(large, srv.wait(srv.submit(large.offsets, large.adj, large.w, 1)))
        st = srv.stats()
    assert st["failed"] == 2 and st["completed"] == 4


def test_server_cancel_and_bounded_wait():
    graphs = [gg.core_lcc(gg.rhg(int(2 ** (10 + 0.3 * i)), 32, 40 + i), 0) for i in range(16)]
    with vc.Server(max_slots=4, solo_min_n=0) as srv:
        tickets = [srv.submit(g.offsets, g.adj, g.w, 1) for g in graphs]
        # four slots: the last request is still queued when it is cancelled
        srv.cancel(tickets[-1])
        srv.cancel(tickets[-1])  # twice is a no-op
        # a bounded wait that runs out leaves the ticket valid
        with pytest.raises(vc.ViecutError) as e:
            vc.viecut_server_wait(srv.s, tickets[-2], graphs[-2].n, 0.0)
        assert e.value.code == vc.VIECUT_ETIMEOUT
        for t, g in zip(tickets[:-1], graphs[:-1]):
            same_as_oracle(g, srv.wait(t, timeout=120.0))
        with pytest.raises(vc.ViecutError) as e:
            srv.wait(tickets[-1])
        assert e.value.code == vc.VIECUT_ECANCELLED
        # a finished request that is cancelled before its poll: the result is dropped
        t = srv.submit(graphs[0].offsets, graphs[0].adj, graphs[0].w, 1)
        import time
        deadline = time.time() + 60
        while srv.stats()["completed"] < 17 and time.time() < deadline:
            time.sleep(0.001)
        srv.cancel(t)
        with pytest.raises(vc.ViecutError) as e:
            srv.poll(t)
        assert e.value.code == vc.VIECUT_ECANCELLED
        with pytest.raises(vc.ViecutError) as e:
            srv.cancel(123456789)
        assert e.value.code == vc.VIECUT_EINVAL
        st = srv.stats()
    assert st["cancelled"] == 2
