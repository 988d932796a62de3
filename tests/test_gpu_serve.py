"""Serving with continuous batching: requests submitted while others are resident
join the device-resident set at the next super-step; every result (cut value and side
bitmap) equals the oracle's and the single-graph run's for that graph alone."""
import random
import threading
import time

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


def request_mix(count, seed):
    rnd = random.Random(seed)
    out = []
    for i in range(count):
        r = rnd.random()
        if r < 0.5:
            g = gg.core_lcc(gg.rhg(int(2 ** rnd.uniform(10, 15)), 32, 1000 * seed + i), 0)
        elif r < 0.8:
            g = gg.with_pair_weights(gg.core_lcc(gg.er(rnd.randint(100, 3000), rnd.uniform(4, 12), 7 * i + seed), 0),
                                     i, 1, 10)
        else:
            g = rnd.choice([H.pr2_counterexample(), H.two_cliques(9, 2), H.random_graph(40, 0.2, 5 * i + seed),
                            gg.from_edges(5, [(0, 1, 1), (1, 2, 1), (0, 2, 1)])])
        out.append((g, rnd.randint(1, 1 << 30)))
    return out


def check_result(g, seed, res, n0=10000):
    cut, bits, lat = res
    ref = oracle.viecut(g.offsets, g.adj, g.w, seed=seed, lp_iters=2, n0=n0)
    assert cut == ref.cut, g.name
    assert np.array_equal(bits[: len(ref.side_bits)], ref.side_bits), g.name
    assert lat >= 0


def test_serve_staggered_arrivals_equal_alone():
    reqs = request_mix(40, 3)
    with vc.Server(max_slots=64, solo_exact=False) as srv:
        tickets = []
        for i, (g, seed) in enumerate(reqs):
            tickets.append(srv.submit(g.offsets, g.adj, g.w, seed))
            if i % 5 == 4:
                time.sleep(0.002)  # later requests arrive while earlier ones are resident
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    for (g, seed), res in zip(reqs, results):
        check_result(g, seed, res)
    assert st["completed"] == len(reqs) and st["admitted"] == len(reqs)
    assert st["joins"] >= 2, st          # admitted in several waves
    assert st["max_resident"] >= 2, st   # work overlapped on the device
    # alone: the plain single-graph path gives the same answers
    for (g, seed), (cut, bits, _) in list(zip(reqs, results))[:8]:
        with vc.MinCut(g.offsets, g.adj, g.w) as mc:
            c, b = mc.run(seed, 2)
        assert c == cut and np.array_equal(b, bits[: len(b)])


def test_serve_concurrent_submitters_and_small_budget():
    reqs = request_mix(24, 9)
    budget = 3 * max(96 * (g.nnz + g.n) + 112 * g.n + (1 << 16) for g, _ in reqs)
    out = {}
    with vc.Server(hbm_budget_bytes=budget, max_slots=16, n0=64) as srv:
        def submitter(part):
            for g, seed in part:
                t = srv.submit(g.offsets, g.adj, g.w, seed)
                out[t] = (g, seed)
                time.sleep(0.001)
        th = [threading.Thread(target=submitter, args=(reqs[k::3],)) for k in range(3)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        results = {t: srv.wait(t) for t in list(out)}
        st = srv.stats()
    for t, res in results.items():
        g, seed = out[t]
        check_result(g, seed, res, n0=64)
    assert st["completed"] == len(reqs) and st["budget_used"] == 0


def test_serve_rejects_bad_requests():
    """Shape and budget faults fail the submit; per-entry faults are found by the device
    check on either lane and answered through poll, while the other requests are served."""
    with vc.Server(hbm_budget_bytes=1 << 20) as srv:
        big = gg.core_lcc(gg.rhg(1 << 14, 32, 1), 0)
        with pytest.raises(vc.ViecutError) as e:
            srv.submit(big.offsets, big.adj, big.w, 1)
        assert e.value.code == vc.VIECUT_EINVAL and "budget" in str(e.value)
        bad = gg.from_edges(3, [(0, 1, 1), (1, 2, 1)])
        bad.offsets[3] = 5  # offsets[n] != m
        with pytest.raises(vc.ViecutError) as e:
            srv.submit(bad.offsets, bad.adj, bad.w, 1)
        assert e.value.code == vc.VIECUT_EINVAL
        with pytest.raises(vc.ViecutError):
            vc.viecut_server_poll(srv.s, 12345, 3)
    for solo_min_n in (0, 3):  # union lane, then solo lane for graphs of >= 3 vertices
        with vc.Server(solo_min_n=solo_min_n) as srv:
            good = H.pr2_counterexample()
            loop = gg.from_edges(3, [(0, 1, 1), (1, 2, 1)])
            loop.adj[0] = 0  # self-loop at vertex 0
            far = gg.from_edges(4, [(0, 1, 1), (2, 3, 2)])
            far.adj[1] = 9   # neighbour id out of range
            zero = gg.from_edges(3, [(0, 1, 1), (1, 2, 1)])
            zero.w[:] = 0    # weight < 1
            tickets = [srv.submit(x.offsets, x.adj, x.w, 3) for x in (good, loop, far, zero, good)]
            for t, why in zip(tickets[1:4], ("self-loop", "out of range", "weight")):
                with pytest.raises(vc.ViecutError) as e:
                    srv.wait(t)
                assert e.value.code == vc.VIECUT_EINVAL and why in str(e.value), (solo_min_n, str(e.value))
            for t in (tickets[0], tickets[4]):
                check_result(good, 3, srv.wait(t))
            st = srv.stats()
            assert st["rejected"] == 3 and st["completed"] == 5 and st["budget_used"] == 0, st


def test_serve_solo_lane_beside_the_union():
    """Requests at or above solo_min_n vertices run alone on their own handle and stream
    while the rest share the union; both lanes give the oracle's results."""
    reqs = request_mix(30, 21)
    big = [gg.core_lcc(gg.rhg(1 << 13, 32, 77 + i), 0) for i in range(4)]
    reqs[3:3] = [(g, 50 + i) for i, g in enumerate(big)]
    with vc.Server(max_slots=32, solo_min_n=4000, solo_exact=False) as srv:
        tickets = [srv.submit(g.offsets, g.adj, g.w, seed) for g, seed in reqs]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    for (g, seed), res in zip(reqs, results):
        check_result(g, seed, res)
    n_solo = sum(1 for g, _ in reqs if g.n >= 4000)
    assert st["solo_completed"] == n_solo >= 4, st
    assert st["completed"] == len(reqs) and st["budget_used"] == 0


def test_serve_exact_step_graphs_on_parallel_solo_lanes():
    """With solo_exact (the default), graphs whose whole run is the exact step (513..n0
    vertices) go to the solo lanes, several of which run side by side; the union keeps
    the small and the large graphs.  Every result equals the oracle's."""
    reqs = request_mix(36, 13)
    with vc.Server(max_slots=32, solo_lanes=3) as srv:
        tickets = [srv.submit(g.offsets, g.adj, g.w, seed) for g, seed in reqs]
        infos = {}
        for t in tickets:
            while True:
                r = srv.poll_info(t)
                if r is not None:
                    infos[t] = r
                    break
                time.sleep(0.0005)
        st = srv.stats()
    for (g, seed), t in zip(reqs, tickets):
        cut, bits, info = infos[t]
        check_result(g, seed, (cut, bits, info["latency_ms"]))
        exact_only = 512 < g.n <= 10000
        assert info["lane"] == (1 if (exact_only or g.n >= 1 << 16) else 0), (g.n, info)
        assert info["queue_ms"] >= 0 and info["run_ms"] >= 0 and info["n"] == g.n
    n_solo = sum(1 for g, _ in reqs if 512 < g.n <= 10000 or g.n >= 1 << 16)
    assert st["solo_completed"] == n_solo > 0 and st["completed"] == len(reqs)


def test_load_reuses_a_handle_across_graphs():
    """viecut_load rebinds a host-made handle to other graphs (larger, then smaller);
    every run equals the oracle's; a device-made handle refuses it."""
    import torch
    gs = [H.random_graph(50, 0.2, 3, wmax=4), gg.workload_rhg_small(4), H.pr2_counterexample(),
          gg.with_pair_weights(gg.core_lcc(gg.er(3000, 8, 2), 0), 2, 1, 9)]
    with vc.MinCut(gs[0].offsets, gs[0].adj, gs[0].w, n0=64) as mc:
        for i, g in enumerate(gs + gs[::-1]):
            mc.load(g.offsets, g.adj, g.w)
            cut, bits = mc.run(7 + i, 2)
            ref = oracle.viecut(g.offsets, g.adj, g.w, seed=7 + i, lp_iters=2, n0=64)
            assert cut == ref.cut and np.array_equal(bits, ref.side_bits), (i, g.name)
        bad = gg.from_edges(3, [(0, 1, 1), (1, 2, 1)])
        bad.adj[0] = 0
        with pytest.raises(vc.ViecutError) as e:
            mc.load(bad.offsets, bad.adj, bad.w)
        assert e.value.code == vc.VIECUT_EINVAL
        with pytest.raises(vc.ViecutError) as e:  # nothing runs on a graph that failed its check
            mc.run(1, 2)
        assert e.value.code == vc.VIECUT_EINVAL
        g = gs[2]
        mc.load(g.offsets, g.adj, g.w)  # a good graph makes the handle usable again
        ref = oracle.viecut(g.offsets, g.adj, g.w, seed=1, lp_iters=2, n0=64)
        assert mc.run(1, 2)[0] == ref.cut
    g = gs[1]
    dev = torch.device("cuda:0")
    d = [torch.from_numpy(x).to(dev) for x in (g.offsets, g.adj, g.w)]
    with vc.MinCut(*d, on_device=True) as mc:
        with pytest.raises(vc.ViecutError) as e:
            mc.load(g.offsets, g.adj, g.w)
        assert e.value.code == vc.VIECUT_EINVAL and "viecut_create" in str(e.value)
