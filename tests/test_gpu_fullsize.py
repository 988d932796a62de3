"""Full-size workloads, in the launch configuration the benchmark times (inputs
resident on the device, default options), compared with the oracle in full: cut
value, side bitmap and the per-step trace (for the planted graph with the oracle's
stored result, which takes it half an hour).  The planted graph is also checked
against the cut value known from its construction."""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1708_06127_gb300 as vc
from tests.test_oracle import planted_lambda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    vc.build()


def bench_config_run(g, seed=1, lp=2):
    import torch
    dev = torch.device("cuda:0")
    off = torch.from_numpy(g.offsets).to(dev)
    adj = torch.from_numpy(g.adj).to(dev)
    w = torch.from_numpy(g.w).to(dev)
    with vc.MinCut(off, adj, w, on_device=True, stream=torch.cuda.current_stream().cuda_stream) as mc:
        cut, bits = mc.run(seed, lp)
        trace = mc.trace()
    return cut, bits, trace


def check(g, seed=1):
    cut, bits, trace = bench_config_run(g, seed)
    ref = oracle.viecut(g.offsets, g.adj, g.w, seed=seed, lp_iters=2, n0=10000, pr_runs_max=8)
    assert trace == ref.trace
    assert cut == ref.cut
    assert np.array_equal(bits, ref.side_bits)
    side = ref.side(g.n)
    assert side.any() and not side.all() and not side[0]
    return ref


def test_rhg_2_22_core16():
    """RHG n = 2^22, average degree 64, exponent 5, 16-core, largest component."""
    g = gg.workload_rhg_large(1)
    check(g, seed=1)


def test_planted_8x2_16_exact():
    """The planted family at 8 blocks of 2^16 vertices (the oracle needs about a
    minute): exact parity."""
    g = gg.planted(8, 1 << 16, 48, 64, 1, 1, 100)
    ref = check(g, seed=1)
    assert ref.cut >= planted_lambda(g, 8, 1 << 16)


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "planted_8x2p20.json")


def test_planted_8x2_20_golden():
    """8 ER blocks of 2^20 vertices (average degree 48), 64 bridges, weights [1, 100],
    against the CPU oracle's result stored by tests/golden/make_planted.py (the oracle
    needs about half an hour at this size): the same graph (SHA-256 of the generated
    CSR), then every step of the contraction trace, the cut value, and the side bitmap
    (SHA-256 and popcount)."""
    ref = json.load(open(GOLDEN))
    p = ref["params"]
    g = gg.planted(p["blocks"], p["block_n"], p["avg_deg"], p["bridges"], p["graph_seed"], p["wlo"], p["whi"])
    h = hashlib.sha256()
    for a in (g.offsets, g.adj, g.w):
        h.update(np.ascontiguousarray(a).tobytes())
    assert h.hexdigest() == ref["graph_sha256"], "the generator drew another graph on this host"
    cut, bits, trace = bench_config_run(g, seed=p["seed"], lp=p["lp_iters"])
    want = [tuple(s) for s in ref["trace"]]
    for k, (a, b) in enumerate(zip(trace, want)):
        assert a == b, (k, a, b)
    assert len(trace) == len(want)
    assert cut == ref["cut"]
    assert hashlib.sha256(np.ascontiguousarray(bits, dtype=np.uint64).tobytes()).hexdigest() == ref["side_sha256"]
    side = np.unpackbits(bits.view(np.uint8), bitorder="little")[: g.n]
    assert int(side.sum()) == ref["side_popcount"]


def test_planted_8x2_20_properties():
    """The same workload checked by properties that hold at any size: the value is at
    least the construction's cut value and equals the weight of the returned side,
    which is a proper subset without vertex 0."""
    g = gg.workload_planted(1)
    cut, bits, trace = bench_config_run(g, seed=1)
    side = np.unpackbits(bits.view(np.uint8), bitorder="little")[: g.n].astype(bool)
    assert side.any() and not side.all() and not side[0]
    src = np.repeat(np.arange(g.n, dtype=np.int32), np.diff(g.offsets))
    cross = side[src] != side[g.adj]
    assert int(g.w[cross].astype(np.int64).sum()) // 2 == cut
    lam = planted_lambda(g, 8, 1 << 20)
    assert cut >= lam
    lh = [s[4] for s in trace]
    assert all(a >= b for a, b in zip(lh, lh[1:])) and lh[-1] == cut
    print(f"planted 8x2^20: value {cut}, construction {lam}, steps {len(trace)}")
