"""Host-side checks of the GPU library that need no GPU: it builds, loads, exports
every entry point its header declares, and fails loudly without a device."""
import os
import re

import numpy as np
import pytest

import paper_1708_06127_gb300 as vc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "viecut.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(viecut_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    vc.build()
    return vc.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["viecut_create", "viecut_run", "viecut_destroy", "viecut_create_device", "viecut_run_device",
              "viecut_step_lp", "viecut_step_contract", "viecut_step_pr_a", "viecut_step_pr_b",
              "viecut_step_noi_round", "viecut_last_error"]:
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing
    bound = {name for name, _, _ in vc.SIGNATURES}
    assert set(declared_functions()) == bound, "Python binding and header disagree"


def test_binding_structs_match_the_library(lib):
    """Every structure the binding restates has the library's size (a field added on
    one side only would shift every later field)."""
    import ctypes
    sizes = np.zeros(9, np.int64)
    n = vc.lib().viecut_struct_sizes(sizes.ctypes.data, 9)
    assert n == 8
    mine = [vc.viecut_opts, vc.viecut_stats, vc.viecut_step, vc.viecut_graph_desc, vc.viecut_batch_stats,
            vc.viecut_server_opts, vc.viecut_server_stats, vc.viecut_request_info]
    assert sizes[:8].tolist() == [ctypes.sizeof(t) for t in mine]
    assert vc.lib().viecut_struct_sizes(None, 1) == vc.VIECUT_EINVAL


def test_opts_defaults(lib):
    o = vc.viecut_opts_init()
    assert (o.n0, o.pr_runs_max, o.device, o.validate, o.timing) == (10000, 8, 0, 1, 0)
    assert (o.lp_group, o.emit_group) == (0, 0)  # 0: picked by timing


def test_group_options_are_checked_before_any_device_call(lib):
    off = np.array([0, 1, 2], np.int64)
    adj = np.array([1, 0], np.int32)
    for bad in ({"lp_group": 4}, {"emit_group": 64}, {"lp_group": -8}):
        with pytest.raises(vc.ViecutError) as e:
            vc.viecut_create(off, adj, 2, 2, np.array([1, 1], np.int32), vc.viecut_opts_init(**bad))
        assert e.value.code == vc.VIECUT_EINVAL and "lp_group" in str(e.value)


def test_correct_option_is_checked_before_any_device_call(lib):
    """correct must be 0 or 1, and batches and the server refuse it (the correcting
    step runs on single-graph handles only)."""
    off = np.array([0, 1, 2], np.int64)
    adj = np.array([1, 0], np.int32)
    w = np.array([1, 1], np.int32)
    assert vc.viecut_opts_init().correct == 0
    with pytest.raises(vc.ViecutError) as e:
        vc.viecut_create(off, adj, 2, 2, w, vc.viecut_opts_init(correct=2))
    assert e.value.code == vc.VIECUT_EINVAL and "correct" in str(e.value)
    with pytest.raises(vc.ViecutError) as e:
        vc.viecut_batch_create([(off, adj, w)], vc.viecut_opts_init(correct=1))
    assert e.value.code == vc.VIECUT_EINVAL and "correct" in str(e.value)
    with pytest.raises(vc.ViecutError) as e:
        vc.viecut_server_start(vc.viecut_server_opts_init(correct=1))
    assert e.value.code == vc.VIECUT_EINVAL and "correct" in str(e.value)


def test_host_validation_rejects_bad_graphs(lib):
    """Full validation of host arrays (validate = 2) happens before any device call,
    so it is testable here: every malformed input must give EINVAL with a message."""
    full = vc.viecut_opts_init(validate=2)
    off = np.array([0, 1, 2], np.int64)
    adj = np.array([1, 0], np.int32)
    cases = [
        (off, np.array([1, 1], np.int32), np.array([1, 1], np.int32), "self-loop"),
        (off, np.array([1, 5], np.int32), np.array([1, 1], np.int32), "out of range"),
        (off, adj, np.array([1, 0], np.int32), "weight"),
        (np.array([0, 2, 1], np.int64), adj, np.array([1, 1], np.int32), "offsets"),
    ]
    for o, a, w, why in cases:
        with pytest.raises(vc.ViecutError) as e:
            vc.viecut_create(o, a, 2, 2, w, full)
        assert e.value.code == vc.VIECUT_EINVAL and why in str(e.value), (why, str(e.value))
    # asymmetric weights are caught by the full check (validate = 2)
    with pytest.raises(vc.ViecutError) as e:
        vc.viecut_create(off, adj, 2, 2, np.array([1, 2], np.int32), vc.viecut_opts_init(validate=2))
    assert e.value.code == vc.VIECUT_EINVAL and "symmetric" in str(e.value)
    with pytest.raises(vc.ViecutError) as e:
        vc.viecut_create(np.array([0], np.int64), adj, 1, 0, adj)
    assert e.value.code == vc.VIECUT_EINVAL


def test_no_device_fails_loudly(lib):
    """Without a GPU a valid graph must produce a CUDA error, never a CPU result."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    off = np.array([0, 1, 2], np.int64)
    adj = np.array([1, 0], np.int32)
    with pytest.raises(vc.ViecutError) as e:
        vc.viecut_create(off, adj, 2, 2, np.array([3, 3], np.int32))
    assert e.value.code == vc.VIECUT_ECUDA


def test_fault_injection_arguments(lib):
    """The allocation-failure hook refuses negative arguments; count 0 switches it off
    (no device is touched)."""
    assert vc.lib().viecut_debug_fail_device_allocs(-1, 1) == vc.VIECUT_EINVAL
    assert vc.lib().viecut_debug_fail_device_allocs(0, -1) == vc.VIECUT_EINVAL
    assert vc.lib().viecut_debug_fail_device_allocs(0, 0) == vc.VIECUT_OK
