"""CPU checks of the C-ABI boundary: libconet.so loads, exports every entry point that
include/conet.h declares, agrees with the oracle on the parameter layout size, and
rejects bad arguments on the host before touching the GPU."""
import ctypes as C
import os
import re

import pytest

from workloads import WORKLOADS, tiny_net, replace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "conet.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(conet_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_12739_gb300 import _lib
    try:
        return _lib.lib()
    except ImportError as e:
        pytest.fail(str(e))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("conet_create", "conet_load_weights", "conet_forward", "conet_backward", "conet_train_step",
                 "conet_destroy", "conet_sim_generate", "conet_ls_lmmse", "conet_loss_ber"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_python_binding_covers_every_declared_symbol():
    from paper_2510_12739_gb300 import _lib
    assert set(declared_symbols()) == set(_lib.SIGNATURES)


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_param_count_matches_oracle_layout(lib, name):
    from oracle import net as onet
    from paper_2510_12739_gb300 import api
    assert api.param_count(WORKLOADS[name].net) == onet.param_count(WORKLOADS[name].net)


@pytest.mark.parametrize("kw", [dict(), dict(norm=1), dict(residual=1, norm=1, n_branches=3),
                                dict(residual=1, norm=1, depthwise=1),
                                dict(n_branches=1, residual=1, norm=1, resnet_baseline=1),
                                dict(fuse_mask=0b01, norm=1), dict(fuse_op=2), dict(fuse_op=2, norm=1, fuse_mask=0b01),
                                dict(fuse_op=2, n_branches=3, depth=3, norm=1)])
def test_param_count_tiny(lib, kw):
    from oracle import net as onet
    from paper_2510_12739_gb300 import api
    cfg = tiny_net(**kw)
    assert api.param_count(cfg) == onet.param_count(cfg)


def test_host_side_argument_errors(lib):
    from paper_2510_12739_gb300 import api
    from paper_2510_12739_gb300._lib import ConetError
    base = WORKLOADS["plain_14x72_b16_fp32"].net
    for bad in (dict(qam_bits=5), dict(n_branches=0), dict(n_branches=5), dict(n_rx=0),
                dict(pilot_syms=(11, 2)), dict(pilot_syms=(2, 14)), dict(width=0), dict(support_inputs=2),
                dict(support_inputs=1, n_branches=1, residual=1, resnet_baseline=1), dict(fuse_op=3),
                dict(fuse_op=2, residual=1, norm=1), dict(fuse_op=2, n_branches=3, width=48),
                dict(support_mask=1), dict(support_inputs=1, support_mask=1 << 7)):
        with pytest.raises(ConetError) as e:
            api.param_count(replace(base, **bad))
        assert e.value.code == -1
    with pytest.raises(ConetError) as e:
        api.param_count(replace(base, n_branches=2, resnet_baseline=1, residual=1))
    assert e.value.code == -1
    n = C.c_size_t()
    assert lib.conet_param_count(None, C.byref(n)) == -1
    assert b"NULL" in lib.conet_last_error()
    # NULL handles / pointers are rejected before any CUDA call
    assert lib.conet_forward(None, None, None, None, 1, None, None) == -1
    assert lib.conet_backward(None, None, 1, None) == -1
    assert lib.conet_loss_ber(None, None, None, 1, 14, 72, 4, 0.0, None, None, None, None, None) == -1
    assert lib.conet_ber_count(None, None, None, 1, 14, 72, 4, None, None, None) == -1
    cfg = api.make_config(base)
    assert lib.conet_sim_generate(C.byref(cfg), None, 0, 0, 1, 0.0, None, None, None, None, None, None) == -1


def test_checkpoint_hash_tracks_the_network_shape(lib):
    """The checkpoint header's hash changes with every field that gives the parameters their
    meaning and not with the workspace size or the train flag."""
    from paper_2510_12739_gb300 import api
    base = WORKLOADS["plain_14x72_b16_fp32"].net
    h0 = api.checkpoint_hash(base)
    assert h0 == api.checkpoint_hash(base)
    for kw in (dict(n_rx=2), dict(n_sc=73), dict(qam_bits=6), dict(n_branches=3), dict(depth=5), dict(width=16),
               dict(norm=1), dict(fuse_mask=0b11), dict(pilot_syms=(2, 12)), dict(pilot_comb=3),
               dict(pilot_seed=1), dict(residual=1), dict(fuse_op=1), dict(feedback=1), dict(support_inputs=1),
               dict(fuse_op=2)):
        assert api.checkpoint_hash(replace(base, **kw)) != h0, kw
    # a full-input network's hash is the one it had before the selective-inputs field existed
    assert h0 == api.checkpoint_hash(replace(base, support_inputs=0))
    sel = replace(base, support_inputs=1)
    assert api.checkpoint_hash(replace(sel, support_mask=0b11)) != api.checkpoint_hash(sel)
    cfg = api.make_config(base, max_batch=7, train=True)
    h = C.c_uint64()
    assert lib.conet_checkpoint_hash(C.byref(cfg), C.byref(h)) == 0 and h.value == h0
    # NULL handles and buffers are rejected on the host
    assert lib.conet_checkpoint_hash(C.byref(cfg), None) == -1
    n = C.c_size_t()
    assert lib.conet_checkpoint_bytes(None, C.byref(n)) == -1
    assert lib.conet_save_checkpoint(None, 0, None, 0) == -1
    assert lib.conet_load_checkpoint(None, None, 0, None) == -1
    assert lib.conet_selftest_timeout(None, 1e-3, None) == -1


def test_whole_network_threshold_matches_header():
    """The binding's automatic whole-network threshold is the header's constant, and the
    mode argument is range-checked on the host."""
    from paper_2510_12739_gb300 import api
    src = open(os.path.join(ROOT, "include", "conet.h")).read()
    m = re.search(r"#define\s+CONET_WHOLE_NET_MIN_SLOTS\s+(\d+)", src)
    assert m and int(m.group(1)) == api.WHOLE_NET_MIN_SLOTS
    lib = api.lib()
    assert lib.conet_whole_network(None, 1, None) == -1
