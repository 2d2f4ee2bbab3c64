"""Failure detection and exact resume on the GPU, without faulting the GPU.

* A bounded device wait that runs out: conet_selftest_timeout launches a kernel whose
  mbarrier wait (the tensor-core pipelines' own bounded wait, with a 1 ms limit) is never
  satisfied; the next conet_sync must return CONET_ERR_TIMEOUT and the context must keep
  working.
* Non-finite LLRs: weights with an infinite head bias make the forward pass write infinite
  LLRs, which conet_sync reports as CONET_ERR_NONFINITE (every path: FP32 fusion stage and
  the tensor-core epilogue); finite weights afterwards sync cleanly.
* Versioned checkpoints: training k steps, saving, and continuing in a fresh handle gives
  bitwise the parameters of an uninterrupted run (the Adam moments and step travel with the
  weights); a checkpoint of another network or a corrupted header is refused."""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from workloads import WORKLOADS, replace

pytestmark = pytest.mark.gpu
TIMEOUT, NONFINITE, WEIGHTS = -7, -6, -5


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _slots(net, sim, B):
    from paper_2510_12739_gb300 import api
    mask, _ = api.pilots(net)
    s = api.sim_generate(net, sim, 5, 0, B)
    return s, mask


def test_timed_out_wait_is_reported_and_context_survives():
    from paper_2510_12739_gb300 import api
    from paper_2510_12739_gb300._lib import ConetError
    w = WORKLOADS["plain_14x72_b16_fp32"]
    rx = api.Receiver(w.net, "bf16", max_batch=4)
    rx.init_he(0)
    s, mask = _slots(w.net, w.sim, 4)
    ref = rx.forward(s["Y"], mask).clone()
    rx.sync()
    rx.selftest_timeout(1e-3)
    with pytest.raises(ConetError) as e:
        rx.sync()
    assert e.value.code == TIMEOUT and "site 100" in str(e.value)
    rx.sync()                                   # the status word was cleared
    again = rx.forward(s["Y"], mask)
    rx.sync()
    assert torch.equal(again, ref)              # the GPU keeps computing the same results


@pytest.mark.parametrize("name,precision", [("plain_14x72_b16_fp32", "fp32"), ("plain_14x72_b16_fp32", "bf16"),
                                            ("resid_14x624_b256_fp32", "fp32"), ("resid_14x624_b256_fp32", "fp16")])
def test_nonfinite_llr_is_flagged(name, precision):
    from oracle import net as onet
    from paper_2510_12739_gb300 import api
    from paper_2510_12739_gb300._lib import ConetError
    w = WORKLOADS[name]
    net = replace(w.net, n_sc=72) if w.net.n_sc > 72 else w.net
    rx = api.Receiver(net, precision, max_batch=2)
    p = onet.init_params(net, 3).astype(np.float32)
    s, mask = _slots(net, w.sim, 2)
    rx.load_weights(p)
    rx.forward(s["Y"], mask)
    rx.sync()
    bad = p.copy()
    bad[-1] = np.inf                            # the head's last bias
    rx.load_weights(bad)
    llr = rx.forward(s["Y"], mask)
    with pytest.raises(ConetError) as e:
        rx.sync()
    assert e.value.code == NONFINITE
    assert not torch.isfinite(llr[..., -1]).any()
    rx.load_weights(p)
    rx.forward(s["Y"], mask)
    rx.sync()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_checkpoint_resume_is_bitwise(precision):
    from paper_2510_12739_gb300 import api
    w = WORKLOADS["train_14x72_b128_bf16"]
    B, k = 32, 6
    run = api.Receiver(w.net, precision, max_batch=B, train=True)
    run.init_he(2)
    for i in range(k):
        run.train_step(w.sim, 9, i, B, 2e-3, want_loss=False)
    blob = run.save_checkpoint(k)
    for i in range(k, 2 * k):
        run.train_step(w.sim, 9, i, B, 2e-3, want_loss=False)
    straight = run.save_weights()
    resumed = api.Receiver(w.net, precision, max_batch=B, train=True)
    resumed.init_he(77)                         # different state, all of it overwritten
    step = resumed.load_checkpoint(blob)
    assert step == k
    for i in range(step, 2 * k):
        resumed.train_step(w.sim, 9, i, B, 2e-3, want_loss=False)
    assert np.array_equal(resumed.save_weights(), straight)
    # the weights alone (no Adam moments) do not resume exactly
    plain = api.Receiver(w.net, precision, max_batch=B, train=True)
    plain.load_weights(np.frombuffer(blob, dtype=np.float32, offset=64, count=plain.n_params))
    for i in range(k, 2 * k):
        plain.train_step(w.sim, 9, i, B, 2e-3, want_loss=False)
    assert not np.array_equal(plain.save_weights(), straight)


def test_checkpoint_of_another_network_or_corrupt_is_refused():
    from paper_2510_12739_gb300 import api
    from paper_2510_12739_gb300._lib import ConetError
    w = WORKLOADS["train_14x72_b128_bf16"]
    a = api.Receiver(w.net, "fp32", max_batch=2, train=True)
    a.init_he(1)
    blob = a.save_checkpoint(3)
    before = a.save_weights()
    other = api.Receiver(replace(w.net, pilot_seed=5), "fp32", max_batch=2, train=True)
    with pytest.raises(ConetError) as e:
        other.load_checkpoint(blob)
    assert e.value.code == WEIGHTS
    bad = bytearray(blob)
    bad[0] ^= 0xFF                              # magic
    with pytest.raises(ConetError) as e:
        a.load_checkpoint(bytes(bad))
    assert e.value.code == WEIGHTS
    bad = bytearray(blob)
    bad[8] = 2                                  # format version
    with pytest.raises(ConetError) as e:
        a.load_checkpoint(bytes(bad))
    assert e.value.code == WEIGHTS
    with pytest.raises(ConetError) as e:
        a.load_checkpoint(blob[:-4])            # truncated
    assert e.value.code == WEIGHTS
    assert np.array_equal(a.save_weights(), before)
