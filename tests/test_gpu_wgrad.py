"""GPU parity of the standalone 3x3 weight-gradient op (conet_conv3x3_wgrad) against the
oracle's conv3x3 backward: sizes that span many RE splits, a ragged last split, the
smallest grids, and every channel count the networks use."""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, normwise, torch
from workloads import random_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def oracle_wgrad(x, dz):
    from oracle import net as onet
    tp = onet.Tape()
    cout, cin = dz.shape[-1], x.shape[-1]
    xi = tp.leaf(x.astype(np.float64))
    wi = tp.leaf(np.zeros((cout, 3, 3, cin)))
    bi = tp.leaf(np.zeros(cout))
    out = onet.conv3x3(tp, xi, wi, bi)
    g = tp.backward(out, dz.astype(np.float64))
    return g[wi], g[bi]


@pytest.mark.parametrize("B,T,F,cin,cout", [(3, 14, 72, 8, 32), (2, 14, 37, 32, 32), (1, 14, 624, 64, 64),
                                            (1, 5, 3, 96, 96), (2, 14, 13, 112, 112), (1, 1, 1, 4, 4),
                                            (16, 14, 72, 32, 32)])
def test_wgrad_matches_oracle(B, T, F, cin, cout):
    from paper_2510_12739_gb300 import api
    x = random_grid(1, (B, T, F, cin))
    dz = random_grid(2, (B, T, F, cout))
    dW, db = api.conv3x3_wgrad(dev(x), dev(dz))
    w_ref, b_ref = oracle_wgrad(x, dz)
    assert normwise(dW.cpu().numpy(), w_ref) < 1e-5
    assert normwise(db.cpu().numpy(), b_ref) < 1e-5


def test_wgrad_is_deterministic_and_rejects_bad_channels():
    from paper_2510_12739_gb300 import api
    from paper_2510_12739_gb300._lib import ConetError
    x = dev(random_grid(3, (4, 14, 100, 32)))
    dz = dev(random_grid(4, (4, 14, 100, 32)))
    a, _ = api.conv3x3_wgrad(x, dz)
    b, _ = api.conv3x3_wgrad(x, dz)
    assert torch.equal(a, b)
    with pytest.raises(ConetError) as e:
        api.conv3x3_wgrad(dev(random_grid(5, (1, 2, 2, 6))), dev(random_grid(6, (1, 2, 2, 4))))
    assert e.value.code == -2
