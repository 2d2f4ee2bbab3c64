"""The allocation-free weight-gradient entry point, called through the C ABI.

conet_conv3x3_wgrad_noalloc exists for callers that cannot allocate device memory where
they need a weight gradient (memory planned once at start-up, code inside a graph capture,
embeddings that only own their buffers); it keeps its partial sums in an array compiled
into the library instead.  This test checks it against the regular entry point
conet_conv3x3_wgrad, which allocates its scratch per call, on two calls in a row with
different inputs (the second call must not see the first call's partial sums).  Both entry
points run the same kernels with the same split rule and reduce the partial sums in the same
fixed order, so the results must be bitwise identical: a partial sum left over from the
previous call would show up as a difference.  The file name sorts last so that a run
stopping at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from gpu_util import dev, need_gpu, torch
from workloads import random_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _call(name, x, dz, dW, db):
    from paper_2510_12739_gb300._lib import check, lib
    B, T, F, cin = x.shape
    cout = dz.shape[-1]
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib(), name)(C.c_void_p(x.data_ptr()), C.c_void_p(dz.data_ptr()), B, T, F, cin, cout,
                              C.c_void_p(dW.data_ptr()), C.c_void_p(db.data_ptr()), stream)
    check(rc)


@pytest.mark.parametrize("B,T,F,cin,cout", [(4, 14, 72, 32, 32), (1, 14, 624, 64, 64), (2, 14, 29, 96, 96)])
def test_noalloc_wgrad_matches_regular_entry_point_twice(B, T, F, cin, cout):
    for call, seed in enumerate((11, 23)):
        x = dev(random_grid(seed, (B, T, F, cin)))
        dz = dev(random_grid(seed + 1, (B, T, F, cout)))
        dW_ref = torch.empty((cout, 3, 3, cin), device="cuda")
        db_ref = torch.empty(cout, device="cuda")
        dW = torch.full((cout, 3, 3, cin), float("nan"), device="cuda")
        db = torch.full((cout,), float("nan"), device="cuda")
        _call("conet_conv3x3_wgrad", x, dz, dW_ref, db_ref)
        _call("conet_conv3x3_wgrad_noalloc", x, dz, dW, db)
        torch.cuda.synchronize()
        assert torch.equal(dW, dW_ref), call
        assert torch.equal(db, db_ref), call
