"""Failure detection without a GPU fault: the tensor-core kernels' bounded barrier waits made to
run out (FMM_ETIMEOUT through fmm_sync, the context usable afterwards) and device allocations
refused by the library's allocation cap (FMM_ENOMEM, the call repeatable once the cap is lifted).
Nothing here faults, traps or waits without a limit: the timeout is the kernels' own bounded wait
with its limit set to zero, and the allocation failure is decided on the host."""
import numpy as np
import pytest
import torch

import paper_2604_19243_gb300 as pkg
from synth import cube_points, charges
from gpu_helpers import make_fmm

pytestmark = pytest.mark.gpu
ENOMEM, ESTATE, ETIMEOUT = 2, 4, 5


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3"])   # plane-layout and register-layout kernels
def test_barrier_timeout_is_reported_and_the_context_recovers(precision):
    x, q = cube_points(60_000, seed=31), charges(60_000, "u11", seed=32)
    f = make_fmm(x, 6, 4, precision, ((0, 0, 0), 1.0))
    qd = torch.from_numpy(q).cuda()
    phi0, grad0 = f.evaluate(qd)
    f.sync()
    f.set_wait_limit(0.0)          # every wait that does not complete at once gives up
    f.evaluate(qd)
    with pytest.raises(pkg.FmmError) as e:
        f.sync()
    assert e.value.status == ETIMEOUT
    f.set_wait_limit(1.0)
    f.sync()                       # the flag was cleared by the failed sync
    phi1, grad1 = f.evaluate(qd)
    f.sync()
    assert torch.equal(phi0, phi1) and torch.equal(grad0, grad1)
    # limits of a few microseconds give up part-way, with copies and MMAs in flight, or not at
    # all: either way the call reports it and the next one is correct
    for limit in (2e-6, 2e-5):
        f.set_wait_limit(limit)
        f.evaluate(qd)
        try:
            f.sync()
        except pkg.FmmError as err:
            assert err.status == ETIMEOUT
        f.set_wait_limit(1.0)
        phi1, grad1 = f.evaluate(qd)
        f.sync()
        assert torch.equal(phi0, phi1) and torch.equal(grad0, grad1)
    f.close()


def test_allocation_cap_gives_enomem_and_the_calls_succeed_after():
    x, q = cube_points(20_000, seed=33), charges(20_000, "u01", seed=34)
    ref = make_fmm(x, 4, 3, "fp32", ((0, 0, 0), 1.0))
    qd = torch.from_numpy(q).cuda()
    phi_ref, grad_ref = ref.evaluate(qd)
    ref.sync()
    ref.close()
    xd = torch.from_numpy(x).cuda()
    f = pkg.FMM(p=4, depth=3, precision="fp32", domain=((0, 0, 0), 1.0), pinv_rtol=1e-7, svd_rtol=1e-6)
    try:
        pkg.set_alloc_limit(1 << 16)           # every allocation above 64 KB fails
        with pytest.raises(pkg.FmmError) as e:
            f.precompute()
        assert e.value.status == ENOMEM
        with pytest.raises(pkg.FmmError) as e:
            f.build_tree(xd)
        assert e.value.status == ENOMEM
        with pytest.raises(pkg.FmmError) as e:   # no tree and no operators were left behind
            f.evaluate(qd)
        assert e.value.status == ESTATE
    finally:
        pkg.set_alloc_limit(None)
    f.build_tree(xd).precompute()
    phi, grad = f.evaluate(qd)
    f.sync()
    assert torch.equal(phi, phi_ref) and torch.equal(grad, grad_ref)
    f.close()
