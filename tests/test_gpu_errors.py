"""Error paths of the C ABI on a GPU: calls out of order, bad arguments, non-finite input."""
import numpy as np
import pytest
import torch

import paper_2604_19243_gb300 as pkg
from synth import cube_points, charges

pytestmark = pytest.mark.gpu


def _status(exc):
    return exc.value.status


def test_call_order():
    f = pkg.FMM(p=3, depth=2)
    q = torch.zeros(10, device="cuda")
    with pytest.raises(pkg.FmmError) as e:
        f.n = 10
        f.evaluate(q)
    assert _status(e) == 4
    f.build_tree(torch.rand(10, 3, device="cuda"))
    with pytest.raises(pkg.FmmError) as e:
        f.evaluate(q)
    assert _status(e) == 4
    f.precompute()
    with pytest.raises(pkg.FmmError) as e:
        f.export_check(2)
    assert _status(e) == 4
    phi, _ = f.evaluate(q)
    assert torch.all(phi == 0)


def test_bad_inputs():
    f = pkg.FMM(p=3, depth=2)
    x = torch.rand(100, 3, device="cuda")
    x[17, 1] = float("nan")
    with pytest.raises(pkg.FmmError) as e:
        f.build_tree(x)
    assert _status(e) == 1
    x[17, 1] = float("inf")
    with pytest.raises(pkg.FmmError) as e:
        f.build_tree(x)
    assert _status(e) == 1
    with pytest.raises(pkg.FmmError) as e:
        f.build_tree(torch.zeros(0, 3, device="cuda"))
    assert _status(e) == 1
    # a valid tree after the failures
    f.build_tree(torch.rand(100, 3, device="cuda")).precompute()
    with pytest.raises(pkg.FmmError) as e:
        f.evaluate(torch.rand(100, device="cuda"), parts=0)
    assert _status(e) == 1


def test_gradient_not_enabled():
    f = pkg.FMM(p=3, depth=2, with_gradient=False)
    f.build_tree(torch.rand(100, 3, device="cuda")).precompute()
    with pytest.raises(pkg.FmmError) as e:
        f.evaluate(torch.rand(100, device="cuda"), gradient=True)
    assert _status(e) == 1
    phi, g = f.evaluate(torch.rand(100, device="cuda"), gradient=False)
    assert g is None and torch.isfinite(phi).all()


def test_rebuild_with_other_size_and_all_points_equal():
    f = pkg.FMM(p=3, depth=3)
    f.build_tree(torch.rand(1000, 3, device="cuda")).precompute()
    f.evaluate(torch.rand(1000, device="cuda"))
    x = torch.ones(50, 3, device="cuda")          # zero extent: unit cube, one leaf
    f.build_tree(x)
    phi, grad = f.evaluate(torch.rand(50, device="cuda"))
    assert torch.all(phi == 0) and torch.all(grad == 0)   # every pair coincident -> skipped
    assert f.info()["n_boxes"][3] == 1
