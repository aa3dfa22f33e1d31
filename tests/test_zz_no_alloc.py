"""The allocation-free entry point fmm_sort_points_noalloc, for callers that cannot let a
library allocate device memory (one allocator owns all of their device memory, or their whole
budget is reserved at start-up).  It must reproduce the first step of fmm_build_tree exactly:
the same Morton keys and the same stable permutation, call after call, although every call
reuses one scratch array inside the library.

This file is collected last so that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2604_19243_gb300 as pkg
from synth import cube_points, sphere_points

pytestmark = pytest.mark.gpu
MAX_POINTS = 1 << 20


def _noalloc(x, depth, origin, side):
    n = x.shape[0]
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    keys = torch.empty(n, dtype=torch.int32, device="cuda")      # uint32 bits
    org = (ctypes.c_double * 3)(*origin)
    st = pkg.lib().fmm_sort_points_noalloc(x.data_ptr(), n, depth, org, ctypes.c_double(side),
                                           perm.data_ptr(), keys.data_ptr(),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, perm.cpu().numpy().astype(np.int64), keys.cpu().numpy().view(np.uint32).astype(np.uint64)


def _reference(x, depth, origin, side):
    f = pkg.FMM(p=3, depth=depth, domain=(origin, side))
    f.build_tree(x)
    t = f.export_tree()
    f.close()
    keys = np.repeat(t["leaf_keys"], np.diff(t["leaf_offsets"]))
    return t["perm"], keys


def test_noalloc_sort_matches_build_tree_twice():
    # calls in a row with different inputs: the shared scratch must not leak between them, a
    # small call after the largest one included, and depth 0, where no radix pass runs and the
    # keys never leave the caller's buffer
    cases = [(sphere_points(300_007, seed=21), 7, (-1.0, -1.0, -1.0), 2.0),
             (cube_points(MAX_POINTS, seed=22), 6, (0.0, 0.0, 0.0), 1.0),
             (sphere_points(5_003, seed=23), 5, (-1.0, -1.0, -1.0), 2.0),
             (cube_points(1_000, seed=24), 0, (0.0, 0.0, 0.0), 1.0)]
    for xs, depth, origin, side in cases:
        x = torch.from_numpy(xs).cuda()
        st, perm, keys = _noalloc(x, depth, origin, side)
        assert st == 0
        rperm, rkeys = _reference(x, depth, origin, side)
        np.testing.assert_array_equal(perm, rperm)
        np.testing.assert_array_equal(keys, rkeys)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    x = torch.zeros(MAX_POINTS + 1, 3, device="cuda")
    st, _, _ = _noalloc(x, 5, (0.0, 0.0, 0.0), 1.0)
    assert st == 1   # FMM_EINVAL
    st, _, _ = _noalloc(x[:10], 11, (0.0, 0.0, 0.0), 1.0)
    assert st == 1


def test_noalloc_rejects_non_finite_coordinates():
    # as fmm_build_tree does; the call after it must sort normally again
    for bad in (float("nan"), float("inf")):
        xs = cube_points(4_096, seed=25)
        xs[1234, 1] = bad
        st, _, _ = _noalloc(torch.from_numpy(xs).cuda(), 5, (0.0, 0.0, 0.0), 1.0)
        assert st == 1   # FMM_EINVAL
    x = torch.from_numpy(cube_points(4_096, seed=26)).cuda()
    st, perm, keys = _noalloc(x, 5, (0.0, 0.0, 0.0), 1.0)
    assert st == 0
    rperm, rkeys = _reference(x, 5, (0.0, 0.0, 0.0), 1.0)
    np.testing.assert_array_equal(perm, rperm)
    np.testing.assert_array_equal(keys, rkeys)
