"""fmm_debug_check: the tree's index tables validated on the device, and the bounds-checked build
libfmm_debug.so (FMM_DEBUG: the kernels that compute indices check them instead of trusting them).

Every case runs in a child process that loads the chosen library (FMM_LIBRARY), evaluates small
uniform (FP32, FP16X3), partitioned, adaptive and FFT cases, and reports the checks that failed
and the outputs; both builds must report no failure, the debug build must have its in-kernel
checks, and the two builds' outputs must be identical bit for bit (the checks only guard
accesses)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import paper_2604_19243_gb300 as pkg
from synth import cube_points, sphere_points, mixed_points, charges
out = {"lib": pkg.LIB_PATH, "cases": {}}
def case(name, f, q, how="uniform"):
    qd = torch.from_numpy(q).cuda()
    if how == "adaptive":
        phi, grad = f.adaptive_evaluate(qd)
    elif how == "partition":
        phi, grad = f.partition_evaluate(qd)
    else:
        phi, grad = f.evaluate(qd)
    torch.cuda.synchronize()
    failed, ink = f.debug_check()
    out["cases"][name] = {"failed": failed, "in_kernel": ink,
                          "phi": float(phi.double().sum()), "grad": float(grad.double().abs().sum()),
                          "phi_bits": phi.cpu().numpy().view(np.uint32)[:: 97].tolist()}
    f.close()
x = cube_points(20000); q = charges(20000, "u11")
for prec in ("fp32", "fp16x3"):
    f = pkg.FMM(p=4, depth=4, precision=prec, domain=((0, 0, 0), 1.0))
    f.build_tree(torch.from_numpy(x).cuda()).precompute()
    case("cube_" + prec, f, q)
f = pkg.FMM(p=4, depth=4, precision="fp16x3", domain=((0, 0, 0), 1.0))
f.build_tree(torch.from_numpy(x).cuda()).precompute()
f.partition_setup(2, 8)
case("cube_partition", f, q, "partition")
xs = sphere_points(30000); qs = charges(30000, "u01")
f = pkg.FMM(p=6, depth=5, precision="fp32", domain=((-1, -1, -1), 2.0), m2l="fft")
f.build_tree(torch.from_numpy(xs).cuda()).precompute()
case("sphere_fft", f, qs)
xm = mixed_points(12000, radius=0.02); qm = charges(12000, "u11")
f = pkg.FMM(p=4, depth=8, precision="fp32", domain=((0, 0, 0), 1.0))
f.build_tree(torch.from_numpy(xm).cuda()).precompute()
f.adaptive_setup(16)
case("mixed_adaptive", f, qm, "adaptive")
f = pkg.FMM(p=4, depth=8, precision="fp32", domain=((0, 0, 0), 1.0))
f.build_tree(torch.from_numpy(xm).cuda()).precompute()
case("mixed_deep_small_leaves", f, qm)
print("RESULT " + json.dumps(out))
"""


def _run(library):
    env = dict(os.environ, FMM_LIBRARY=library)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_debug_build_checks_pass_and_match_the_normal_build():
    normal, debug = _run("libfmm.so"), _run("libfmm_debug.so")
    assert normal["lib"].endswith("libfmm.so") and debug["lib"].endswith("libfmm_debug.so")
    assert normal["cases"].keys() == debug["cases"].keys()
    for name, c in normal["cases"].items():
        d = debug["cases"][name]
        assert c["failed"] == [] and d["failed"] == [], (name, c["failed"], d["failed"])
        assert not c["in_kernel"] and d["in_kernel"], name
        assert c["phi_bits"] == d["phi_bits"] and c["phi"] == d["phi"] and c["grad"] == d["grad"], name
