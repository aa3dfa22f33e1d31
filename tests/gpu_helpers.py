"""Shared helpers of the GPU tests: contexts over seeded workloads and error norms."""
import numpy as np

import paper_2604_19243_gb300 as pkg

PINV_RTOL = 1e-7
SVD_RTOL = 1e-6


def rel(a, b):
    """Relative L2 error of a against b (complex values keep their imaginary parts)."""
    cplx = np.iscomplexobj(a) or np.iscomplexobj(b)
    dt = np.complex128 if cplx else np.float64
    a = np.asarray(a, dtype=dt).ravel()
    b = np.asarray(b, dtype=dt).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_fmm(x, p, depth, precision="fp32", domain=None, with_gradient=True, mean_free=False, **kw):
    import torch
    dt = torch.float64 if precision == "fp64" else torch.float32
    f = pkg.FMM(p=p, depth=depth, precision=precision, domain=domain, pinv_rtol=PINV_RTOL,
                svd_rtol=SVD_RTOL, with_gradient=with_gradient, mean_free=mean_free, **kw)
    f.build_tree(torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt))
    f.precompute()
    return f


def run(f, q, gradient=True, parts=pkg.PART_ALL):
    import torch
    dt = torch.float64 if f.precision == "fp64" else torch.float32
    phi, grad = f.evaluate(torch.from_numpy(np.ascontiguousarray(q)).to("cuda", dt), gradient, parts)
    torch.cuda.synchronize()
    return phi.cpu().numpy().astype(np.float64), (grad.cpu().numpy().astype(np.float64) if gradient else None)
