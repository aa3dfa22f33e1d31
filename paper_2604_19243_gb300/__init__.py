"""Python binding of libfmm, a GB300 (sm_103a) kernel-independent FMM for the 3D Laplace kernel,
the modified Helmholtz kernel exp(-kappa r) / (4 pi r) (`kernel="yukawa"`) and the Helmholtz
kernel exp(i kappa r) / (4 pi r) with complex densities (`kernel="helmholtz"`).

Argument marshalling only: every step of the FMM runs in the CUDA library behind the C ABI of
include/fmm.h.  Importing this package does not build anything; call
`paper_2604_19243_gb300.build.build()` first.  If the library is missing, every call raises.

    fmm = FMM(p=6, depth=5, precision="fp16x3", domain=((0, 0, 0), 1.0))
    fmm.build_tree(x)            # x: (N, 3) float32 torch tensor (CUDA or CPU) or NumPy array
    fmm.precompute()
    phi, grad = fmm.evaluate(q)  # same device and dtype as q
    _, grad = fmm.evaluate(q, potential=False)   # gradient only
    psi, _ = fmm.adjoint(g)      # the transpose of q -> phi
    fmm.partition_setup(3, 64)   # the distributed scheme on 64 virtual ranks of this GPU
    phi, grad = fmm.partition_evaluate(q)        # equal to evaluate(q) bit for bit
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# FMM_LIBRARY selects another build of the library by file name within _build/ (the tests load
# the bounds-checked libfmm_debug.so this way); the default is libfmm.so
LIB_PATH = os.path.join(HERE, "_build", os.path.basename(os.environ.get("FMM_LIBRARY", "libfmm.so")))

PRECISIONS = {"fp32": 0, "fp64": 1, "tf32x3": 2, "bf16x3": 3, "bf16x6": 4, "fp16x3": 5}
STATUS = {0: "FMM_OK", 1: "FMM_EINVAL", 2: "FMM_ENOMEM", 3: "FMM_ECUDA", 4: "FMM_ESTATE",
          5: "FMM_ETIMEOUT", 6: "FMM_EUNSUPPORTED"}
PART_NEAR, PART_FAR, PART_ALL = 1, 2, 3
KERNELS = {"laplace": 0, "yukawa": 1, "helmholtz": 2}

# C entry points declared in include/fmm.h (checked by the export test)
ENTRY_POINTS = ("fmm_default_options", "fmm_create", "fmm_build_tree", "fmm_precompute",
                "fmm_evaluate", "fmm_evaluate_parts", "fmm_adjoint", "fmm_get_tree_info",
                "fmm_export_tree", "fmm_export_level", "fmm_export_check", "fmm_last_timings",
                "fmm_sync", "fmm_sort_points_noalloc", "fmm_kernel_launches",
                "fmm_measure_fp32_peak", "fmm_partition_setup", "fmm_partition_evaluate",
                "fmm_partition_info", "fmm_partition_export", "fmm_partition_timings",
                "fmm_adaptive_setup", "fmm_adaptive_info", "fmm_adaptive_export", "fmm_adaptive_evaluate",
                "fmm_set_wait_limit", "fmm_set_alloc_limit", "fmm_debug_check", "fmm_last_error", "fmm_destroy")
DEBUG_BITS = {"perm": 1 << 0, "leaf": 1 << 1, "ulist": 1 << 2, "keys": 1 << 3, "tree": 1 << 4, "class": 1 << 5,
              "order": 1 << 6, "p2p": 1 << 7, "scatter": 1 << 8, "sort": 1 << 9}


class Options(ctypes.Structure):
    _fields_ = [("order_p", ctypes.c_int), ("depth", ctypes.c_int), ("precision", ctypes.c_int),
                ("svd_rtol", ctypes.c_double), ("pinv_rtol", ctypes.c_double),
                ("with_gradient", ctypes.c_int), ("has_domain", ctypes.c_int),
                ("origin", ctypes.c_double * 3), ("side", ctypes.c_double),
                ("mean_free", ctypes.c_int), ("kernel", ctypes.c_int), ("kappa", ctypes.c_double),
                ("m2l", ctypes.c_int)]


class TreeInfo(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("depth", ctypes.c_int32),
                ("n_surface", ctypes.c_int32), ("m2l_rank_in", ctypes.c_int32),
                ("m2l_rank_out", ctypes.c_int32), ("n_boxes", ctypes.c_int64 * 11),
                ("n_u_entries", ctypes.c_int64), ("p2p_pairs", ctypes.c_int64),
                ("origin", ctypes.c_double * 3), ("side", ctypes.c_double)]


class RankInfo(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("n_ranks", ctypes.c_int32), ("d_global", ctypes.c_int32),
                ("n_local_roots", ctypes.c_int32), ("first_root", ctypes.c_int64),
                ("first_point", ctypes.c_int64), ("n_points", ctypes.c_int64),
                ("n_boxes", ctypes.c_int64 * 11), ("n_ghost_v", ctypes.c_int64 * 11),
                ("n_ghost_u", ctypes.c_int64), ("n_ghost_points", ctypes.c_int64),
                ("n_query_u", ctypes.c_int64), ("n_query_v", ctypes.c_int64),
                ("n_neighbours_u", ctypes.c_int32), ("n_neighbours_v", ctypes.c_int32),
                ("bytes_u", ctypes.c_int64), ("bytes_v", ctypes.c_int64),
                ("bytes_gather", ctypes.c_int64), ("bytes_scatter", ctypes.c_int64)]


class AdaptiveTreeInfo(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int32), ("n_rows", ctypes.c_int64),
                ("n_leaves", ctypes.c_int64 * 11), ("n_refined", ctypes.c_int64 * 11),
                ("n_entries", ctypes.c_int64 * 4)]


# fmm_adaptive_export kinds
ADAPTIVE_STATE, ADAPTIVE_COUNT, ADAPTIVE_U, ADAPTIVE_V, ADAPTIVE_W, ADAPTIVE_X = range(6)

# fmm_partition_export kinds
PARTITION_OWN, PARTITION_GHOST_V, PARTITION_GHOST_U = 0, 1, 2
PARTITION_NEIGHBOURS_U, PARTITION_NEIGHBOURS_V, PARTITION_LAYOUT = 3, 4, 5
PARTITION_PHASES = ("densities_u_exchange", "local_upward", "v_exchange", "gather", "global",
                    "scatter", "local_downward", "uli_tail", "output", "total")


class FmmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None


def lib():
    """The loaded libfmm (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfmm is not built ({LIB_PATH} missing); run "
                               "paper_2604_19243_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        sigs = {
            "fmm_default_options": [ctypes.POINTER(Options)],
            "fmm_create": [ctypes.POINTER(Options), vp, ctypes.POINTER(vp)],
            "fmm_build_tree": [vp, vp, i64],
            "fmm_precompute": [vp],
            "fmm_evaluate": [vp, vp, vp, vp],
            "fmm_evaluate_parts": [vp, vp, vp, vp, i32],
            "fmm_adjoint": [vp, vp, vp, vp],
            "fmm_get_tree_info": [vp, ctypes.POINTER(TreeInfo)],
            "fmm_export_tree": [vp, vp, vp, vp, vp, vp],
            "fmm_export_level": [vp, i32, vp, vp, vp, vp, vp],
            "fmm_export_check": [vp, i32, i32, vp],
            "fmm_last_timings": [vp, vp, i32],
            "fmm_sync": [vp],
            "fmm_sort_points_noalloc": [vp, i64, i32, vp, ctypes.c_double, vp, vp, vp],
            "fmm_measure_fp32_peak": [i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
            "fmm_partition_setup": [vp, i32, i32],
            "fmm_partition_evaluate": [vp, vp, vp, vp],
            "fmm_partition_info": [vp, i32, ctypes.POINTER(RankInfo)],
            "fmm_partition_export": [vp, i32, i32, i32, vp, vp],
            "fmm_partition_timings": [vp, vp, i32],
            "fmm_adaptive_setup": [vp, i32],
            "fmm_adaptive_info": [vp, ctypes.POINTER(AdaptiveTreeInfo)],
            "fmm_adaptive_export": [vp, i32, vp, vp, vp],
            "fmm_adaptive_evaluate": [vp, vp, vp, vp, i32],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.fmm_set_wait_limit.argtypes = [vp, ctypes.c_double]
        L.fmm_set_wait_limit.restype = ctypes.c_int
        L.fmm_debug_check.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int32)]
        L.fmm_debug_check.restype = ctypes.c_int
        L.fmm_set_alloc_limit.argtypes = [ctypes.c_size_t]
        L.fmm_set_alloc_limit.restype = None
        L.fmm_kernel_launches.argtypes = []
        L.fmm_kernel_launches.restype = ctypes.c_longlong
        L.fmm_last_error.argtypes = [vp]
        L.fmm_last_error.restype = ctypes.c_char_p
        L.fmm_destroy.argtypes = [vp]
        L.fmm_destroy.restype = None
        _lib = L
    return _lib


def _ptr(a):
    """Raw address of a torch tensor or NumPy array (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def kernel_launches():
    """Kernels launched by libfmm in this process so far."""
    return int(lib().fmm_kernel_launches())


def set_alloc_limit(nbytes=None):
    """Process-wide cap on any single device allocation of the library (None: no cap); a larger
    request makes the call that needed it fail with FMM_ENOMEM (failure injection)."""
    lib().fmm_set_alloc_limit(ctypes.c_size_t(-1).value if nbytes is None else int(nbytes))


def measure_fp32_peak(iters=2048):
    """FP32 FMA throughput of the current device in TFLOP/s: (scalar, float2 form)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    st = lib().fmm_measure_fp32_peak(int(iters), ctypes.byref(a), ctypes.byref(b))
    if st != 0:
        raise FmmError(st, "fmm_measure_fp32_peak failed")
    return a.value, b.value


class FMM:
    """One FMM context: a tree over a point set and the operators of one expansion order."""

    def __init__(self, p=6, depth=4, precision="fp32", svd_rtol=1e-6, pinv_rtol=1e-7,
                 with_gradient=True, domain=None, stream=None, mean_free=False, kernel="laplace",
                 kappa=0.0, m2l="dense"):
        L = lib()
        opt = Options()
        L.fmm_default_options(ctypes.byref(opt))
        opt.order_p, opt.depth = p, depth
        opt.precision = PRECISIONS[precision]
        opt.svd_rtol, opt.pinv_rtol = svd_rtol, pinv_rtol
        opt.with_gradient = int(with_gradient)
        opt.mean_free = int(mean_free)
        opt.kernel = KERNELS[kernel]
        opt.kappa = float(kappa)
        opt.m2l = {"dense": 0, "fft": 1}[m2l]
        if domain is not None:
            opt.has_domain = 1
            for a in range(3):
                opt.origin[a] = float(domain[0][a])
            opt.side = float(domain[1])
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except Exception:
                stream = 0
        self._ctx = ctypes.c_void_p()
        st = L.fmm_create(ctypes.byref(opt), ctypes.c_void_p(stream), ctypes.byref(self._ctx))
        if st != 0:
            raise FmmError(st, "fmm_create rejected the options")
        self.p, self.depth, self.precision = p, depth, precision
        self.kernel, self.kappa = kernel, float(kappa)
        self.dtype = np.float64 if precision == "fp64" else np.float32
        # densities and outputs: complex for the Helmholtz kernel (interleaved re, im)
        self.vdtype = ((np.complex128 if precision == "fp64" else np.complex64) if kernel == "helmholtz"
                       else self.dtype)
        self.n = 0

    def _check(self, st):
        if st != 0:
            raise FmmError(st, lib().fmm_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            lib().fmm_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- marshalling helpers ------------------------------------------------------------
    def _like(self, ref, shape):
        """An output array of values (densities' dtype) beside `ref`."""
        if isinstance(ref, np.ndarray):
            return np.empty(shape, dtype=self.vdtype)
        import torch
        return torch.empty(shape, dtype=ref.dtype, device=ref.device)

    def _as_input(self, a, values=False):
        """Coordinates (values=False) or densities (values=True) in the context's types."""
        dt = self.vdtype if values else self.dtype
        if isinstance(a, np.ndarray):
            return np.ascontiguousarray(a, dtype=dt)
        import torch
        want = {np.float64: torch.float64, np.float32: torch.float32, np.complex64: torch.complex64,
                np.complex128: torch.complex128}[dt]
        return a.detach().to(want).contiguous()

    # -- C entry points -----------------------------------------------------------------
    def build_tree(self, x):
        x = self._as_input(x)
        self.n = int(x.shape[0])
        self._check(lib().fmm_build_tree(self._ctx, _ptr(x), self.n))
        return self

    def precompute(self):
        self._check(lib().fmm_precompute(self._ctx))
        return self

    def evaluate(self, q, gradient=True, parts=PART_ALL, potential=True):
        """(phi, grad); potential=False gives the gradient-only evaluation (phi is None)."""
        q = self._as_input(q, values=True)
        phi = self._like(q, (self.n,)) if potential else None
        grad = self._like(q, (self.n, 3)) if gradient else None
        self._check(lib().fmm_evaluate_parts(self._ctx, _ptr(q), _ptr(phi), _ptr(grad), parts))
        return phi, grad

    def evaluate_into(self, q, phi, grad=None, parts=PART_ALL):
        """fmm_evaluate_parts on caller-owned arrays (host or device, contiguous); phi may be
        None when grad is given (gradient only)."""
        self._check(lib().fmm_evaluate_parts(self._ctx, _ptr(q), _ptr(phi), _ptr(grad), parts))

    def adjoint(self, g, gradient=False):
        g = self._as_input(g, values=True)
        psi = self._like(g, (self.n,))
        grad = self._like(g, (self.n, 3)) if gradient else None
        self._check(lib().fmm_adjoint(self._ctx, _ptr(g), _ptr(psi), _ptr(grad)))
        return psi, grad

    def info(self):
        ti = TreeInfo()
        self._check(lib().fmm_get_tree_info(self._ctx, ctypes.byref(ti)))
        return {"n_points": ti.n_points, "depth": ti.depth, "n_surface": ti.n_surface,
                "m2l_rank_in": ti.m2l_rank_in, "m2l_rank_out": ti.m2l_rank_out,
                "n_boxes": list(ti.n_boxes)[: ti.depth + 1], "n_u_entries": ti.n_u_entries,
                "p2p_pairs": ti.p2p_pairs, "origin": list(ti.origin), "side": ti.side}

    def export_tree(self):
        inf = self.info()
        nl = inf["n_boxes"][inf["depth"]]
        perm = np.empty(self.n, np.int64)
        keys = np.empty(nl, np.uint64)
        loff = np.empty(nl + 1, np.int64)
        uoff = np.empty(nl + 1, np.int64)
        uidx = np.empty(inf["n_u_entries"], np.int64)
        self._check(lib().fmm_export_tree(self._ctx, _ptr(perm), _ptr(keys), _ptr(loff),
                                          _ptr(uoff), _ptr(uidx)))
        return {"perm": perm, "leaf_keys": keys, "leaf_offsets": loff, "u_offsets": uoff,
                "u_idx": uidx}

    def export_level(self, level, lists=True):
        inf = self.info()
        nb = inf["n_boxes"][level]
        keys = np.empty(nb, np.uint64)
        if not lists:
            self._check(lib().fmm_export_level(self._ctx, level, _ptr(keys), None, None, None, None))
            return {"keys": keys}
        cnt = ctypes.c_int64()
        off = np.empty(nb + 1, np.int64)
        self._check(lib().fmm_export_level(self._ctx, level, _ptr(keys), _ptr(off), None, None,
                                           ctypes.addressof(cnt)))
        idx = np.empty(cnt.value, np.int64)
        tv = np.empty(cnt.value, np.int32)
        self._check(lib().fmm_export_level(self._ctx, level, None, None, _ptr(idx), _ptr(tv),
                                           ctypes.addressof(cnt)))
        return {"keys": keys, "v_offsets": off, "v_idx": idx, "v_tvec": tv}

    def v_count(self, level):
        """Total length of the V lists of `level` (the lists are counted on the device, not copied)."""
        cnt = ctypes.c_int64()
        self._check(lib().fmm_export_level(self._ctx, level, None, None, None, None, ctypes.addressof(cnt)))
        return cnt.value

    def export_check(self, level, kind="upward"):
        """Check potentials of the last evaluate at `level`: n_boxes x n_surface, or n_boxes x
        2 n_surface (real parts, then imaginary parts) for the Helmholtz kernel."""
        inf = self.info()
        width = inf["n_surface"] * (2 if self.kernel == "helmholtz" else 1)
        out = np.empty((inf["n_boxes"][level], width), dtype=self.dtype)
        self._check(lib().fmm_export_check(self._ctx, level, {"upward": 0, "downward": 1}[kind],
                                           _ptr(out)))
        return out

    def sync(self):
        """Wait for the context's stream; raises if a kernel reported a device-side failure."""
        self._check(lib().fmm_sync(self._ctx))

    # -- partitioned evaluation on virtual ranks -------------------------------------------
    def partition_setup(self, d_global, n_ranks):
        """Split the built tree at d_global over n_ranks virtual ranks (needs precompute)."""
        self._check(lib().fmm_partition_setup(self._ctx, int(d_global), int(n_ranks)))

    def partition_evaluate(self, q, gradient=True, potential=True):
        """As evaluate, through the partition: (phi, grad)."""
        q = self._as_input(q, values=True)
        phi = self._like(q, (self.n,)) if potential else None
        grad = self._like(q, (self.n, 3)) if gradient else None
        self._check(lib().fmm_partition_evaluate(self._ctx, _ptr(q), _ptr(phi), _ptr(grad)))
        return phi, grad

    def partition_evaluate_into(self, q, phi, grad=None):
        self._check(lib().fmm_partition_evaluate(self._ctx, _ptr(q), _ptr(phi), _ptr(grad)))

    def partition_info(self, rank):
        ri = RankInfo()
        self._check(lib().fmm_partition_info(self._ctx, int(rank), ctypes.byref(ri)))
        out = {}
        for name, _ in RankInfo._fields_:
            v = getattr(ri, name)
            out[name] = list(v) if name in ("n_boxes", "n_ghost_v") else v
        return out

    def partition_export(self, rank, level, kind):
        cnt = ctypes.c_int64()
        self._check(lib().fmm_partition_export(self._ctx, int(rank), int(level), int(kind), None,
                                               ctypes.addressof(cnt)))
        out = np.empty(cnt.value, np.uint64)
        self._check(lib().fmm_partition_export(self._ctx, int(rank), int(level), int(kind), _ptr(out),
                                               ctypes.addressof(cnt)))
        return out

    def partition_layout(self):
        """(local root keys in Morton order, owner rank of each)."""
        v = self.partition_export(0, 0, PARTITION_LAYOUT)
        return (v & np.uint64(0xffffffff)).astype(np.int64), (v >> np.uint64(32)).astype(np.int64)

    def partition_timings(self):
        ms = np.zeros(len(PARTITION_PHASES), np.float64)
        self._check(lib().fmm_partition_timings(self._ctx, _ptr(ms), len(ms)))
        return dict(zip(PARTITION_PHASES, ms.tolist()))

    def adaptive_setup(self, capacity):
        """Adaptive tree of the current tree (refined while a box holds more than `capacity`
        points, down to the tree's depth) and its U, V, W and X lists."""
        self._check(lib().fmm_adaptive_setup(self._ctx, int(capacity)))

    def adaptive_info(self):
        ai = AdaptiveTreeInfo()
        self._check(lib().fmm_adaptive_info(self._ctx, ctypes.byref(ai)))
        depth = self.info()["depth"]
        return {"capacity": ai.capacity, "n_rows": ai.n_rows, "n_leaves": list(ai.n_leaves)[: depth + 1],
                "n_refined": list(ai.n_refined)[: depth + 1], "n_entries": list(ai.n_entries)}

    def adaptive_export(self, kind):
        """Per-row values (ADAPTIVE_STATE, ADAPTIVE_COUNT) as an array, or a list kind
        (ADAPTIVE_U .. ADAPTIVE_X) as (offsets[rows + 1], members): rows are the boxes of all
        levels, level by level, ascending Morton key within a level."""
        cnt = np.zeros(2, np.int64)
        self._check(lib().fmm_adaptive_export(self._ctx, int(kind), None, None, _ptr(cnt)))
        idx = np.empty(int(cnt[1]), np.int64)
        if kind < ADAPTIVE_U:
            self._check(lib().fmm_adaptive_export(self._ctx, int(kind), None, _ptr(idx), _ptr(cnt)))
            return idx
        off = np.empty(int(cnt[0]) + 1, np.int64)
        self._check(lib().fmm_adaptive_export(self._ctx, int(kind), _ptr(off), _ptr(idx), _ptr(cnt)))
        return off, idx

    def adaptive_evaluate(self, q, gradient=True, parts=PART_ALL, potential=True):
        """(phi, grad) over the adaptive tree of `adaptive_setup` (fmm_adaptive_evaluate)."""
        q = self._as_input(q, values=True)
        phi = self._like(q, (self.n,)) if potential else None
        grad = self._like(q, (self.n, 3)) if gradient else None
        self._check(lib().fmm_adaptive_evaluate(self._ctx, _ptr(q), _ptr(phi), _ptr(grad), parts))
        return phi, grad

    def adaptive_evaluate_into(self, q, phi, grad=None, parts=PART_ALL):
        """fmm_adaptive_evaluate on caller-owned arrays; phi may be None when grad is given."""
        self._check(lib().fmm_adaptive_evaluate(self._ctx, _ptr(q), _ptr(phi), _ptr(grad), parts))

    def debug_check(self):
        """fmm_debug_check: (names of the failed checks, whether this library has the in-kernel checks)."""
        flags, ink = ctypes.c_uint32(0), ctypes.c_int32(0)
        self._check(lib().fmm_debug_check(self._ctx, ctypes.byref(flags), ctypes.byref(ink)))
        return sorted(k for k, b in DEBUG_BITS.items() if flags.value & b), bool(ink.value)

    def set_wait_limit(self, seconds):
        """Bound on the tensor-core kernels' barrier waits (default 1 s; 0 forces the timeout path)."""
        self._check(lib().fmm_set_wait_limit(self._ctx, float(seconds)))
        return self

    def timings(self):
        """Milliseconds of the last evaluate/adjoint: near, upward, m2l, downward, total."""
        ms = np.zeros(5, np.float64)
        self._check(lib().fmm_last_timings(self._ctx, _ptr(ms), 5))
        return dict(zip(("near", "upward", "m2l", "downward", "total"), ms.tolist()))


from .autograd import FmmFunction, fmm_energy  # noqa: E402,F401
