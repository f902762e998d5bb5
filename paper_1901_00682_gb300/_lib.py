"""ctypes binding of the dd_tv C ABI (include/dd_tv.h).

Argument marshalling only: every step of the solver runs in libddtv.so.  Loading
fails loudly (ImportError) when the library has not been built; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libddtv.so")

L2, L1, SEG = 0, 1, 2
PATH_FUSED, PATH_PLAIN, PATH_FULLDIM = 0, 1, 2
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTCONV, EUNSUPPORTED = range(7)
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOTCONV", 6: "EUNSUPPORTED"}
MAX_INNER = 1024
N_VARIANTS = 4  # hardware mappings of exact 128 x 128 subdomains (dd_tv_params.variant)


class Params(ctypes.Structure):
    _fields_ = [
        ("height", ctypes.c_int), ("width", ctypes.c_int),
        ("sub_rows", ctypes.c_int), ("sub_cols", ctypes.c_int),
        ("fidelity", ctypes.c_int),
        ("alpha", ctypes.c_double), ("c1", ctypes.c_double), ("c2", ctypes.c_double),
        ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
        ("tau", ctypes.c_double), ("sigma", ctypes.c_double),
        ("tau0", ctypes.c_double), ("sigma0", ctypes.c_double), ("gamma", ctypes.c_double),
        ("outer_tol", ctypes.c_double), ("energy_ref", ctypes.c_double),
        ("energy_every", ctypes.c_int), ("path", ctypes.c_int), ("variant", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("outer_done", ctypes.c_int), ("pixel_iters", ctypes.c_longlong),
        ("energy", ctypes.c_double), ("rel_err", ctypes.c_double),
        ("ms", ctypes.c_double), ("converged", ctypes.c_int), ("inner_max", ctypes.c_int),
    ]


# every symbol the header declares, with (restype, argtypes)
_vp, _i, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_PP = ctypes.POINTER(Params)
_SP = ctypes.POINTER(Stats)
_DP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "dd_tv_default_params": (None, [_PP]),
    "dd_tv_create": (_i, [ctypes.POINTER(_vp), _PP]),
    "dd_tv_destroy": (_i, [_vp]),
    "dd_tv_last_error": (ctypes.c_char_p, [_vp]),
    "dd_tv_set_stream": (_i, [_vp, _vp]),
    "dd_tv_solve": (_i, [_vp, _vp, _vp, _vp, _SP]),
    "dd_tv_solve_device": (_i, [_vp, _vp, _vp, _vp, _SP]),
    "dd_tv_load": (_i, [_vp, _vp, _vp]),
    "dd_tv_iterate": (_i, [_vp, _i]),
    "dd_tv_get_u": (_i, [_vp, _vp]),
    "dd_tv_outer_count": (_i, [_vp]),
    "dd_tv_inner_counts": (_i, [_vp, _vp, _vp]),
    "dd_tv_get_state": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "dd_tv_set_state": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i]),
    "dd_tv_energy": (_i, [_vp, _vp, _vp, _vp, _DP]),
    "dd_tv_gap": (_i, [_vp, _DP, _DP]),
    "dd_tv_current_energy": (_i, [_vp, _DP]),
    "dd_tv_set_profiling": (_i, [_vp, _i]),
    "dd_tv_profile_read": (_i, [_vp, _DP, ctypes.POINTER(ctypes.c_longlong)]),
    "dd_tv_measure_smem_bandwidth": (_i, [_DP]),
    "dd_tv_energy_noalloc": (_i, [_vp, _vp, _vp, _i, _i, _i, _d, _d, _d, _vp, _DP]),
    "dd_tv_batch_create": (_i, [ctypes.POINTER(_vp), _vp, _i, _vp]),
    "dd_tv_batch_destroy": (_i, [_vp]),
    "dd_tv_batch_last_error": (ctypes.c_char_p, [_vp]),
    "dd_tv_batch_set_stream": (_i, [_vp, _vp]),
    "dd_tv_batch_load": (_i, [_vp, _vp]),
    "dd_tv_batch_iterate": (_i, [_vp, _i]),
    "dd_tv_batch_get_u": (_i, [_vp, _i, _vp]),
    "dd_tv_batch_energy": (_i, [_vp, _i, _DP]),
    "dd_tv_batch_pixels": (ctypes.c_longlong, [_vp]),
    "dd_tv_adjoint_forward": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "dd_tv_adjoint_backward": (_i, [_vp, _vp, _vp, _DP]),
    "dd_tv_adjoint_release": (_i, [_vp]),
    "dd_tv_set_alpha": (_i, [_vp, _d]),
    "dd_tv_fault_probe": (_i, [_vp, _i, _DP]),
    "dd_tv_create_shard": (_i, [ctypes.POINTER(_vp), _PP, _i, _i]),
    "dd_tv_shard_rows": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "dd_tv_shard_export": (_i, [_vp, _vp, _vp]),
    "dd_tv_shard_import": (_i, [_vp, _vp, _vp]),
    "dd_tv_shard_edge_rows": (_i, [_vp, _vp, _vp]),
    "dd_tv_shard_energy": (_i, [_vp, _vp, _DP]),
}

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Loads libddtv.so (raises ImportError if it is missing: build it first)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"{path} not found: build the CUDA library with "
                                  "`python -m paper_1901_00682_gb300.build`")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class DDTVError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def check(code: int, handle=None):
    if code != OK:
        msg = load().dd_tv_last_error(handle)
        raise DDTVError(code, msg.decode() if msg else "")


def measure_smem_bandwidth() -> float:
    """Shared-memory load bandwidth of the current device in GB/s (probe kernel)."""
    v = ctypes.c_double()
    check(load().dd_tv_measure_smem_bandwidth(ctypes.byref(v)), None)
    return v.value


def default_params() -> Params:
    p = Params()
    load().dd_tv_default_params(ctypes.byref(p))
    return p


def make_params(height, width, sub_rows=1, sub_cols=1, fidelity=L2, alpha=10.0, c1=0.0, c2=0.0,
                outer_iters=100, inner_iters=10, tau=None, sigma=None, tau0=10.0, sigma0=None,
                gamma=None, outer_tol=0.0, energy_ref=math.nan, energy_every=5, path=PATH_FUSED,
                variant=0, inner_tol=0.0) -> Params:
    """Params with the paper's defaults (Section 5) for every unspecified step size:
    tau = 50 (1 for segmentation), sigma = 1/(2 tau), sigma0 = 1/(8 tau0),
    gamma = 1/(8 tau)."""
    fid = {"l2": L2, "l1": L1, "seg": SEG}.get(fidelity, fidelity)
    p = default_params()
    tau = tau if tau is not None else (1.0 if fid == SEG else 50.0)
    p.height, p.width, p.sub_rows, p.sub_cols = height, width, sub_rows, sub_cols
    p.fidelity, p.alpha, p.c1, p.c2 = fid, alpha, c1, c2
    p.outer_iters, p.inner_iters = outer_iters, inner_iters
    p.tau = tau
    p.sigma = sigma if sigma is not None else 0.5 / tau
    p.tau0 = tau0
    p.sigma0 = sigma0 if sigma0 is not None else 0.125 / tau0
    p.gamma = gamma if gamma is not None else 1.0 / (8.0 * tau)
    p.outer_tol, p.energy_ref, p.energy_every = outer_tol, energy_ref, energy_every
    p.path = {"fused": PATH_FUSED, "plain": PATH_PLAIN, "fulldim": PATH_FULLDIM}.get(path, path)
    p.variant = variant
    p.inner_tol = inner_tol
    return p


def _ptr(t):
    """Raw pointer of a torch tensor / numpy array / int / None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


class Solver:
    """Owns one dd_tv handle.  Device tensors are torch CUDA tensors (float32/uint8,
    contiguous); work runs on torch's current stream unless `stream` is given."""

    def __init__(self, params: Params, stream=None, shard=None):
        """shard = (tile_row_begin, tile_row_end): a row-block shard of the problem
        `params` describes (dd_tv_create_shard); None: the whole image."""
        self.lib = load()
        self.params = params
        h = ctypes.c_void_p()
        if shard is None:
            check(self.lib.dd_tv_create(ctypes.byref(h), ctypes.byref(params)), None)
        else:
            check(self.lib.dd_tv_create_shard(ctypes.byref(h), ctypes.byref(params), int(shard[0]),
                                              int(shard[1])), None)
        self.h = h
        self.shard = shard
        self.set_stream(stream)

    def set_stream(self, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        check(self.lib.dd_tv_set_stream(self.h, ctypes.c_void_p(s)), self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.dd_tv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls
    def load(self, f, mask=None):
        check(self.lib.dd_tv_load(self.h, _ptr(f), _ptr(mask)), self.h)

    def iterate(self, n_outer: int):
        check(self.lib.dd_tv_iterate(self.h, int(n_outer)), self.h)

    def get_u(self, out):
        check(self.lib.dd_tv_get_u(self.h, _ptr(out)), self.h)
        return out

    def outer_count(self) -> int:
        return self.lib.dd_tv_outer_count(self.h)

    def inner_counts(self):
        """(counts of the last outer iteration, sub_rows x sub_cols int array; the
        largest count since the last load / solve / call)."""
        import numpy as np
        p = self.params
        NR, NC = (1, 1) if p.path == PATH_FULLDIM else (p.sub_rows, p.sub_cols)
        out = np.zeros((NR, NC), dtype=np.int32)
        mx = ctypes.c_int()
        check(self.lib.dd_tv_inner_counts(self.h, out.ctypes.data, ctypes.byref(mx)), self.h)
        return out, mx.value

    def solve_host(self, f_host, mask_host=None, u_host=None):
        """dd_tv_solve on host numpy arrays; returns (u, Stats, status)."""
        import numpy as np
        f_host = np.ascontiguousarray(f_host, dtype=np.float32)
        if mask_host is not None:
            mask_host = np.ascontiguousarray(mask_host, dtype=np.uint8)
        if u_host is None:
            u_host = np.empty_like(f_host)
        st = Stats()
        rc = self.lib.dd_tv_solve(self.h, _ptr(f_host), _ptr(mask_host), _ptr(u_host), ctypes.byref(st))
        if rc not in (OK, ENOTCONV):
            check(rc, self.h)
        return u_host, st, rc

    def solve_device(self, f, mask=None, u=None, stats=True):
        import torch
        if u is None:
            u = torch.empty_like(f)
        st = Stats() if stats else None
        rc = self.lib.dd_tv_solve_device(self.h, _ptr(f), _ptr(mask), _ptr(u),
                                         ctypes.byref(st) if stats else None)
        if rc not in (OK, ENOTCONV):
            check(rc, self.h)
        return u, st, rc

    def get_state(self):
        """State as torch tensors in the torn exchange layout (see include/dd_tv.h)."""
        import torch
        p = self.params
        full = p.path == PATH_FULLDIM
        NR, NC = (1, 1) if full else (p.sub_rows, p.sub_cols)
        H, W = p.height, p.width
        dev = torch.device("cuda")
        z = lambda *s: torch.zeros(*s, dtype=torch.float32, device=dev)
        u, P1, P2 = z(H, W), z(H + NR, W), z(H, W + NC)
        lamh, lamv = z(NR - 1, W), z(NC - 1, H)
        P1p, P2p = z(H + NR, W), z(H, W + NC)
        check(self.lib.dd_tv_get_state(self.h, _ptr(u), _ptr(P1), _ptr(P2), _ptr(lamh) if lamh.numel() else None,
                                       _ptr(lamv) if lamv.numel() else None, _ptr(P1p), _ptr(P2p)), self.h)
        return dict(u=u, P1=P1, P2=P2, lamh=lamh, lamv=lamv, P1prev=P1p, P2prev=P2p)

    def set_state(self, st, outer_count: int):
        check(self.lib.dd_tv_set_state(self.h, _ptr(st["u"]), _ptr(st["P1"]), _ptr(st["P2"]),
                                       _ptr(st["lamh"]) if st["lamh"].numel() else None,
                                       _ptr(st["lamv"]) if st["lamv"].numel() else None,
                                       _ptr(st["P1prev"]), _ptr(st["P2prev"]), int(outer_count)), self.h)

    def energy(self, u, f, mask=None) -> float:
        J = ctypes.c_double()
        check(self.lib.dd_tv_energy(self.h, _ptr(u), _ptr(f), _ptr(mask), ctypes.byref(J)), self.h)
        return J.value

    def current_energy(self) -> float:
        J = ctypes.c_double()
        check(self.lib.dd_tv_current_energy(self.h, ctypes.byref(J)), self.h)
        return J.value

    def set_profiling(self, on: bool):
        check(self.lib.dd_tv_set_profiling(self.h, 1 if on else 0), self.h)

    def profile_read(self):
        """({'interface','local','energy'} -> summed ms, same keys -> launches)."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_longlong * 3)()
        check(self.lib.dd_tv_profile_read(self.h, ms, n), self.h)
        keys = ("interface", "local", "energy")
        return dict(zip(keys, list(ms))), dict(zip(keys, list(n)))

    def gap(self):
        J, D = ctypes.c_double(), ctypes.c_double()
        check(self.lib.dd_tv_gap(self.h, ctypes.byref(J), ctypes.byref(D)), self.h)
        return J.value, D.value

    def fault_probe(self, kind: int):
        """Forces the timeout path (kind 0: a bounded device wait that runs out; kind 1:
        the status word set from the host).  Returns (status code, message, device ms
        of the wait); DD_TV_ETIMEOUT is the expected code."""
        ms = ctypes.c_double()
        rc = self.lib.dd_tv_fault_probe(self.h, int(kind), ctypes.byref(ms))
        msg = self.lib.dd_tv_last_error(self.h)
        return rc, (msg.decode() if msg else ""), ms.value

    def set_alpha(self, alpha: float):
        check(self.lib.dd_tv_set_alpha(self.h, float(alpha)), self.h)
        self.params.alpha = float(alpha)

    def adjoint_forward(self, f, mask, n_outer: int, checkpoint_every: int, u_out):
        """u_N of n_outer outer iterations from f, keeping checkpoints for the reverse pass."""
        check(self.lib.dd_tv_adjoint_forward(self.h, _ptr(f), _ptr(mask), int(n_outer), int(checkpoint_every),
                                             _ptr(u_out)), self.h)
        return u_out

    def adjoint_backward(self, grad_u, grad_f_out) -> float:
        """Writes dL/df into grad_f_out and returns dL/dalpha for dL/du_N = grad_u."""
        ga = ctypes.c_double()
        check(self.lib.dd_tv_adjoint_backward(self.h, _ptr(grad_u), _ptr(grad_f_out), ctypes.byref(ga)), self.h)
        return ga.value

    # -- row-block shards
    def shard_rows(self):
        """(first image row, rows) of the handle's image."""
        r0, n = ctypes.c_int(), ctypes.c_int()
        check(self.lib.dd_tv_shard_rows(self.h, ctypes.byref(r0), ctypes.byref(n)), self.h)
        return r0.value, n.value

    def shard_export(self, top, bottom):
        check(self.lib.dd_tv_shard_export(self.h, _ptr(top), _ptr(bottom)), self.h)

    def shard_import(self, above, below):
        check(self.lib.dd_tv_shard_import(self.h, _ptr(above), _ptr(below)), self.h)

    def shard_edge_rows(self, first, last):
        check(self.lib.dd_tv_shard_edge_rows(self.h, _ptr(first), _ptr(last)), self.h)

    def shard_energy(self, row_below) -> float:
        J = ctypes.c_double()
        check(self.lib.dd_tv_shard_energy(self.h, _ptr(row_below), ctypes.byref(J)), self.h)
        return J.value

    def adjoint_release(self):
        check(self.lib.dd_tv_adjoint_release(self.h), self.h)


class BatchImage(ctypes.Structure):
    _fields_ = [("height", ctypes.c_int), ("width", ctypes.c_int), ("fidelity", ctypes.c_int),
                ("alpha", ctypes.c_double), ("c1", ctypes.c_double), ("c2", ctypes.c_double),
                ("tau", ctypes.c_double), ("sigma", ctypes.c_double)]


class BatchParams(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("inner_iters", ctypes.c_int), ("tau0", ctypes.c_double),
                ("sigma0", ctypes.c_double), ("variant", ctypes.c_int)]


def _bcheck(code, handle):
    if code != OK:
        msg = load().dd_tv_batch_last_error(handle)
        raise DDTVError(code, msg.decode() if msg else "")


class Batch:
    """Owns one dd_tv_batch handle: many images solved together (Algorithm 1 per image).

    images: list of dicts with height, width, fidelity ("l2", "l1", "seg" or code),
    alpha, c1, c2 and optionally tau, sigma (defaults: the paper's per fidelity)."""

    def __init__(self, images, inner_iters=10, tau0=10.0, sigma0=None, variant=0, stream=None, tile=128):
        self.lib = load()
        self.tile = tile
        n = len(images)
        arr = (BatchImage * n)()
        for k, im in enumerate(images):
            fid = {"l2": L2, "l1": L1, "seg": SEG}.get(im.get("fidelity", L2), im.get("fidelity", L2))
            arr[k] = BatchImage(im["height"], im["width"], fid, im.get("alpha", 10.0), im.get("c1", 0.0),
                                im.get("c2", 0.0), im.get("tau", 0.0), im.get("sigma", 0.0))
        bp = BatchParams(tile, inner_iters, tau0, sigma0 if sigma0 is not None else 0.125 / tau0, variant)
        h = ctypes.c_void_p()
        _bcheck(self.lib.dd_tv_batch_create(ctypes.byref(h), arr, n, ctypes.byref(bp)), None)
        self.h = h
        self.n = n
        self.images = images
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        _bcheck(self.lib.dd_tv_batch_set_stream(self.h, ctypes.c_void_p(s)), self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.dd_tv_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, fs):
        ptrs = (ctypes.c_void_p * self.n)(*[f.data_ptr() for f in fs])
        self._keep = fs
        _bcheck(self.lib.dd_tv_batch_load(self.h, ptrs), self.h)

    def iterate(self, n_outer):
        _bcheck(self.lib.dd_tv_batch_iterate(self.h, int(n_outer)), self.h)

    def get_u(self, i, out):
        _bcheck(self.lib.dd_tv_batch_get_u(self.h, int(i), out.data_ptr()), self.h)
        return out

    def energy(self, i):
        J = ctypes.c_double()
        _bcheck(self.lib.dd_tv_batch_energy(self.h, int(i), ctypes.byref(J)), self.h)
        return J.value

    def pixels(self):
        return self.lib.dd_tv_batch_pixels(self.h)
