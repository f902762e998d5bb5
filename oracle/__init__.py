"""FP64 CPU oracle of the domain decomposition primal-dual method (TEST INFRASTRUCTURE).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and its
Python binding) never imports, links or calls it, and shares no code with it.

The arithmetic lives in ``dd_tv_oracle.c`` (plain loops in double precision,
following the paper step by step); this module compiles it with gcc, loads it with
ctypes and gives it a numpy interface.  Layout conventions are documented at the top
of the C file:

* image arrays are H x W row-major;
* the torn dual field (Section 2.4) is ``P1`` of shape (H + NR, W) and ``P2`` of
  shape (H, W + NC): every subdomain keeps its own copy of the normal components on
  its four sides;
* multipliers are ``lamh`` (NR - 1, W) and ``lamv`` (NC - 1, H).

Parity pins (tests/test_oracle_*.py) check it against closed forms, brute-force
QP/LP solves of tiny problems, exact operator identities and the convergence
results of the paper (Proposition 2 on DD equivalence, Theorem 2, Corollary 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from contextlib import contextmanager
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_tv_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

L2, L1, SEG = 0, 1, 2
_FID = {"l2": L2, "l1": L1, "seg": SEG, L2: L2, L1: L1, SEG: SEG}


def _compile(src: str, out: str) -> None:
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (OpenMP, no FP contraction) into oracle/_build."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        _compile(_SRC, _LIB)
    return _LIB


def source() -> str:
    """The text of dd_tv_oracle.c."""
    with open(_SRC) as fh:
        return fh.read()


def build_variant(text: str, out_dir: str) -> str:
    """Compiles a modified copy of the oracle source (``text``) into ``out_dir`` and
    returns the library path.  Used only by the tests that plant a mistake in a copy
    of the oracle to show that a pin catches it."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "dd_tv_oracle_variant.c")
    with open(src, "w") as fh:
        fh.write(text)
    out = os.path.join(out_dir, "liboracle_variant.so")
    _compile(src, out)
    return out


@contextmanager
def using_library(path: str):
    """Routes every call of this module to the oracle library at ``path`` (a build of
    ``build_variant``) for the duration of the block."""
    global _lib
    main = _load()
    lib = ctypes.CDLL(path)
    for name, fn in _SIGNATURES.items():
        g = getattr(lib, name)
        g.restype, g.argtypes = fn
    with _lock:
        _lib = lib
    try:
        yield
    finally:
        with _lock:
            _lib = main


class _Params(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("NR", ctypes.c_int), ("NC", ctypes.c_int),
                ("fidelity", ctypes.c_int), ("alpha", ctypes.c_double), ("c1", ctypes.c_double),
                ("c2", ctypes.c_double), ("tau", ctypes.c_double), ("sigma", ctypes.c_double),
                ("tau0", ctypes.c_double), ("sigma0", ctypes.c_double), ("gamma", ctypes.c_double),
                ("inner", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_ubyte)
_P = ctypes.POINTER(_Params)
_I = ctypes.POINTER(ctypes.c_int)


_i, _dd = ctypes.c_int, ctypes.c_double
_SIGNATURES = {
    "orc_prox": (None, [_i, _i, _D, _D, _U8, _dd, _dd, _dd, _D]),
    "orc_div": (None, [_i, _i, _D, _D, _D]),
    "orc_grad": (None, [_i, _i, _D, _D, _D]),
    "orc_tv": (_dd, [_i, _i, _D]),
    "orc_fidelity": (_dd, [_i, _i, _D, _D, _U8, _dd, _dd]),
    "orc_energy": (_dd, [_P, _D, _D, _U8]),
    "orc_dual_value": (_dd, [_P, _D, _D, _D, _U8]),
    "orc_jump": (None, [_P, _D, _D, _D, _D]),
    "orc_jump_adjoint": (None, [_P, _D, _D, _D, _D]),
    "orc_tile_div": (None, [_i, _i, _D, _D, _D]),
    "orc_tile_grad": (None, [_i, _i, _i, _i, _i, _i, _D, _D, _D]),
    "orc_local_solve": (None, [_P, _i, _i, _i, _i, _i, _i, _D, _U8, _D, _D, _D, _D, _D, _i]),
    "orc_dd_run": (_i, [_P, _D, _U8, _i, _D, _D, _D, _D, _D, _D, _D, _D]),
    "orc_dd_run_ex": (_i, [_P, _D, _U8, _i, _dd, _I, _I, _D, _D, _D, _D, _D, _D, _D, _D, _D]),
    "orc_cp_run": (_i, [_P, _D, _U8, _i, _D, _D, _D, _D, _D]),
    "orc_rof_accel_run": (_i, [_P, _D, _i, _D, _D, _D, _D, _D]),
    "orc_torn_to_global": (None, [_P, _D, _D, _D, _D]),
}


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _u8(a):
    if a is None:
        return None
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(_U8)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _mask(m):
    return None if m is None else np.ascontiguousarray(m, dtype=np.uint8)


def part_start(a: int, length: int, n: int) -> int:
    """First pixel row/column of tile a when ``length`` is split into n tiles."""
    return (a * length) // n


@dataclass
class Problem:
    """The model problem and method parameters (Section 3, Algorithm 1, Section 5).

    Defaults are the paper's experimental settings: tau = 50, sigma tau = 1/2,
    tau_0 = 10, sigma_0 tau_0 = 1/8, gamma = 1/(8 tau)."""

    H: int
    W: int
    NR: int = 1
    NC: int = 1
    fidelity: int | str = L2
    alpha: float = 10.0
    c1: float = 0.0
    c2: float = 0.0
    tau: float = 50.0
    sigma: float | None = None
    tau0: float = 10.0
    sigma0: float | None = None
    gamma: float | None = None
    inner: int = 10

    def c(self) -> _Params:
        sigma = self.sigma if self.sigma is not None else 0.5 / self.tau
        sigma0 = self.sigma0 if self.sigma0 is not None else 0.125 / self.tau0
        gamma = self.gamma if self.gamma is not None else 1.0 / (8.0 * self.tau)
        return _Params(self.H, self.W, self.NR, self.NC, _FID[self.fidelity], self.alpha, self.c1, self.c2,
                       self.tau, sigma, self.tau0, sigma0, gamma, self.inner)


@dataclass
class DDState:
    """State of Algorithm 1 between outer iterations."""

    u: np.ndarray
    P1: np.ndarray
    P2: np.ndarray
    P1prev: np.ndarray
    P2prev: np.ndarray
    lamh: np.ndarray
    lamv: np.ndarray
    n: int = 0
    energies: list = field(default_factory=list)

    def copy(self) -> "DDState":
        return DDState(self.u.copy(), self.P1.copy(), self.P2.copy(), self.P1prev.copy(), self.P2prev.copy(),
                       self.lamh.copy(), self.lamv.copy(), self.n, list(self.energies))


def initial_u(pr: Problem, f: np.ndarray, mask=None) -> np.ndarray:
    """u^0: f (with f = 0 on D) for L2/L1 fidelities, 1/2 for segmentation."""
    if _FID[pr.fidelity] == SEG:
        return np.full((pr.H, pr.W), 0.5)
    u = np.array(f, dtype=np.float64, copy=True)
    if mask is not None:
        u[np.asarray(mask) != 0] = 0.0
    return u


def dd_init(pr: Problem, f: np.ndarray, mask=None) -> DDState:
    """p~^0 = p~^{-1} = 0, lambda^0 = 0, u^0 from ``initial_u``."""
    H, W, NR, NC = pr.H, pr.W, pr.NR, pr.NC
    return DDState(initial_u(pr, f, mask), np.zeros((H + NR, W)), np.zeros((H, W + NC)),
                   np.zeros((H + NR, W)), np.zeros((H, W + NC)), np.zeros((NR - 1, W)), np.zeros((NC - 1, H)))


def dd_run(pr: Problem, f: np.ndarray, n_outer: int, state: DDState | None = None, mask=None,
           trace: bool = False, inner_tol: float = 0.0, counts=None, record: bool = False) -> DDState:
    """Runs ``n_outer`` iterations of Algorithm 1 (in place on ``state``).

    inner_tol > 0: adaptive inner stopping (Section 5, eq. stop_inner1) with at most
    ``pr.inner`` iterations.  counts: int array (n_outer, NR*NC) forcing the inner
    iterations of every local solve.  record: keep, on the state, ``inner_counts``
    (n_outer, NR*NC) and ``inner_res`` (n_outer, NR*NC, pr.inner; NaN past the last
    iteration), the relative change of p of every inner iteration."""
    lib = _load()
    f64 = _f64(f)
    m = _mask(mask)
    st = state if state is not None else dd_init(pr, f64, m)
    tr = np.zeros(max(n_outer, 1)) if trace else None
    p = pr.c()
    T = pr.NR * pr.NC
    cin = None
    if counts is not None:
        cin = np.ascontiguousarray(counts, dtype=np.int32).reshape(n_outer, T)
        if cin.min(initial=1) < 0 or cin.max(initial=0) > pr.inner:
            raise ValueError("forced inner counts must lie in [0, inner]")
    cout = np.zeros((max(n_outer, 1), T), dtype=np.int32) if record else None
    res = np.full((max(n_outer, 1), T, pr.inner), np.nan) if record else None
    ip = lambda a: None if a is None else a.ctypes.data_as(_I)
    lib.orc_dd_run_ex(ctypes.byref(p), _d(f64), _u8(m), n_outer, float(inner_tol), ip(cin), ip(cout), _d(res),
                      _d(st.u), _d(st.P1), _d(st.P2), _d(st.P1prev), _d(st.P2prev), _d(st.lamh), _d(st.lamv),
                      _d(tr))
    st.n += n_outer
    if trace:
        st.energies.extend(tr[:n_outer].tolist())
    if record:
        st.inner_counts = cout[:n_outer]
        st.inner_res = res[:n_outer]
    return st


@dataclass
class CPState:
    u: np.ndarray
    p1: np.ndarray
    p2: np.ndarray
    pb1: np.ndarray
    pb2: np.ndarray
    n: int = 0


def cp_init(pr: Problem, f, mask=None) -> CPState:
    H, W = pr.H, pr.W
    return CPState(initial_u(pr, f, mask), np.zeros((H + 1, W)), np.zeros((H, W + 1)), np.zeros((H + 1, W)),
                   np.zeros((H, W + 1)))


def cp_run(pr: Problem, f, iters: int, state: CPState | None = None, mask=None) -> CPState:
    """Plain primal-dual iteration on the undecomposed problem (N = 1 comparator)."""
    lib = _load()
    f64 = _f64(f)
    m = _mask(mask)
    st = state if state is not None else cp_init(pr, f64, m)
    p = pr.c()
    lib.orc_cp_run(ctypes.byref(p), _d(f64), _u8(m), iters, _d(st.u), _d(st.p1), _d(st.p2), _d(st.pb1),
                   _d(st.pb2))
    st.n += iters
    return st


@dataclass
class AccelState:
    u: np.ndarray
    ubar: np.ndarray
    p1: np.ndarray
    p2: np.ndarray
    steps: np.ndarray
    n: int = 0


def rof_accel_init(pr: Problem, f) -> AccelState:
    H, W = pr.H, pr.W
    u = np.array(f, dtype=np.float64, copy=True)
    # t0 s0 ||D||^2 <= 1 with ||D||^2 <= 8
    return AccelState(u, u.copy(), np.zeros((H + 1, W)), np.zeros((H, W + 1)),
                      np.array([1.0 / np.sqrt(8.0), 1.0 / np.sqrt(8.0)]))


def rof_accel_run(pr: Problem, f, iters: int, state: AccelState | None = None) -> AccelState:
    """Accelerated full-dimension ROF iteration (u strongly convex), for J*."""
    lib = _load()
    f64 = _f64(f)
    st = state if state is not None else rof_accel_init(pr, f64)
    p = pr.c()
    lib.orc_rof_accel_run(ctypes.byref(p), _d(f64), iters, _d(st.u), _d(st.ubar), _d(st.p1), _d(st.p2),
                          _d(st.steps))
    st.n += iters
    return st


# ---------------------------------------------------------------- small helpers

def energy(pr: Problem, u, f, mask=None) -> float:
    lib = _load()
    p = pr.c()
    return lib.orc_energy(ctypes.byref(p), _d(_f64(u)), _d(_f64(f)), _u8(_mask(mask)))


def tv(u) -> float:
    u = _f64(u)
    return _load().orc_tv(u.shape[0], u.shape[1], _d(u))


def dual_value(pr: Problem, p1, p2, f, mask=None) -> float:
    p = pr.c()
    return _load().orc_dual_value(ctypes.byref(p), _d(_f64(p1)), _d(_f64(p2)), _d(_f64(f)), _u8(_mask(mask)))


def prox(fid, v, f, s, mask=None, c1=0.0, c2=0.0):
    v, f = _f64(v), _f64(f)
    out = np.empty_like(v)
    _load().orc_prox(_FID[fid], v.size, _d(v), _d(f), _u8(_mask(mask)), s, c1, c2, _d(out))
    return out


def div(p1, p2):
    p1, p2 = _f64(p1), _f64(p2)
    H, W = p2.shape[0], p1.shape[1]
    out = np.empty((H, W))
    _load().orc_div(H, W, _d(p1), _d(p2), _d(out))
    return out


def grad(u):
    u = _f64(u)
    H, W = u.shape
    g1, g2 = np.empty((H + 1, W)), np.empty((H, W + 1))
    _load().orc_grad(H, W, _d(u), _d(g1), _d(g2))
    return g1, g2


def tile_div(p1, p2):
    p1, p2 = _f64(p1), _f64(p2)
    mr, mc = p2.shape[0], p1.shape[1]
    out = np.empty((mr, mc))
    _load().orc_tile_div(mr, mc, _d(p1), _d(p2), _d(out))
    return out


def tile_grad(u, top, bottom, left, right):
    u = _f64(u)
    mr, mc = u.shape
    g1, g2 = np.empty((mr + 1, mc)), np.empty((mr, mc + 1))
    _load().orc_tile_grad(mr, mc, int(top), int(bottom), int(left), int(right), _d(u), _d(g1), _d(g2))
    return g1, g2


def jump(pr: Problem, P1, P2):
    jh = np.zeros((max(pr.NR - 1, 0), pr.W))
    jv = np.zeros((max(pr.NC - 1, 0), pr.H))
    p = pr.c()
    _load().orc_jump(ctypes.byref(p), _d(_f64(P1)), _d(_f64(P2)), _d(jh) if jh.size else None,
                     _d(jv) if jv.size else None)
    return jh, jv


def jump_adjoint(pr: Problem, lamh, lamv):
    P1 = np.zeros((pr.H + pr.NR, pr.W))
    P2 = np.zeros((pr.H, pr.W + pr.NC))
    p = pr.c()
    lh, lv = _f64(lamh), _f64(lamv)
    _load().orc_jump_adjoint(ctypes.byref(p), _d(lh) if lh.size else None, _d(lv) if lv.size else None,
                             _d(P1), _d(P2))
    return P1, P2


def local_solve(pr: Problem, f, u, p1, p2, ph1, ph2, iters, sides=(1, 1, 1, 1), mask=None):
    """One local solve on a single tile (in place on u, p1, p2); ph1/ph2 None => no proximal term."""
    mr, mc = u.shape
    p = pr.c()
    _load().orc_local_solve(ctypes.byref(p), mr, mc, *[int(s) for s in sides], _d(_f64(f)), _u8(_mask(mask)),
                            _d(u), _d(p1), _d(p2), _d(_f64(ph1)), _d(_f64(ph2)), iters)


def torn_to_global(pr: Problem, P1, P2):
    p1 = np.zeros((pr.H + 1, pr.W))
    p2 = np.zeros((pr.H, pr.W + 1))
    p = pr.c()
    _load().orc_torn_to_global(ctypes.byref(p), _d(_f64(P1)), _d(_f64(P2)), _d(p1), _d(p2))
    return p1, p2


def global_to_torn(pr: Problem, p1, p2):
    """Duplicates every interface dof of a global field into both tiles' copies."""
    H, W, NR, NC = pr.H, pr.W, pr.NR, pr.NC
    P1 = np.zeros((H + NR, W))
    P2 = np.zeros((H, W + NC))
    for a in range(NR):
        r0, r1 = part_start(a, H, NR), part_start(a + 1, H, NR)
        P1[r0 + a:r1 + a + 1, :] = p1[r0:r1 + 1, :]
    for b in range(NC):
        c0, c1 = part_start(b, W, NC), part_start(b + 1, W, NC)
        P2[:, c0 + b:c1 + b + 1] = p2[:, c0:c1 + 1]
    return P1, P2


def dd_gap(pr: Problem, st: DDState, f, mask=None):
    """(J(u), d(p_avg)) for a DD iterate; d is -inf where no certificate exists."""
    p1, p2 = torn_to_global(pr, st.P1, st.P2)
    return energy(pr, st.u, f, mask), dual_value(pr, p1, p2, f, mask)
