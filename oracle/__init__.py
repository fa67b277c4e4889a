"""FP64 CPU oracle for FOFSE (Seiler & Kaup, arXiv 2207.01205) -- test infrastructure.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never does; the two share no code.

The arithmetic lives in ``fofse_oracle.c`` (plain C, IEEE double, no FP
contraction), compiled on first use with gcc into ``oracle/_build``.  This
module only marshals numpy arrays into it.  The algorithm and the readings of
the paper it takes are documented at the top of the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fofse_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfofse_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS_OK, STATUS_NO_SUPPORT, STATUS_NONFINITE = 0, 1, 2


class OraclePlan(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("border", ctypes.c_int), ("fft_size", ctypes.c_int),
                ("iters", ctypes.c_int), ("support", ctypes.c_int), ("rho", ctypes.c_double),
                ("gamma", ctypes.c_double), ("compensation", ctypes.c_int), ("basis", ctypes.c_int)]


class OracleVolumePlan(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("border", ctypes.c_int), ("depth", ctypes.c_int),
                ("fft_size", ctypes.c_int), ("fft_time", ctypes.c_int), ("iters", ctypes.c_int),
                ("rho", ctypes.c_double), ("gamma", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, IEEE double, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # FOFSE_ORACLE_LIB: a build of a deliberately broken copy of the
            # oracle, loaded by the mutation test to show that a pin fails
            _lib = ctypes.CDLL(os.environ.get("FOFSE_ORACLE_LIB") or build())
            _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_fp = ctypes.POINTER(ctypes.c_float)
_u8p = ctypes.POINTER(ctypes.c_ubyte)
_c_int, _c_double = ctypes.c_int, ctypes.c_double


def _declare(L):
    L.oracle_distance.argtypes = [_c_int, _c_int, _dp]
    L.oracle_weights.argtypes = [_c_int, _c_int, _c_int, _c_double, _u8p, _dp]
    L.oracle_cut_area.argtypes = [_fp, _u8p, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int,
                                  _dp, _u8p]
    L.oracle_project.argtypes = [_c_int, _c_int, _dp, _dp, _dp]
    L.oracle_select.argtypes = [_c_int, _dp, _dp, _ip, _ip, _dp]
    L.oracle_extrapolate_area.argtypes = [_c_int, _c_int, _dp, _dp, _c_double, _c_int, _dp, _ip, _ip,
                                          _dp, _dp, _dp, _dp]
    L.oracle_extrapolate_area.restype = _c_int
    L.oracle_extrapolate_area_fd.argtypes = L.oracle_extrapolate_area.argtypes
    L.oracle_extrapolate_area_fd.restype = _c_int
    L.oracle_replay_area.argtypes = [_c_int, _c_int, _dp, _dp, _c_double, _c_int, _ip, _ip, _dp, _dp,
                                     _dp, _dp]
    L.oracle_replay_area.restype = _c_int
    L.oracle_adjoint_area.argtypes = [_c_int, _c_int, _dp, _dp, _c_double, _c_int, _ip, _ip, _dp, _dp,
                                      _dp, _dp]
    L.oracle_adjoint_area.restype = _c_int
    L.oracle_adjoint_area_dct.argtypes = L.oracle_adjoint_area.argtypes
    L.oracle_adjoint_area_dct.restype = _c_int
    L.oracle_replay_area_dct.argtypes = [_c_int, _c_int, _dp, _dp, _c_double, _c_int, _ip, _ip, _dp,
                                         _dp, _dp]
    L.oracle_replay_area_dct.restype = _c_int
    L.oracle_rho_chain.argtypes = [_c_int, _dp, _dp, _c_double, _dp]
    L.oracle_rho_chain.restype = _c_double
    L.oracle_tangent_area.argtypes = [_c_int, _c_int, _dp, _dp, _dp, _c_double, _c_double, _c_int,
                                      _ip, _ip, _dp]
    L.oracle_tangent_area.restype = _c_int
    L.oracle_batch.argtypes = [_fp, _u8p, _c_int, _c_int, _c_int, _ip, _c_int,
                               ctypes.POINTER(OraclePlan), _c_int, _c_int, _dp, _ip, _dp, _ip, _ip,
                               _dp, _dp, _dp, _c_int]
    L.oracle_batch.restype = _c_int
    L.oracle_batch_mode.argtypes = L.oracle_batch.argtypes + [_c_int, _dp, _dp]
    L.oracle_extrapolate_area_ofse.argtypes = [_c_int, _c_int, _dp, _dp, _c_int, _dp, _ip, _ip, _dp,
                                               _dp, _dp, _dp, _dp, _dp]
    L.oracle_extrapolate_area_ofse.restype = _c_int
    L.oracle_extrapolate_area_dct.argtypes = [_c_int, _c_int, _dp, _dp, ctypes.c_double, _c_int, _dp,
                                              _ip, _ip, _dp, _dp, _dp]
    L.oracle_extrapolate_area_dct.restype = _c_int
    L.oracle_error_curve.argtypes = [_c_int, _c_int, _c_int, _c_int, _ip, _ip, _dp, _dp, _c_int, _dp, _dp,
                                     _c_int]
    L.oracle_error_curve.restype = None
    L.oracle_batch_mode.restype = _c_int
    L.oracle_batch_adjoint.argtypes = [_fp, _u8p, _c_int, _c_int, _c_int, _ip, _c_int,
                                       ctypes.POINTER(OraclePlan), _c_int, _ip, _ip, _c_int, _dp,
                                       _c_int, _dp, _dp, _c_int]
    L.oracle_batch_adjoint.restype = _c_int
    L.oracle_distance3.argtypes = [_c_int, _c_int, _c_int, _dp]
    L.oracle_weights3.argtypes = [_c_int, _c_int, _c_int, _c_double, _u8p, _dp]
    L.oracle_cut_volume.argtypes = [_fp, _u8p] + [_c_int] * 10 + [_dp, _u8p]
    L.oracle_project3.argtypes = [_c_int, _c_int, _c_int, _c_int, _dp, _dp, _dp]
    L.oracle_select3.argtypes = [_c_int, _c_int, _dp, _dp, _ip, _dp]
    L.oracle_extrapolate_volume.argtypes = [_c_int, _c_int, _c_int, _c_int, _dp, _dp, _c_double,
                                            _c_int, _dp, _ip, _dp, _dp, _dp, _dp]
    L.oracle_extrapolate_volume.restype = _c_int
    L.oracle_batch_volume.argtypes = [_fp, _u8p, _c_int, _c_int, _c_int, _c_int, _ip, _c_int,
                                      ctypes.POINTER(OracleVolumePlan), _dp, _ip, _dp, _ip, _dp,
                                      _dp, _dp, _c_int]
    L.oracle_batch_volume.restype = _c_int
    L.oracle_batch_volume_mode.argtypes = L.oracle_batch_volume.argtypes + [_c_int]
    L.oracle_batch_volume_mode.restype = _c_int
    L.oracle_extrapolate_volume_fd.argtypes = L.oracle_extrapolate_volume.argtypes
    L.oracle_extrapolate_volume_fd.restype = _c_int
    L.oracle_replay_volume.argtypes = [_c_int, _c_int, _c_int, _c_int, _dp, _dp, _c_double, _c_int,
                                       _ip, _dp, _dp, _dp, _dp]
    L.oracle_replay_volume.restype = _c_int
    L.oracle_adjoint_volume.argtypes = [_c_int, _c_int, _c_int, _c_int, _dp, _dp, _c_double, _c_int,
                                        _ip, _dp, _dp, _dp, _dp]
    L.oracle_adjoint_volume.restype = _c_int


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ----------------------------------------------------------------------------
# single-area functions
# ----------------------------------------------------------------------------

def distance(block: int, border: int) -> np.ndarray:
    Ls = block + 2 * border
    d = np.empty((Ls, Ls))
    lib().oracle_distance(block, border, _p(d, _dp))
    return d


def weights(block: int, border: int, rho: float, avail_L: np.ndarray, support: int = 0) -> np.ndarray:
    """Eq. 4 with the isotropic model of Eq. 15 over the area L."""
    Ls = block + 2 * border
    a = np.ascontiguousarray(avail_L, dtype=np.uint8).reshape(Ls, Ls)
    w = np.empty((Ls, Ls))
    lib().oracle_weights(block, border, support, float(rho), _p(a, _u8p), _p(w, _dp))
    return w


def cut_area(frame, avail, y, x, block, border):
    frame = np.ascontiguousarray(frame, dtype=np.float32)
    avail = np.ascontiguousarray(avail, dtype=np.uint8)
    H, W = frame.shape
    Ls = block + 2 * border
    fL = np.empty((Ls, Ls))
    aL = np.empty((Ls, Ls), dtype=np.uint8)
    lib().oracle_cut_area(_p(frame, _fp), _p(avail, _u8p), H, W, W, int(y), int(x), block, border,
                          _p(fL, _dp), _p(aL, _u8p))
    return fL, aL


def project(rw: np.ndarray, T: int) -> np.ndarray:
    """All T^2 weighted projections P[k] = sum rw exp(-j2pi k.x/T) (Eq. 8)."""
    rw = _f64(rw)
    Ls = rw.shape[0]
    pr = np.empty((T, T))
    pi = np.empty((T, T))
    lib().oracle_project(Ls, T, _p(rw, _dp), _p(pr, _dp), _p(pi, _dp))
    return pr + 1j * pi


def select(P: np.ndarray):
    """Eq. 9 over the canonical set; returns (u1, u2, relative gap)."""
    T = P.shape[0]
    pr, pi = _f64(P.real), _f64(P.imag)
    u1, u2, gap = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    lib().oracle_select(T, _p(pr, _dp), _p(pi, _dp), ctypes.byref(u1), ctypes.byref(u2),
                        ctypes.byref(gap))
    return u1.value, u2.value, gap.value


class AreaResult:
    def __init__(self, status, g, u, dc, gap, w0):
        self.status, self.g, self.u, self.dc, self.gap, self.w0 = status, g, u, dc, gap, w0


def extrapolate_area(fL, wL, T: int, gamma: float, iters: int, transform_domain: bool = False) -> AreaResult:
    """Spatial re-projection FOFSE over one area L (Sec. 2); with
    ``transform_domain`` the paper's transform-domain form instead."""
    fL, wL = _f64(fL), _f64(wL)
    Ls = fL.shape[0]
    g = np.empty((Ls, Ls))
    u1 = np.zeros(iters, dtype=np.int32)
    u2 = np.zeros(iters, dtype=np.int32)
    dr = np.zeros(iters)
    di = np.zeros(iters)
    gap = np.zeros(iters)
    w0 = ctypes.c_double()
    fn = lib().oracle_extrapolate_area_fd if transform_domain else lib().oracle_extrapolate_area
    st = fn(Ls, T, _p(fL, _dp), _p(wL, _dp), float(gamma), iters,
                                       _p(g, _dp), _p(u1, _ip), _p(u2, _ip), _p(dr, _dp),
                                       _p(di, _dp), _p(gap, _dp), ctypes.byref(w0))
    return AreaResult(st, g, np.stack([u1, u2], axis=1), dr + 1j * di, gap, w0.value)


def extrapolate_area_ofse(fL, wL, T: int, iters: int):
    """Spatial re-projection with OFSE's compensation (Eq. 10-13); returns the
    AreaResult and the compensation factors gamma_u per iteration (complex)."""
    fL, wL = _f64(fL), _f64(wL)
    Ls = fL.shape[0]
    g = np.empty((Ls, Ls))
    u1 = np.zeros(iters, dtype=np.int32)
    u2 = np.zeros(iters, dtype=np.int32)
    dr, di, gr, gi, gap = (np.zeros(iters) for _ in range(5))
    w0 = ctypes.c_double()
    st = lib().oracle_extrapolate_area_ofse(Ls, T, _p(fL, _dp), _p(wL, _dp), iters, _p(g, _dp),
                                            _p(u1, _ip), _p(u2, _ip), _p(dr, _dp), _p(di, _dp),
                                            _p(gr, _dp), _p(gi, _dp), _p(gap, _dp),
                                            ctypes.byref(w0))
    return AreaResult(st, g, np.stack([u1, u2], axis=1), dr + 1j * di, gap, w0.value), gr + 1j * gi


def extrapolate_area_dct(fL, wL, T: int, gamma: float, iters: int) -> AreaResult:
    """FOFSE with the 2-D DCT-II basis (spatial re-projection, FP64); dc real."""
    fL, wL = _f64(fL), _f64(wL)
    Ls = fL.shape[0]
    g = np.empty((Ls, Ls))
    u1 = np.zeros(iters, dtype=np.int32)
    u2 = np.zeros(iters, dtype=np.int32)
    dc, gap = np.zeros(iters), np.zeros(iters)
    w0 = ctypes.c_double()
    st = lib().oracle_extrapolate_area_dct(Ls, T, _p(fL, _dp), _p(wL, _dp), float(gamma), iters,
                                           _p(g, _dp), _p(u1, _ip), _p(u2, _ip), _p(dc, _dp),
                                           _p(gap, _dp), ctypes.byref(w0))
    return AreaResult(st, g, np.stack([u1, u2], axis=1), dc.astype(complex), gap, w0.value)


def error_curve(Ls: int, T: int, block: int, border: int, path, dc, truth_B, basis: int = 0) -> np.ndarray:
    """Squared error over B (model clipped to [0, 255]) after each iteration of
    the given path and coefficients (Fig. 4 / Fig. 5 quantity); basis 0 = DFT
    pairs, 1 = DCT-II."""
    path = np.ascontiguousarray(np.asarray(path).reshape(-1, 2), dtype=np.int32)
    u1, u2 = np.ascontiguousarray(path[:, 0]), np.ascontiguousarray(path[:, 1])
    dc = np.asarray(dc)
    dr, di = _f64(dc.real), _f64(dc.imag)
    tb = _f64(truth_B)
    n = path.shape[0]
    out = np.zeros(n)
    lib().oracle_error_curve(Ls, T, block, border, _p(u1, _ip), _p(u2, _ip), _p(dr, _dp),
                             _p(di, _dp), n, _p(tb, _dp), _p(out, _dp), int(basis))
    return out


def replay_area(fL, wL, T: int, gamma: float, path) -> tuple:
    """Forward along a fixed path; returns (g over L, coefficients)."""
    fL, wL = _f64(fL), _f64(wL)
    path = _i32(path)
    Ls, iters = fL.shape[0], path.shape[0]
    u1, u2 = _i32(path[:, 0]), _i32(path[:, 1])
    g = np.empty((Ls, Ls))
    dr = np.zeros(iters)
    di = np.zeros(iters)
    lib().oracle_replay_area(Ls, T, _p(fL, _dp), _p(wL, _dp), float(gamma), iters, _p(u1, _ip),
                             _p(u2, _ip), _p(g, _dp), _p(dr, _dp), _p(di, _dp), None)
    return g, dr + 1j * di


def adjoint_area(fL, wL, T: int, gamma: float, path, gbar, basis: int = 0):
    """Reverse-mode adjoint along a fixed path: returns (fbar, wbar, gammabar);
    basis 0 = DFT pairs, 1 = DCT-II."""
    fL, wL, gbar = _f64(fL), _f64(wL), _f64(gbar)
    path = _i32(path)
    Ls, iters = fL.shape[0], path.shape[0]
    u1, u2 = _i32(path[:, 0]), _i32(path[:, 1])
    fbar = np.empty((Ls, Ls))
    wbar = np.empty((Ls, Ls))
    gb = ctypes.c_double()
    fn = lib().oracle_adjoint_area_dct if basis == 1 else lib().oracle_adjoint_area
    fn(Ls, T, _p(fL, _dp), _p(wL, _dp), float(gamma), iters, _p(u1, _ip), _p(u2, _ip),
       _p(gbar, _dp), _p(fbar, _dp), _p(wbar, _dp), ctypes.byref(gb))
    return fbar, wbar, gb.value


def replay_area_dct(fL, wL, T: int, gamma: float, path) -> tuple:
    """DCT-II basis: forward along a fixed path; returns (g over L, coefficients)."""
    fL, wL = _f64(fL), _f64(wL)
    path = _i32(path)
    Ls, iters = fL.shape[0], path.shape[0]
    u1, u2 = _i32(path[:, 0]), _i32(path[:, 1])
    g = np.empty((Ls, Ls))
    dc = np.zeros(iters)
    lib().oracle_replay_area_dct(Ls, T, _p(fL, _dp), _p(wL, _dp), float(gamma), iters, _p(u1, _ip),
                                 _p(u2, _ip), _p(g, _dp), _p(dc, _dp), None)
    return g, dc


def rho_chain(wL, dist, rho, wbar) -> float:
    wL, dist, wbar = _f64(wL), _f64(dist), _f64(wbar)
    return lib().oracle_rho_chain(wL.size, _p(wL, _dp), _p(dist, _dp), float(rho), _p(wbar, _dp))


def tangent_area(fL, wL, wdot, T: int, gamma: float, gamma_dot: float, path):
    """Forward-mode derivative of the final model along a fixed path."""
    fL, wL, wdot = _f64(fL), _f64(wL), _f64(wdot)
    path = _i32(path)
    Ls, iters = fL.shape[0], path.shape[0]
    u1, u2 = _i32(path[:, 0]), _i32(path[:, 1])
    gdot = np.empty((Ls, Ls))
    lib().oracle_tangent_area(Ls, T, _p(fL, _dp), _p(wL, _dp), _p(wdot, _dp), float(gamma),
                              float(gamma_dot), iters, _p(u1, _ip), _p(u2, _ip), _p(gdot, _dp))
    return gdot


# ----------------------------------------------------------------------------
# batches
# ----------------------------------------------------------------------------

class BatchResult:
    """blocks: (n, bmax, bmax) B estimates (unclipped); status, w0 per block;
    path (n, imax, 2), dc (n, imax) complex, gap (n, imax) per iteration."""

    def __init__(self, blocks, status, w0, path, dc, gap, threads):
        self.blocks, self.status, self.w0 = blocks, status, w0
        self.path, self.dc, self.gap, self.threads = path, dc, gap, threads


def plans_to_c(plans):
    arr = (OraclePlan * len(plans))()
    for i, p in enumerate(plans):
        arr[i] = OraclePlan(p.block, p.border, p.fft_size, p.iters, getattr(p, "support", 0),
                            float(p.rho), float(p.gamma), int(getattr(p, "compensation", 0)),
                            int(getattr(p, "basis", 0)))
    return arr


def run_batch(frame, avail, blocks, plans, threads: int | None = None, with_path: bool = True,
              transform_domain: bool = False) -> BatchResult:
    """Extrapolate every block of ``blocks`` ((n, 3) int: y, x, plan index);
    ``transform_domain`` runs the transform-domain form (the CPU program timed
    beside the GPU) instead of the spatial re-projection."""
    frame = np.ascontiguousarray(frame, dtype=np.float32)
    avail = np.ascontiguousarray(avail, dtype=np.uint8)
    blocks = _i32(blocks).reshape(-1, 3)
    H, W = frame.shape
    n = blocks.shape[0]
    bmax = max(p.block for p in plans)
    imax = max(p.iters for p in plans)
    out = np.zeros((n, bmax * bmax))
    status = np.zeros(n, dtype=np.int32)
    w0 = np.zeros(n)
    u1 = np.zeros((n, imax), dtype=np.int32) if with_path else None
    u2 = np.zeros((n, imax), dtype=np.int32) if with_path else None
    dr = np.zeros((n, imax)) if with_path else None
    di = np.zeros((n, imax)) if with_path else None
    gap = np.zeros((n, imax)) if with_path else None
    gre = np.zeros((n, imax)) if with_path else None
    gim = np.zeros((n, imax)) if with_path else None
    cplans = plans_to_c(plans)
    threads = threads or os.cpu_count() or 1
    used = lib().oracle_batch_mode(_p(frame, _fp), _p(avail, _u8p), H, W, W, _p(blocks, _ip), n,
                                   cplans, bmax * bmax, imax, _p(out, _dp), _p(status, _ip),
                                   _p(w0, _dp), _p(u1, _ip), _p(u2, _ip), _p(dr, _dp), _p(di, _dp),
                                   _p(gap, _dp), threads, 1 if transform_domain else 0,
                                   _p(gre, _dp), _p(gim, _dp))
    res_blocks = np.zeros((n, bmax, bmax))
    for i in range(n):
        b = plans[blocks[i, 2]].block
        res_blocks[i, :b, :b] = out[i, :b * b].reshape(b, b)
    path = np.stack([u1, u2], axis=2) if with_path else None
    dc = (dr + 1j * di) if with_path else None
    res = BatchResult(res_blocks, status, w0, path, dc, gap, used)
    res.ofse_gamma = (gre + 1j * gim) if with_path else None  # per iteration, OFSE plans only
    return res


def block_gradients(frame, avail, y, x, plan, path, e_B):
    """Oracle adjoint of one block along ``path``: dloss/df on L (only A),
    dloss/drho and dloss/dgamma, with e_B = dloss/dB (b x b)."""
    b, br = plan.block, plan.border
    fL, aL = cut_area(frame, avail, y, x, b, br)
    wL = weights(b, br, plan.rho, aL, getattr(plan, "support", 0))
    Ls = b + 2 * br
    gbar = np.zeros((Ls, Ls))
    gbar[br:br + b, br:br + b] = e_B
    fbar, wbar, gam = adjoint_area(fL, wL, plan.fft_size, plan.gamma, path, gbar)
    rho_bar = rho_chain(wL, distance(b, br), plan.rho, wbar)
    return fbar, rho_bar, gam


def batch_adjoint(frame, avail, blocks, plans, path, e_blocks, threads: int | None = None):
    """Frozen-path gradients of sum_i <e_i, B_hat_i> over a batch: returns
    (grad_frame (H, W), grad_rho_gamma (n_plans, 2)).  ``path``: (n, imax, 2)
    int selection paths; ``e_blocks``: (n, bmax, bmax) dloss/dB."""
    frame = np.ascontiguousarray(frame, dtype=np.float32)
    avail = np.ascontiguousarray(avail, dtype=np.uint8)
    blocks = _i32(blocks).reshape(-1, 3)
    H, W = frame.shape
    n = blocks.shape[0]
    imax = path.shape[1]
    u1 = _i32(path[:, :, 0])
    u2 = _i32(path[:, :, 1])
    bmax = e_blocks.shape[1]
    e = np.zeros((n, bmax * bmax))
    for i in range(n):
        b = plans[blocks[i, 2]].block
        e[i, :b * b] = np.asarray(e_blocks[i, :b, :b], dtype=np.float64).ravel()
    gf = np.zeros((H, W))
    grg = np.zeros((len(plans), 2))
    lib().oracle_batch_adjoint(_p(frame, _fp), _p(avail, _u8p), H, W, W, _p(blocks, _ip), n,
                               plans_to_c(plans), len(plans), _p(u1, _ip), _p(u2, _ip), imax,
                               _p(e, _dp), bmax * bmax, _p(gf, _dp), _p(grg, _dp),
                               threads or os.cpu_count() or 1)
    return gf, grg


# ----------------------------------------------------------------------------
# video volumes (the method over three-dimensional sets, Sec. 1)
# ----------------------------------------------------------------------------

def distance3(block: int, border: int, depth: int) -> np.ndarray:
    """(Lt, Ls, Ls) distances to the centre of B in the centre frame."""
    Ls, Lt = block + 2 * border, 2 * depth + 1
    d = np.empty((Lt, Ls, Ls))
    lib().oracle_distance3(block, border, depth, _p(d, _dp))
    return d


def weights3(block: int, border: int, depth: int, rho: float, avail_L: np.ndarray) -> np.ndarray:
    aL = np.ascontiguousarray(avail_L, dtype=np.uint8)
    w = np.empty(aL.shape)
    lib().oracle_weights3(block, border, depth, float(rho), _p(aL, _u8p), _p(w, _dp))
    return w


def cut_volume(video, avail, t, y, x, block, border, depth):
    """(fL, aL) of the volume around B (top-left (y, x) in frame t)."""
    video = np.ascontiguousarray(video, dtype=np.float32)
    avail = np.ascontiguousarray(avail, dtype=np.uint8)
    F, H, W = video.shape
    Ls, Lt = block + 2 * border, 2 * depth + 1
    fL = np.empty((Lt, Ls, Ls))
    aL = np.empty((Lt, Ls, Ls), dtype=np.uint8)
    lib().oracle_cut_volume(_p(video, _fp), _p(avail, _u8p), F, H, W, W, int(t), int(y), int(x),
                            block, border, depth, _p(fL, _dp), _p(aL, _u8p))
    return fL, aL


def project3(rw: np.ndarray, T: int, Tt: int) -> np.ndarray:
    """P[k1, k2, k3] = sum rw exp(-j2pi (k1 m / T + k2 n / T + k3 tau / Tt)),
    rw indexed (tau, m, n); returns shape (T, T, Tt)."""
    rw = _f64(rw)
    Lt, Ls = rw.shape[0], rw.shape[1]
    pr = np.empty((T, T, Tt))
    pi = np.empty((T, T, Tt))
    lib().oracle_project3(Lt, Ls, T, Tt, _p(rw, _dp), _p(pr, _dp), _p(pi, _dp))
    return pr + 1j * pi


def select3(P: np.ndarray):
    """Eq. 9 over the canonical set of the 3-D grid; returns ((u1, u2, u3), gap)."""
    T, Tt = P.shape[0], P.shape[2]
    pr, pi = _f64(P.real), _f64(P.imag)
    u = np.zeros(3, dtype=np.int32)
    gap = ctypes.c_double()
    lib().oracle_select3(T, Tt, _p(pr, _dp), _p(pi, _dp), _p(u, _ip), ctypes.byref(gap))
    return tuple(int(v) for v in u), gap.value


def extrapolate_volume(fL, wL, T: int, Tt: int, gamma: float, iters: int,
                       transform_domain: bool = False) -> AreaResult:
    """FOFSE over one volume (spatial re-projection; with ``transform_domain``
    the transform-domain form): g (Lt, Ls, Ls), path (iters, 3), dc complex,
    gap, w0."""
    fL, wL = _f64(fL), _f64(wL)
    Lt, Ls = fL.shape[0], fL.shape[1]
    g = np.empty((Lt, Ls, Ls))
    path = np.zeros((iters, 3), dtype=np.int32)
    dr, di, gap = np.zeros(iters), np.zeros(iters), np.zeros(iters)
    w0 = ctypes.c_double()
    fn = lib().oracle_extrapolate_volume_fd if transform_domain else lib().oracle_extrapolate_volume
    st = fn(Lt, Ls, T, Tt, _p(fL, _dp), _p(wL, _dp), float(gamma), iters, _p(g, _dp),
            _p(path, _ip), _p(dr, _dp), _p(di, _dp), _p(gap, _dp), ctypes.byref(w0))
    return AreaResult(st, g, path, dr + 1j * di, gap, w0.value)


def run_batch_volume(video, avail, blocks, plan, threads: int | None = None,
                     transform_domain: bool = False) -> BatchResult:
    """Extrapolate every block of ``blocks`` ((n, 3) int: t, y, x) of a video
    (F, H, W) with one volume plan (fields block, border, depth, fft_size,
    fft_time, rho, gamma, iters).  path (n, iters, 3).  ``transform_domain``
    runs the transform-domain form instead of the spatial re-projection."""
    video = np.ascontiguousarray(video, dtype=np.float32)
    avail = np.ascontiguousarray(avail, dtype=np.uint8)
    blocks = _i32(blocks).reshape(-1, 3)
    F, H, W = video.shape
    n, b, it = blocks.shape[0], plan.block, plan.iters
    out = np.zeros((n, b, b))
    status = np.zeros(n, dtype=np.int32)
    w0 = np.zeros(n)
    path = np.zeros((n, it, 3), dtype=np.int32)
    dr, di, gap = np.zeros((n, it)), np.zeros((n, it)), np.zeros((n, it))
    cp = OracleVolumePlan(plan.block, plan.border, plan.depth, plan.fft_size, plan.fft_time,
                          plan.iters, float(plan.rho), float(plan.gamma))
    threads = threads or os.cpu_count() or 1
    used = lib().oracle_batch_volume_mode(_p(video, _fp), _p(avail, _u8p), F, H, W, W,
                                          _p(blocks, _ip), n, ctypes.byref(cp), _p(out, _dp),
                                          _p(status, _ip), _p(w0, _dp), _p(path, _ip),
                                          _p(dr, _dp), _p(di, _dp), _p(gap, _dp), threads,
                                          1 if transform_domain else 0)
    return BatchResult(out, status, w0, path, dr + 1j * di, gap, used)


def replay_volume(fL, wL, T: int, Tt: int, gamma: float, path) -> tuple:
    """The volume recursion along a given path ((iters, 3)): (status, g, dc)."""
    fL, wL = _f64(fL), _f64(wL)
    path = _i32(path).reshape(-1, 3)
    Lt, Ls, iters = fL.shape[0], fL.shape[1], path.shape[0]
    g = np.empty(fL.shape)
    dr, di = np.zeros(iters), np.zeros(iters)
    st = lib().oracle_replay_volume(Lt, Ls, T, Tt, _p(fL, _dp), _p(wL, _dp), float(gamma), iters,
                                    _p(path, _ip), _p(g, _dp), _p(dr, _dp), _p(di, _dp), None)
    return st, g, dr + 1j * di


def adjoint_volume(fL, wL, T: int, Tt: int, gamma: float, path, gbar):
    """Reverse-mode adjoint of the volume recursion along ``path`` for the
    loss <gbar, g>: (fbar, wbar, gammabar)."""
    fL, wL, gbar = _f64(fL), _f64(wL), _f64(gbar)
    path = _i32(path).reshape(-1, 3)
    Lt, Ls, iters = fL.shape[0], fL.shape[1], path.shape[0]
    fbar, wbar = np.empty(fL.shape), np.empty(fL.shape)
    gam = ctypes.c_double()
    lib().oracle_adjoint_volume(Lt, Ls, T, Tt, _p(fL, _dp), _p(wL, _dp), float(gamma), iters,
                                _p(path, _ip), _p(gbar, _dp), _p(fbar, _dp), _p(wbar, _dp),
                                ctypes.byref(gam))
    return fbar, wbar, gam.value
