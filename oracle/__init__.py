"""FP64 CPU oracle for the CRN particle filter and SMC^2 of arXiv 2407.17296.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA library and imports nothing from the product
package: every input arrives as a plain numpy array or integer.

Contents
  * ``philox4x32_10``, ``normals``, ``uniform_open`` -- the counter-based
    generator (Salmon et al., SC'11) and Box-Muller, in C (oracle.c);
  * ``pf`` -- one CRN particle-filter run with its forward-mode gradient
    (Sec. II, App. A, App. B), in C;
  * ``ancestors`` -- a_i = min{j : c_j >= tau_i} from normalised weights;
  * ``kalman`` -- exact linear-Gaussian log-likelihood and gradient (numpy);
  * ``smc2`` -- the outer SMC^2 sampler (Sec. III) in numpy.
"""
import ctypes
import os

import numpy as np

from .build import build_oracle

LG_DIAG = 0
SV = 1
LG_OPT = 2
SYSTEMATIC = 0
MULTINOMIAL = 1

STREAM_PROP = 0
STREAM_RESAMPLE = 1
STREAM_INIT = 2
STREAM_OUTER_XI = 3
STREAM_OUTER_NU = 4
STREAM_NUTS = 5

STAT_NAMES = ("near_ties", "tie_followed", "nontie_mismatch", "flag_ties",
              "flag_mismatch", "resample_steps", "bad_hint", "tie_conditioned")

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = build_oracle()
    lib = ctypes.CDLL(path)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint32, ctypes.c_uint32, ctypes.c_long, dp]
    lib.oracle_normals.restype = None
    lib.oracle_uniform_open.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_int]
    lib.oracle_uniform_open.restype = ctypes.c_double
    lib.oracle_ancestors.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int)]
    lib.oracle_ancestors.restype = None
    vp = ctypes.c_void_p
    lib.oracle_pf.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp,   # family dx dy D H
        vp, vp, ctypes.c_int, ctypes.c_int,                           # theta y T M
        ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,            # seed iter row
        ctypes.c_int, ctypes.c_double, ctypes.c_int,                  # scheme ess_frac want_grad
        vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_double,       # hints replay band flag_band
        ctypes.c_double,                                              # band_rel
        vp, vp, vp, vp, vp, vp]                                       # outputs
    lib.oracle_pf.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: 4 counter words, 2 key words -> 4 output words."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normals(seed, it, row, t, stream, n):
    """n standard normals of the stream (key from seed/it/row, counter (t, call, stream, 0))."""
    lib = _load()
    out = np.zeros(int(n), dtype=np.float64)
    if n:
        lib.oracle_normals(int(seed), int(it) & 0xFFFFFFFF, int(row) & 0xFFFFFFFF,
                           int(t), int(stream), int(n),
                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def uniform_open(seed, it, row, t, stream, call=0, word=0):
    """One uniform on (0,1] of the stream."""
    return float(_load().oracle_uniform_open(int(seed), int(it) & 0xFFFFFFFF,
                                             int(row) & 0xFFFFFFFF, int(t), int(stream),
                                             int(call), int(word)))


def ancestors(w, tau):
    """a_i = min{j : c_j >= tau_i} for the normalised cumulative sums c of weights w."""
    lib = _load()
    w = np.ascontiguousarray(w, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    out = np.zeros(len(tau), dtype=np.int32)
    lib.oracle_ancestors(w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(w),
                         tau.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(tau),
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out


def pf(family, dx, dy, H, theta, y, M, seed, it, row, scheme=SYSTEMATIC, ess_frac=0.5,
       want_grad=True, hint_anc=None, hint_flag=None, replay=False, band=1e-6,
       flag_band=1e-6, want_tape=True, band_rel=0.0):
    """One CRN particle-filter run in FP64 (see oracle.c for the algorithm).

    family: LG_DIAG, SV or LG_OPT; H: (dy, dx) float array or None for identity;
    theta: (D,) float64; y: (T, dy) observations (used as float32).
    Returns a dict with loglik, grad (D,), anc (T, M) uint16, flag (T,) uint8,
    stats (dict of counters) and worst (largest non-tie mismatch distance).
    band_rel widens the tie band to max(band, band_rel * L) with L the accumulated largest
    |log g| since the last resampling (see oracle.c); 0 keeps the fixed band.
    """
    lib = _load()
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    D = int(theta.shape[0])
    y32 = np.ascontiguousarray(np.asarray(y, dtype=np.float32).reshape(-1, dy))
    T = int(y32.shape[0])
    Hd = None if H is None else np.ascontiguousarray(H, dtype=np.float64).reshape(dy, dx)
    ha = None if hint_anc is None else np.ascontiguousarray(hint_anc, dtype=np.uint16).reshape(T, M)
    hf = None if hint_flag is None else np.ascontiguousarray(hint_flag, dtype=np.uint8).reshape(T)
    ll = np.zeros(1, dtype=np.float64)
    grad = np.zeros(D, dtype=np.float64)
    anc = np.zeros((T, M), dtype=np.uint16) if want_tape else None
    flag = np.zeros(T, dtype=np.uint8) if want_tape else None
    stats = np.zeros(len(STAT_NAMES), dtype=np.int64)
    worst = np.zeros(1, dtype=np.float64)
    rc = lib.oracle_pf(int(family), int(dx), int(dy), D, _ptr(Hd), _ptr(theta), _ptr(y32),
                       T, int(M), int(seed), int(it) & 0xFFFFFFFF, int(row) & 0xFFFFFFFF,
                       int(scheme), float(ess_frac), int(bool(want_grad)),
                       _ptr(ha), _ptr(hf), int(bool(replay)), float(band), float(flag_band),
                       float(band_rel), _ptr(ll), _ptr(grad), _ptr(anc), _ptr(flag), _ptr(stats), _ptr(worst))
    if rc != 0:
        raise ValueError("oracle_pf rejected its arguments")
    return {"loglik": float(ll[0]), "grad": grad if want_grad else None, "anc": anc,
            "flag": flag, "stats": dict(zip(STAT_NAMES, (int(v) for v in stats))),
            "worst": float(worst[0])}
