"""FP64 CPU oracle for the BLINK dirty-image path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  The product (the CUDA library
under ``paper_2405_13478_gb300``) never imports it, and this package imports
nothing from the product.

The arithmetic lives in ``blink_oracle.c`` (plain C, FP64); this module only
compiles it with gcc and marshals numpy arrays through ctypes.  Each function
cites the passage of the paper it follows (Sokolowski et al., arXiv 2405.13478):

* :func:`uv`            -- Sec. 5.2.1 step 1: baseline = antenna position
  difference in wavelengths, lambda = c/nu in FP64; w dropped (Sec. 4.3, Eq. 5).
* :func:`cells`         -- Sec. 4.4.1 Eq. 9 (cell size) and Sec. 5.2.1 step 1
  (zero spatial frequency in the centre bin).
* :func:`grid`          -- Sec. 5.2.1 steps 2-3 and Sec. 4.4.2 (natural and
  uniform weighting).
* :func:`image_direct`  -- Sec. 4.3 Eq. 6 written out as the double sum.
* :func:`image_fft`     -- Sec. 5.2.2: inverse 2-D FFT, FFT shift, real part.
* :func:`image_batch`   -- Sec. 5.2.4: many (time, channel) layers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "blink_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

DROPPED = np.iinfo(np.int32).min
C_LIGHT = 299792458.0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no CUDA involved).  Returns the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared",
               "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        F = ctypes.POINTER(ctypes.c_float)
        I32 = ctypes.POINTER(ctypes.c_int32)
        I64 = ctypes.POINTER(ctypes.c_int64)
        lib.orc_version.restype = ctypes.c_int
        lib.orc_n_baselines.restype = ctypes.c_int64
        lib.orc_n_baselines.argtypes = [ctypes.c_int]
        lib.orc_uv.restype = None
        lib.orc_uv.argtypes = [D, ctypes.c_int, ctypes.c_double, D, D]
        lib.orc_cells.restype = ctypes.c_int64
        lib.orc_cells.argtypes = [D, D, ctypes.c_int64, ctypes.c_double, ctypes.c_int, I32, I32]
        lib.orc_grid.restype = ctypes.c_int
        lib.orc_grid.argtypes = [I32, I32, F, ctypes.c_int64, ctypes.c_int, ctypes.c_int, D,
                                 I32, D]
        lib.orc_image_direct.restype = ctypes.c_int
        lib.orc_image_direct.argtypes = [D, ctypes.c_int, D, D]
        lib.orc_image_fft.restype = ctypes.c_int
        lib.orc_image_fft.argtypes = [D, ctypes.c_int, D, D]
        lib.orc_fft1d.restype = ctypes.c_int
        lib.orc_fft1d.argtypes = [D, ctypes.c_int, ctypes.c_int, D]
        lib.orc_grid_c128.restype = ctypes.c_int
        lib.orc_grid_c128.argtypes = [I32, I32, D, ctypes.c_int64, ctypes.c_int, ctypes.c_int, D,
                                      I32, D]
        for fn in ("orc_degrid_direct", "orc_degrid_fft"):
            getattr(lib, fn).restype = ctypes.c_int
            getattr(lib, fn).argtypes = [I32, I32, ctypes.c_int64, ctypes.c_int, ctypes.c_int, D, D]
        lib.orc_gain_grad.restype = None
        lib.orc_gain_grad.argtypes = [ctypes.c_int, D, D, D, D]
        lib.orc_image_batch.restype = ctypes.c_int
        lib.orc_apply_gains.argtypes = [ctypes.c_int, D, F, D]
        lib.orc_apply_gains.restype = None
        lib.orc_image_batch_ex.argtypes = [D, ctypes.c_int, ctypes.c_int, I32, I32, D, D, I64, I64,
                                           F, D, ctypes.c_int64, ctypes.c_int64, D, D, D,
                                           ctypes.c_int, ctypes.c_int]
        lib.orc_image_batch.argtypes = [D, ctypes.c_int, ctypes.c_int, I32, I32, D, D, I64, I64,
                                        F, D, D, ctypes.c_int, ctypes.c_int]
        _lib = lib
        return lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def n_baselines(n_ant: int) -> int:
    return int(_load().orc_n_baselines(n_ant))


def uv(ant_xyz: np.ndarray, freq_hz: float):
    """Baseline (u, v) in wavelengths for all pairs i<j (lexicographic)."""
    xyz = np.ascontiguousarray(ant_xyz, dtype=np.float64)
    nb = n_baselines(xyz.shape[0])
    u = np.empty(nb, np.float64)
    v = np.empty(nb, np.float64)
    _load().orc_uv(_p(xyz, ctypes.c_double), xyz.shape[0], float(freq_hz),
                   _p(u, ctypes.c_double), _p(v, ctypes.c_double))
    return u, v


def cells(u: np.ndarray, v: np.ndarray, delta_u: float, n_px: int):
    """Signed cell offsets (k_u, k_v); DROPPED marks baselines not gridded."""
    u = np.ascontiguousarray(u, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    ku = np.empty(u.size, np.int32)
    kv = np.empty(u.size, np.int32)
    _load().orc_cells(_p(u, ctypes.c_double), _p(v, ctypes.c_double), u.size, float(delta_u),
                      int(n_px), _p(ku, ctypes.c_int32), _p(kv, ctypes.c_int32))
    return ku, kv


def grid(ku, kv, vis, n_px: int, weighting: int):
    """Full complex128 grid [N][N] (centre bin = DC), counts [N][N], summed weight."""
    ku = np.ascontiguousarray(ku, np.int32)
    kv = np.ascontiguousarray(kv, np.int32)
    vis = np.ascontiguousarray(vis, np.complex64)
    g = np.empty((n_px, n_px), np.complex128)
    cnt = np.empty((n_px, n_px), np.int32)
    ws = np.zeros(1, np.float64)
    st = _load().orc_grid(_p(ku, ctypes.c_int32), _p(kv, ctypes.c_int32),
                          _p(vis.view(np.float32), ctypes.c_float), ku.size, int(n_px),
                          int(weighting), _p(g.view(np.float64), ctypes.c_double),
                          _p(cnt, ctypes.c_int32), _p(ws, ctypes.c_double))
    if st != 0:
        raise ValueError(f"orc_grid rejected its arguments ({st})")
    return g, cnt, float(ws[0])


def image_direct(g: np.ndarray):
    """Dirty image by the double sum over occupied cells; returns (image, max|Im|)."""
    g = np.ascontiguousarray(g, np.complex128)
    n = g.shape[0]
    img = np.empty((n, n), np.float64)
    mi = np.zeros(1, np.float64)
    if _load().orc_image_direct(_p(g.view(np.float64), ctypes.c_double), n,
                                _p(img, ctypes.c_double), _p(mi, ctypes.c_double)) != 0:
        raise ValueError("orc_image_direct rejected its arguments")
    return img, float(mi[0])


def image_fft(g: np.ndarray):
    """Dirty image by FP64 FFT with shifts; returns (image, max|Im|)."""
    g = np.ascontiguousarray(g, np.complex128)
    n = g.shape[0]
    img = np.empty((n, n), np.float64)
    mi = np.zeros(1, np.float64)
    if _load().orc_image_fft(_p(g.view(np.float64), ctypes.c_double), n,
                             _p(img, ctypes.c_double), _p(mi, ctypes.c_double)) != 0:
        raise ValueError("orc_image_fft rejected its arguments")
    return img, float(mi[0])


def fft1d(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised 1-D DFT with exp(sign * 2 pi i j k / n)."""
    x = np.ascontiguousarray(x, np.complex128)
    out = np.empty_like(x)
    if _load().orc_fft1d(_p(x.view(np.float64), ctypes.c_double), x.size, int(sign),
                         _p(out.view(np.float64), ctypes.c_double)) != 0:
        raise ValueError("orc_fft1d rejected its arguments")
    return out


def apply_gains(n_ant: int, gains, vis):
    """V'_ij = g_i conj(g_j) V_ij for the pairs (i < j), in complex128."""
    g = np.ascontiguousarray(gains, np.complex128)
    v = np.ascontiguousarray(vis, np.complex64).reshape(-1)
    out = np.empty(v.size, np.complex128)
    _load().orc_apply_gains(int(n_ant), _p(g.view(np.float64), ctypes.c_double),
                            _p(v.view(np.float32), ctypes.c_float),
                            _p(out.view(np.float64), ctypes.c_double))
    return out


def image_batch(ant_xyz, layers, vis, mode: str = "fft", n_threads: int = 0, gains=None,
                gain_stride: int = 0, ref=None, gain_period: int = 0):
    """Whole path over many layers.

    ``layers`` is a sequence of dicts with keys n_px, weighting, freq_hz,
    delta_u, vis_offset (complex elements into ``vis``).  Optional: ``gains``
    (complex, layer l uses the row starting at r * gain_stride, r = l mod
    gain_period, or r = l when gain_period is 0) applied to the visibilities, and ``ref`` (flat, packed like the returned images)
    subtracted from the images.  Returns (list of float64 images, wsum array).
    """
    xyz = np.ascontiguousarray(ant_xyz, np.float64)
    vis = np.ascontiguousarray(vis, np.complex64).reshape(-1)
    L = len(layers)
    npx = np.array([l["n_px"] for l in layers], np.int32)
    wt = np.array([l["weighting"] for l in layers], np.int32)
    fr = np.array([l["freq_hz"] for l in layers], np.float64)
    du = np.array([l["delta_u"] for l in layers], np.float64)
    vo = np.array([l["vis_offset"] for l in layers], np.int64)
    sizes = npx.astype(np.int64) ** 2
    oo = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    out = np.empty(int(sizes.sum()), np.float64)
    ws = np.zeros(L, np.float64)
    if gains is None and ref is None:
        st = _load().orc_image_batch(
            _p(xyz, ctypes.c_double), xyz.shape[0], L, _p(npx, ctypes.c_int32),
            _p(wt, ctypes.c_int32), _p(fr, ctypes.c_double), _p(du, ctypes.c_double),
            _p(vo, ctypes.c_int64), _p(oo, ctypes.c_int64),
            _p(vis.view(np.float32), ctypes.c_float), _p(out, ctypes.c_double),
            _p(ws, ctypes.c_double), 1 if mode == "direct" else 0, int(n_threads))
    else:
        g = None if gains is None else np.ascontiguousarray(gains, np.complex128).reshape(-1)
        r = None if ref is None else np.ascontiguousarray(ref, np.float64).reshape(-1)
        if r is not None and r.size < out.size:
            raise ValueError("reference images smaller than the output")
        rows = min(L, int(gain_period)) if gain_period > 0 else L
        if g is not None and g.size < (rows - 1) * int(gain_stride) + xyz.shape[0]:
            raise ValueError("gain rows smaller than the layers need")
        st = _load().orc_image_batch_ex(
            _p(xyz, ctypes.c_double), xyz.shape[0], L, _p(npx, ctypes.c_int32),
            _p(wt, ctypes.c_int32), _p(fr, ctypes.c_double), _p(du, ctypes.c_double),
            _p(vo, ctypes.c_int64), _p(oo, ctypes.c_int64),
            _p(vis.view(np.float32), ctypes.c_float),
            None if g is None else _p(g.view(np.float64), ctypes.c_double), int(gain_stride),
            int(gain_period), None if r is None else _p(r, ctypes.c_double), _p(out, ctypes.c_double),
            _p(ws, ctypes.c_double), 1 if mode == "direct" else 0, int(n_threads))
    if st != 0:
        raise ValueError(f"orc_image_batch failed ({st})")
    imgs = [out[oo[i]:oo[i] + sizes[i]].reshape(npx[i], npx[i]) for i in range(L)]
    return imgs, ws


def image(ant_xyz, freq_hz, delta_u, n_px, weighting, vis, mode: str = "fft"):
    """Convenience: one layer through the whole path; returns (image, wsum, max|Im|)."""
    u, v = uv(ant_xyz, freq_hz)
    ku, kv = cells(u, v, delta_u, n_px)
    g, _, ws = grid(ku, kv, vis, n_px, weighting)
    img, mi = image_direct(g) if mode == "direct" else image_fft(g)
    return img, ws, mi


def grid_c128(ku, kv, vis, n_px: int, weighting: int):
    """grid() with complex128 visibilities (finite-difference pins)."""
    ku = np.ascontiguousarray(ku, np.int32)
    kv = np.ascontiguousarray(kv, np.int32)
    vis = np.ascontiguousarray(vis, np.complex128)
    g = np.empty((n_px, n_px), np.complex128)
    cnt = np.empty((n_px, n_px), np.int32)
    ws = np.zeros(1, np.float64)
    st = _load().orc_grid_c128(_p(ku, ctypes.c_int32), _p(kv, ctypes.c_int32),
                               _p(vis.view(np.float64), ctypes.c_double), ku.size, int(n_px),
                               int(weighting), _p(g.view(np.float64), ctypes.c_double),
                               _p(cnt, ctypes.c_int32), _p(ws, ctypes.c_double))
    if st != 0:
        raise ValueError("orc_grid_c128 rejected its arguments")
    return g, cnt, float(ws[0])


def degrid(ku, kv, resid, weighting: int, mode: str = "fft"):
    """Adjoint: gradient w.r.t. the visibilities of a loss whose image
    gradient is ``resid``: gamma_b = 2 w_b H[k_b] (dL/dRe + i dL/dIm)."""
    ku = np.ascontiguousarray(ku, np.int32)
    kv = np.ascontiguousarray(kv, np.int32)
    r = np.ascontiguousarray(resid, np.float64)
    gam = np.empty(ku.size, np.complex128)
    fn = _load().orc_degrid_direct if mode == "direct" else _load().orc_degrid_fft
    if fn(_p(ku, ctypes.c_int32), _p(kv, ctypes.c_int32), ku.size, r.shape[0], int(weighting),
          _p(r, ctypes.c_double), _p(gam.view(np.float64), ctypes.c_double)) != 0:
        raise ValueError("orc_degrid rejected its arguments")
    return gam


def gain_grad(n_ant: int, gamma_v, gains, model, out=None):
    """Chain rule from visibility gradients to per-antenna gain gradients
    (V_ij = g_i conj(g_j) M_ij); accumulates into ``out``."""
    gv = np.ascontiguousarray(gamma_v, np.complex128)
    g = np.ascontiguousarray(gains, np.complex128)
    m = np.ascontiguousarray(model, np.complex128)
    out = np.zeros(n_ant, np.complex128) if out is None else out
    _load().orc_gain_grad(int(n_ant), _p(gv.view(np.float64), ctypes.c_double),
                          _p(g.view(np.float64), ctypes.c_double),
                          _p(m.view(np.float64), ctypes.c_double),
                          _p(out.view(np.float64), ctypes.c_double))
    return out
