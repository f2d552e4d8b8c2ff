"""Thin ctypes binding of the C ABI in ``include/blink.h``.

Argument marshalling only: PyTorch supplies device memory and the current
CUDA stream; every step of the imaging path runs in the library's kernels.
There is no CPU fallback -- if ``libblink.so`` is missing or no GPU is present
the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Sequence

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libblink.so")

OK, ERR_INVALID, ERR_UNSUPPORTED, ERR_CUDA, ERR_TIMEOUT, ERR_WORKSPACE = 0, -1, -2, -3, -4, -5
NATURAL, UNIFORM = 0, 1
NORMALIZE = 0x1
TRANSFORM_FFT, TRANSFORM_BF16, TRANSFORM_BF16X3, TRANSFORM_FP16, TRANSFORM_FP16X3 = (
    0x00, 0x10, 0x20, 0x30, 0x40)
DROPPED = -(2 ** 31)

# Symbols declared in include/blink.h (checked by the CPU test suite).
EXPORTS = (
    "blink_abi_version", "blink_supported_sizes", "blink_ctx_create", "blink_ctx_destroy",
    "blink_last_error", "blink_cells", "blink_grid", "blink_image_batch", "blink_plan_create",
    "blink_plan_image", "blink_plan_destroy", "blink_plan_layer_info",
    "blink_image_batch_noalloc", "blink_image_batch_host", "blink_degrid", "blink_plan_degrid",
    "blink_apply_gains", "blink_gain_grad", "blink_plan_check", "blink_plan_autotune",
    "blink_plan_tuning", "blink_plan_set_tuning", "blink_plan_capture", "blink_plan_replay",
    "blink_plan_image_ex", "blink_ctx_set_wait_limit", "blink_probe_fma_peak",
    "blink_plan_degrid_scaled", "blink_plan_adjoint_bytes", "blink_plan_degrid_adjoint",
)


class BlinkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"blink status {status}: {msg}")
        self.status = status


class Layer(ctypes.Structure):
    _fields_ = [("n_px", ctypes.c_int32), ("weighting", ctypes.c_int32),
                ("freq_hz", ctypes.c_double), ("delta_u", ctypes.c_double),
                ("vis_offset", ctypes.c_int64), ("out_offset", ctypes.c_int64)]


class Epilogue(ctypes.Structure):
    """blink_epilogue: gains applied at gridding, reference image subtracted,
    per-layer sums of squares of the output."""
    _fields_ = [("d_gains", ctypes.c_void_p), ("gain_stride", ctypes.c_int64),
                ("gain_period", ctypes.c_int64), ("d_ref", ctypes.c_void_p),
                ("d_sqnorm", ctypes.c_void_p), ("d_adjoint", ctypes.c_void_p)]


def _epilogue(gains, gain_stride, ref, gain_period=0, sqnorm=None, adjoint=None):
    """A blink_epilogue for the optional tensors (None when all are absent)."""
    if gains is None and ref is None and sqnorm is None and adjoint is None:
        return None
    _check_dev(gains, ref, sqnorm, adjoint)
    if gains is not None and gains.dtype != _complex64():
        raise ValueError("gains must be complex64")
    if ref is not None and ref.dtype != _float32():
        raise ValueError("reference images must be float32")
    if sqnorm is not None and sqnorm.dtype != _float64():
        raise ValueError("sqnorm must be float64")
    return Epilogue(0 if gains is None else gains.data_ptr(), int(gain_stride), int(gain_period),
                    0 if ref is None else ref.data_ptr(), 0 if sqnorm is None else sqnorm.data_ptr(),
                    0 if adjoint is None else adjoint.data_ptr())


def _complex64():
    import torch
    return torch.complex64


def _float64():
    import torch
    return torch.float64


def _float32():
    import torch
    return torch.float32


_lib = None


def lib(path: str = LIB_PATH):
    """Load libblink.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"BLINK CUDA library not built: {path} is missing "
                           "(run paper_2405_13478_gb300/build.py)")
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    L.blink_abi_version.restype = I
    L.blink_supported_sizes.restype = I
    L.blink_supported_sizes.argtypes = [ctypes.POINTER(ctypes.c_int32), I]
    L.blink_ctx_create.restype = I
    L.blink_ctx_create.argtypes = [ctypes.POINTER(P), I]
    L.blink_ctx_destroy.restype = None
    L.blink_ctx_destroy.argtypes = [P]
    L.blink_last_error.restype = ctypes.c_char_p
    L.blink_last_error.argtypes = [P]
    LP = ctypes.POINTER(Layer)
    L.blink_cells.restype = I
    L.blink_cells.argtypes = [P, P, I, LP, I, P, P]
    L.blink_grid.restype = I
    L.blink_grid.argtypes = [P, P, I, LP, I, P, P, P, P]
    L.blink_image_batch.restype = I
    L.blink_image_batch.argtypes = [P, P, I, LP, I, P, P, P, ctypes.c_uint32, P]
    L.blink_plan_create.restype = I
    L.blink_plan_create.argtypes = [P, P, I, LP, I, ctypes.POINTER(P), P]
    L.blink_plan_image.restype = I
    L.blink_plan_image.argtypes = [P, P, P, P, ctypes.c_uint32, P]
    L.blink_ctx_set_wait_limit.restype = I
    L.blink_ctx_set_wait_limit.argtypes = [P, ctypes.c_int64]
    L.blink_plan_image_ex.restype = I
    L.blink_plan_image_ex.argtypes = [P, P, P, P, ctypes.c_uint32, ctypes.POINTER(Epilogue), P]
    L.blink_plan_destroy.restype = None
    L.blink_plan_destroy.argtypes = [P]
    L.blink_image_batch_host.restype = I
    L.blink_image_batch_host.argtypes = [P, P, I, LP, I, P, P, P, ctypes.c_uint32, P]
    L.blink_degrid.restype = I
    L.blink_degrid.argtypes = [P, P, I, LP, I, P, P, ctypes.c_uint32, P]
    L.blink_plan_degrid.restype = I
    L.blink_plan_degrid.argtypes = [P, P, P, ctypes.c_uint32, P]
    L.blink_plan_degrid_scaled.restype = I
    L.blink_plan_degrid_scaled.argtypes = [P, P, P, P, ctypes.c_uint32, P]
    L.blink_plan_adjoint_bytes.restype = I
    L.blink_plan_adjoint_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    L.blink_plan_degrid_adjoint.restype = I
    L.blink_plan_degrid_adjoint.argtypes = [P, P, P, P, ctypes.c_uint32, P]
    L.blink_apply_gains.restype = I
    L.blink_apply_gains.argtypes = [P, I, LP, I, P, P, P, P]
    L.blink_gain_grad.restype = I
    L.blink_gain_grad.argtypes = [P, I, LP, I, P, P, P, P, P]
    L.blink_plan_autotune.restype = I
    L.blink_plan_autotune.argtypes = [P, P, P, P]
    L.blink_plan_tuning.restype = I
    L.blink_plan_tuning.argtypes = [P, I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int64)]
    L.blink_plan_set_tuning.restype = I
    L.blink_plan_set_tuning.argtypes = [P, I, I, ctypes.c_int64]
    L.blink_plan_capture.restype = I
    L.blink_plan_capture.argtypes = [P, P, P, P, ctypes.c_uint32, ctypes.POINTER(Epilogue), P]
    L.blink_plan_replay.restype = I
    L.blink_plan_replay.argtypes = [P, P]
    L.blink_plan_check.restype = I
    L.blink_plan_check.argtypes = [P, P]
    L.blink_plan_layer_info.restype = I
    L.blink_plan_layer_info.argtypes = [P, I, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_int64)]
    L.blink_probe_fma_peak.restype = I
    L.blink_probe_fma_peak.argtypes = [I, I, ctypes.POINTER(ctypes.c_double)]
    _lib = L
    return L


def fma_peak_tflops(device: int, bits: int) -> float:
    """Measured FMA rate (TFLOP/s, 2 flops per FMA) of the CUDA cores of
    `device` in FP32 (bits=32) or FP64 (bits=64)."""
    out = ctypes.c_double(0.0)
    st = lib().blink_probe_fma_peak(int(device), int(bits), ctypes.byref(out))
    if st != OK:
        raise BlinkError(st, f"FMA probe ({bits}-bit) failed")
    return out.value


def supported_sizes():
    L = lib()
    n = L.blink_supported_sizes(None, 0)
    buf = (ctypes.c_int32 * n)()
    L.blink_supported_sizes(buf, n)
    return list(buf)


LAYER_DTYPE = None


def layer_dtype():
    """numpy structured dtype with the memory layout of blink_layer."""
    global LAYER_DTYPE
    if LAYER_DTYPE is None:
        import numpy as np
        LAYER_DTYPE = np.dtype([("n_px", "<i4"), ("weighting", "<i4"), ("freq_hz", "<f8"),
                                ("delta_u", "<f8"), ("vis_offset", "<i8"), ("out_offset", "<i8")])
        assert LAYER_DTYPE.itemsize == ctypes.sizeof(Layer)
    return LAYER_DTYPE


def layer_array(n_px, weighting, freq_hz, delta_u, vis_offset, out_offset):
    """Vectorised blink_layer array from equal-length array-likes."""
    import numpy as np
    n = len(np.atleast_1d(vis_offset))
    arr = np.zeros(n, dtype=layer_dtype())
    arr["n_px"] = n_px
    arr["weighting"] = weighting
    arr["freq_hz"] = freq_hz
    arr["delta_u"] = delta_u
    arr["vis_offset"] = vis_offset
    arr["out_offset"] = out_offset
    return arr


def make_layers(layers):
    """blink_layer array for the C ABI from a list of dicts or a layer_array()."""
    import numpy as np
    if isinstance(layers, np.ndarray):
        if layers.dtype != layer_dtype() or not layers.flags.c_contiguous:
            raise ValueError("layer arrays must come from layer_array()")
        return layers.ctypes.data_as(ctypes.POINTER(Layer))
    arr = (Layer * max(1, len(layers)))()
    for k, d in enumerate(layers):
        arr[k] = Layer(int(d["n_px"]), int(d["weighting"]), float(d["freq_hz"]),
                       float(d["delta_u"]), int(d["vis_offset"]), int(d.get("out_offset", 0)))
    return arr


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream=None):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check_dev(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("tensors passed to the BLINK library must be CUDA tensors")
        if t is not None and not t.is_contiguous():
            raise ValueError("tensors passed to the BLINK library must be contiguous")


class Context:
    """A library context on one CUDA device (owns the device workspace pool)."""

    def __init__(self, device: int = 0):
        self._lib = lib()
        h = ctypes.c_void_p()
        st = self._lib.blink_ctx_create(ctypes.byref(h), int(device))
        if st != OK:
            raise BlinkError(st, f"blink_ctx_create(device={device}) failed")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            self._lib.blink_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, st):
        if st != OK:
            raise BlinkError(st, self._lib.blink_last_error(self.handle).decode())

    def set_wait_limit(self, limit_ns):
        """Bounded-wait limit of the tensor-core kernels (ns; < 0 = default 1 s)."""
        self._raise(self._lib.blink_ctx_set_wait_limit(self.handle, int(limit_ns)))

    def cells(self, ant_xyz, layers, cells_out, stream=None):
        """Cell indices: int32 [n_layers][B][2]."""
        _check_dev(ant_xyz, cells_out)
        arr = make_layers(layers)
        self._raise(self._lib.blink_cells(self.handle, _ptr(ant_xyz), ant_xyz.shape[0], arr,
                                          len(layers), _ptr(cells_out), _stream(stream)))

    def grid(self, ant_xyz, layers, vis, grid_out, wsum_out=None, stream=None):
        """Gridded, weighted visibilities: complex64 Hermitian-complete grids (DC at N/2, N/2)."""
        _check_dev(ant_xyz, vis, grid_out, wsum_out)
        arr = make_layers(layers)
        self._raise(self._lib.blink_grid(self.handle, _ptr(ant_xyz), ant_xyz.shape[0], arr,
                                         len(layers), _ptr(vis), _ptr(grid_out), _ptr(wsum_out),
                                         _stream(stream)))

    def image_batch(self, ant_xyz, layers, vis, images_out, wsum_out=None, flags=0, stream=None):
        """Float32 dirty images (the whole path)."""
        _check_dev(ant_xyz, vis, images_out, wsum_out)
        arr = make_layers(layers)
        self._raise(self._lib.blink_image_batch(self.handle, _ptr(ant_xyz), ant_xyz.shape[0], arr,
                                                len(layers), _ptr(vis), _ptr(images_out),
                                                _ptr(wsum_out), int(flags), _stream(stream)))

    def image_batch_host(self, ant_xyz, layers, vis, images_out, wsum_out=None, flags=0,
                         stream=None):
        """The whole path with host-resident inputs and outputs (numpy arrays or CPU
        tensors; pinned memory gives full copy bandwidth)."""
        import numpy as np

        def hp(x):
            if x is None:
                return ctypes.c_void_p(0)
            if isinstance(x, np.ndarray):
                if not x.flags.c_contiguous:
                    raise ValueError("host arrays must be contiguous")
                return ctypes.c_void_p(x.ctypes.data)
            if x.is_cuda or not x.is_contiguous():
                raise ValueError("host tensors must be contiguous CPU tensors")
            return ctypes.c_void_p(x.data_ptr())

        arr = make_layers(layers)
        xyz = np.ascontiguousarray(ant_xyz, dtype=np.float64)
        self._raise(self._lib.blink_image_batch_host(
            self.handle, ctypes.c_void_p(xyz.ctypes.data), xyz.shape[0], arr, len(layers), hp(vis),
            hp(images_out), hp(wsum_out), int(flags), _stream(stream)))

    def degrid(self, ant_xyz, layers, dimage, dvis_out, flags=0, stream=None):
        """Adjoint: dL/dV (complex64 at vis_offset) from dL/dimage."""
        _check_dev(ant_xyz, dimage, dvis_out)
        arr = make_layers(layers)
        self._raise(self._lib.blink_degrid(self.handle, _ptr(ant_xyz), ant_xyz.shape[0], arr,
                                           len(layers), _ptr(dimage), _ptr(dvis_out), int(flags),
                                           _stream(stream)))

    def apply_gains(self, n_ant, layers, model, gains, vis_out, stream=None):
        """vis = g_i conj(g_j) model for every baseline of every layer."""
        _check_dev(model, gains, vis_out)
        arr = make_layers(layers)
        self._raise(self._lib.blink_apply_gains(self.handle, int(n_ant), arr, len(layers),
                                                _ptr(model), _ptr(gains), _ptr(vis_out),
                                                _stream(stream)))

    def gain_grad(self, n_ant, layers, dvis, model, gains, dgains_out, stream=None):
        """Per-antenna gain gradient from visibility gradients (summed over layers)."""
        _check_dev(dvis, model, gains, dgains_out)
        arr = make_layers(layers)
        self._raise(self._lib.blink_gain_grad(self.handle, int(n_ant), arr, len(layers),
                                              _ptr(dvis), _ptr(model), _ptr(gains),
                                              _ptr(dgains_out), _stream(stream)))

    def plan(self, ant_xyz, layers, stream=None) -> "Plan":
        return Plan(self, ant_xyz, layers, stream)


class Plan:
    """Tables built once (uv, cells, weights); image() launches gridding + transform only."""

    def __init__(self, ctx: Context, ant_xyz, layers, stream=None):
        _check_dev(ant_xyz)
        self.ctx = ctx
        self.n_layers = len(layers)
        arr = make_layers(layers)
        h = ctypes.c_void_p()
        ctx._raise(ctx._lib.blink_plan_create(ctx.handle, _ptr(ant_xyz), ant_xyz.shape[0], arr,
                                              len(layers), ctypes.byref(h), _stream(stream)))
        self.handle = h

    def image(self, vis, images_out, wsum_out=None, flags=0, stream=None, gains=None,
              gain_stride=0, ref=None, gain_period=0, sqnorm=None, adjoint=None):
        """Dirty images of the plan's layers.  Optional fused epilogue: ``gains``
        (complex64, layer l uses the row at r * gain_stride, r = l mod
        gain_period or l) applied to the visibilities, ``ref`` (float32, laid
        out like ``images_out``) subtracted from the images, ``sqnorm``
        (float64 [layers]) receiving each layer's sum of squares of the
        stored output, ``adjoint`` (float32, adjoint_bytes() / 4 elements)
        receiving the adjoint's column transforms of the stored output for
        degrid_adjoint()."""
        _check_dev(vis, images_out, wsum_out)
        epi = _epilogue(gains, gain_stride, ref, gain_period, sqnorm, adjoint)
        if epi is None:
            st = self.ctx._lib.blink_plan_image(self.handle, _ptr(vis), _ptr(images_out),
                                                _ptr(wsum_out), int(flags), _stream(stream))
        else:
            st = self.ctx._lib.blink_plan_image_ex(self.handle, _ptr(vis), _ptr(images_out),
                                                   _ptr(wsum_out), int(flags), ctypes.byref(epi),
                                                   _stream(stream))
        self.ctx._raise(st)

    def degrid(self, dimage, dvis_out, flags=0, stream=None, layer_scale=None):
        """Visibility gradient of the image gradient ``dimage``; with
        ``layer_scale`` (float32 [layers]) layer l's result is multiplied by
        layer_scale[l]."""
        _check_dev(dimage, dvis_out, layer_scale)
        if layer_scale is None:
            st = self.ctx._lib.blink_plan_degrid(self.handle, _ptr(dimage), _ptr(dvis_out), int(flags),
                                                 _stream(stream))
        else:
            if layer_scale.dtype != _float32():
                raise ValueError("layer_scale must be float32")
            st = self.ctx._lib.blink_plan_degrid_scaled(self.handle, _ptr(dimage), _ptr(layer_scale),
                                                        _ptr(dvis_out), int(flags), _stream(stream))
        self.ctx._raise(st)

    def adjoint_bytes(self) -> int:
        n = ctypes.c_int64()
        self.ctx._raise(self.ctx._lib.blink_plan_adjoint_bytes(self.handle, ctypes.byref(n)))
        return int(n.value)

    def degrid_adjoint(self, adjoint, dvis_out, flags=0, stream=None, layer_scale=None):
        """degrid(images, ...) for the images whose column transforms an
        image(..., adjoint=) call kept in ``adjoint``."""
        _check_dev(adjoint, dvis_out, layer_scale)
        if layer_scale is not None and layer_scale.dtype != _float32():
            raise ValueError("layer_scale must be float32")
        self.ctx._raise(self.ctx._lib.blink_plan_degrid_adjoint(self.handle, _ptr(adjoint), _ptr(layer_scale),
                                                                _ptr(dvis_out), int(flags), _stream(stream)))

    def autotune(self, vis, images_out, stream=None):
        """Time the candidate kernel configurations per image size, keep the fastest."""
        _check_dev(vis, images_out)
        self.ctx._raise(self.ctx._lib.blink_plan_autotune(self.handle, _ptr(vis), _ptr(images_out),
                                                          _stream(stream)))

    def tuning(self):
        """[(n_px, path, wave_bytes)] chosen per size group."""
        out, g = [], 0
        while True:
            n, pth, wb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
            if self.ctx._lib.blink_plan_tuning(self.handle, g, ctypes.byref(n), ctypes.byref(pth),
                                               ctypes.byref(wb)) != OK:
                return out
            out.append((n.value, pth.value, wb.value))
            g += 1

    def set_tuning(self, group, path, wave_bytes=0):
        """Force size group `group` onto kernel path 0-4 (see blink_plan_set_tuning)."""
        self.ctx._raise(self.ctx._lib.blink_plan_set_tuning(self.handle, int(group), int(path),
                                                            int(wave_bytes)))

    def capture(self, vis, images_out, wsum_out=None, flags=0, stream=None, gains=None,
                gain_stride=0, ref=None, gain_period=0, sqnorm=None, adjoint=None):
        """Record the batch's launches (with the optional epilogue) into a CUDA
        graph bound to these buffers."""
        _check_dev(vis, images_out, wsum_out)
        epi = _epilogue(gains, gain_stride, ref, gain_period, sqnorm, adjoint)
        self.ctx._raise(self.ctx._lib.blink_plan_capture(
            self.handle, _ptr(vis), _ptr(images_out), _ptr(wsum_out), int(flags),
            None if epi is None else ctypes.byref(epi), _stream(stream)))

    def replay(self, stream=None):
        """Launch the captured graph (the whole batch, every image size)."""
        self.ctx._raise(self.ctx._lib.blink_plan_replay(self.handle, _stream(stream)))

    def check(self, stream=None):
        """Synchronise and raise if a bounded device-side wait timed out."""
        self.ctx._raise(self.ctx._lib.blink_plan_check(self.handle, _stream(stream)))

    def layer_info(self, layer: int):
        w = ctypes.c_float()
        n = ctypes.c_int64()
        self.ctx._raise(self.ctx._lib.blink_plan_layer_info(self.handle, int(layer),
                                                            ctypes.byref(w), ctypes.byref(n)))
        return float(w.value), int(n.value)

    def close(self):
        if getattr(self, "handle", None):
            self.ctx._lib.blink_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def layer_out_offsets(layers: Iterable[dict]):
    """Packs images contiguously: returns (layers with out_offset, total floats)."""
    out, off = [], 0
    for d in layers:
        d = dict(d)
        d["out_offset"] = off
        off += int(d["n_px"]) ** 2
        out.append(d)
    return out, off
