"""Thin ctypes binding of libdctgb (include/dctgb.h) with the same entry-point
names.  It only marshals arguments: torch tensors become device pointers,
sizes and pitches; every step of the codec runs in the library's kernels.
There is no CPU fallback: without the library or a CUDA device the calls
raise.
"""
import ctypes
import math
import os

import numpy as np
import torch

from . import build as _build

DCT_OK = 0
STATUS_NAMES = {0: "DCT_OK", 1: "DCT_ERR_INVALID_ARG", 2: "DCT_ERR_UNSUPPORTED", 3: "DCT_ERR_ALLOC",
                4: "DCT_ERR_CUDA", 5: "DCT_ERR_TIMEOUT", 6: "DCT_ERR_STATE"}
DCT_LAYOUT_GRAY8 = 0
DCT_LAYOUT_YUV420 = 1
DCT_OP_COMPRESS = 1
DCT_OP_RECONSTRUCT = 2
DCT_OP_SSE = 4
DCT_OP_TWO_PASS = 8

# statistics words written by dct_compress(stats=...) per plane
STATS_WORDS = 80
STATS_LAYOUT = dict(band=(0, 64), sum=64, sum2=65, min=66, max=67, abs_dx=68, abs_dy=69,
                    dx2=70, dy2=71, low_ac=(72, 76), blocks=76, samples=77)


class DctError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class dct_plane(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("pitch", ctypes.c_int32)]


class dct_plan_desc(ctypes.Structure):
    _fields_ = [("max_width", ctypes.c_int32), ("max_height", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class dct_spec_info(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32), ("N", ctypes.c_int32), ("R", ctypes.c_int32),
                ("quant_shift", ctypes.c_int32), ("dequant_clamp", ctypes.c_int32), ("psnr_max", ctypes.c_int32),
                ("sigma_odd_upper", ctypes.c_uint32), ("sigma_odd_lower", ctypes.c_uint32),
                ("sigma_even", ctypes.c_uint32), ("stats_words", ctypes.c_int32)]


class dct_batch_item(ctypes.Structure):
    _fields_ = [("src", dct_plane), ("coeffs", ctypes.c_void_p), ("recon", ctypes.c_void_p),
                ("recon_pitch", ctypes.c_int32), ("quality", ctypes.c_int32), ("chroma", ctypes.c_int32),
                ("qtab_host", ctypes.POINTER(ctypes.c_uint16))]


class dct_launch_shape(ctypes.Structure):
    _fields_ = [("threads_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("tile_blocks", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_P = ctypes.c_void_p
_U16P = ctypes.POINTER(ctypes.c_uint16)
_SIGNATURES = {
    "dct_spec_query": (ctypes.c_int, [ctypes.POINTER(dct_spec_info)]),
    "dct_tables": (ctypes.c_int, [ctypes.c_int, _U16P, ctypes.c_int, ctypes.c_int, _U16P,
                                  ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int32)]),
    "dct_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(dct_plan_desc), _P]),
    "dct_plan_destroy": (ctypes.c_int, [_P]),
    "dct_compress": (ctypes.c_int, [_P, ctypes.POINTER(dct_plane), ctypes.c_int, ctypes.c_int, _U16P, ctypes.c_int,
                                    _P, _P, _P]),
    "dct_reconstruct": (ctypes.c_int, [_P, _P, ctypes.POINTER(dct_plane), ctypes.c_int, ctypes.c_int, _U16P,
                                       ctypes.c_int, ctypes.POINTER(dct_plane), _P, _P]),
    "dct_codec_fused": (ctypes.c_int, [_P, ctypes.POINTER(dct_plane), ctypes.c_int, ctypes.c_int, _U16P,
                                       ctypes.c_int, _P, ctypes.POINTER(dct_plane), _P, _P]),
    "dct_psnr": (ctypes.c_int, [_P, ctypes.POINTER(dct_plane), ctypes.POINTER(dct_plane), ctypes.c_int, _P,
                                ctypes.POINTER(ctypes.c_double), ctypes.c_double, _P]),
    "dct_psnr_from_sse": (ctypes.c_double, [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double]),
    "dct_batch_prepare": (ctypes.c_int, [_P, ctypes.POINTER(dct_batch_item), ctypes.c_int, ctypes.c_uint32, _P,
                                         ctypes.POINTER(dct_launch_shape), _P]),
    "dct_batch_launch": (ctypes.c_int, [_P, _P]),
    "dct_autotune": (ctypes.c_int, [_P, ctypes.POINTER(dct_launch_shape), ctypes.POINTER(ctypes.c_float), _P]),
    "dct_last_error": (ctypes.c_char_p, []),
}

_LIB = None


def load(build_if_needed=True):
    """Loads (building first if needed) the in-tree libdctgb.so."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_needed and not _build.up_to_date():
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libdctgb.so is missing; run paper_1306_1373_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def declared_symbols():
    return list(_SIGNATURES)


def _check(status):
    if status != DCT_OK:
        raise DctError(status, load().dct_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _require_cuda(*tensors):
    for t in tensors:
        if t is not None and not t.is_cuda:
            raise ValueError("tensors must live on a CUDA device")


def as_plane(t):
    """A 2-D uint8 CUDA tensor (rows may be padded: stride(0) = pitch) -> dct_plane."""
    if t.dtype != torch.uint8 or t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("planes are 2-D uint8 tensors with unit column stride")
    _require_cuda(t)
    return dct_plane(t.data_ptr(), t.shape[1], t.shape[0], t.stride(0))


def _planes(ts):
    arr = (dct_plane * len(ts))(*[as_plane(t) for t in ts])
    return arr


def _qtab(qtab):
    if qtab is None:
        return None, 0
    a = np.ascontiguousarray(np.asarray(qtab, dtype=np.uint16).reshape(-1))
    return a, a.size


def _u16p(a):
    return None if a is None else a.ctypes.data_as(_U16P)


def n_blocks(height, width):
    return ((height + 7) // 8) * ((width + 7) // 8)


def coeff_count(shapes):
    """int16 coefficients for planes of the given (height, width) shapes."""
    return sum(n_blocks(h, w) * 64 for h, w in shapes)


def dct_spec_query():
    info = dct_spec_info()
    _check(load().dct_spec_query(ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in dct_spec_info._fields_}


def dct_tables(quality, qtab=None, chroma=False):
    """(Q, M, W) host tables for one plane, as int64 (8, 8) numpy arrays."""
    q = np.zeros(64, dtype=np.uint16)
    m = np.zeros(64, dtype=np.uint32)
    w = np.zeros(64, dtype=np.int32)
    qa, n = _qtab(qtab)
    _check(load().dct_tables(int(quality), _u16p(qa), n, int(bool(chroma)), q.ctypes.data_as(_U16P),
                             m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                             w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return (q.astype(np.int64).reshape(8, 8), m.astype(np.int64).reshape(8, 8), w.astype(np.int64).reshape(8, 8))


def dct_psnr_from_sse(sse, n_samples, max_value=0.0):
    return load().dct_psnr_from_sse(int(sse), int(n_samples), float(max_value))


class Plan:
    """Owns a dct_plan_t; use as a context manager or call close()."""

    def __init__(self, max_width, max_height, layout=DCT_LAYOUT_GRAY8, max_batch=0, stream=None):
        self.handle = ctypes.c_void_p()
        desc = dct_plan_desc(int(max_width), int(max_height), int(layout), int(max_batch), 0)
        _check(load().dct_plan_create(ctypes.byref(self.handle), ctypes.byref(desc), _stream_ptr(stream)))
        self.layout = layout
        self._keep = None

    def close(self):
        if self.handle:
            _check(load().dct_plan_destroy(self.handle))
            self.handle = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dct_plan_create(max_width, max_height, layout=DCT_LAYOUT_GRAY8, max_batch=0, stream=None):
    return Plan(max_width, max_height, layout, max_batch, stream)


def dct_plan_destroy(plan):
    plan.close()


def dct_compress(plan, planes, quality, qtab=None, coeffs=None, stats=None, stream=None):
    """Forward path on a list of uint8 planes; returns the int16 coefficients
    (allocated when ``coeffs`` is None).  ``stats`` (uint64 tensor of
    STATS_WORDS per plane, viewed as int64) receives the statistics."""
    shapes = [tuple(p.shape) for p in planes]
    if coeffs is None:
        coeffs = torch.empty(coeff_count(shapes), dtype=torch.int16, device=planes[0].device)
    _require_cuda(coeffs, stats)
    qa, n = _qtab(qtab)
    _check(load().dct_compress(plan.handle, _planes(planes), len(planes), int(quality), _u16p(qa), n,
                               ctypes.c_void_p(coeffs.data_ptr()),
                               ctypes.c_void_p(stats.data_ptr()) if stats is not None else None,
                               _stream_ptr(stream)))
    return coeffs


def dct_reconstruct(plan, coeffs, out_planes, quality, qtab=None, ref_planes=None, sse=None, stream=None):
    """Inverse path into the given uint8 output planes; with ``ref_planes``
    the per-plane SSE goes to ``sse`` (int64 tensor, allocated if None) and
    is returned."""
    _require_cuda(coeffs)
    qa, n = _qtab(qtab)
    refs = None
    if ref_planes is not None:
        refs = _planes(ref_planes)
        if sse is None:
            sse = torch.empty(len(out_planes), dtype=torch.int64, device=coeffs.device)
    _check(load().dct_reconstruct(plan.handle, ctypes.c_void_p(coeffs.data_ptr()), _planes(out_planes),
                                  len(out_planes), int(quality), _u16p(qa), n, refs,
                                  ctypes.c_void_p(sse.data_ptr()) if sse is not None else None,
                                  _stream_ptr(stream)))
    return sse


def dct_codec_fused(plan, planes, quality, qtab=None, coeffs=None, recon_planes=None, sse=None, stream=None):
    """One pass: forward, quantise, dequantise, inverse and SSE.  Returns the
    per-plane SSE tensor (int64)."""
    if sse is None:
        sse = torch.empty(len(planes), dtype=torch.int64, device=planes[0].device)
    _require_cuda(sse, coeffs)
    qa, n = _qtab(qtab)
    _check(load().dct_codec_fused(plan.handle, _planes(planes), len(planes), int(quality), _u16p(qa), n,
                                  ctypes.c_void_p(coeffs.data_ptr()) if coeffs is not None else None,
                                  _planes(recon_planes) if recon_planes is not None else None,
                                  ctypes.c_void_p(sse.data_ptr()), _stream_ptr(stream)))
    return sse


def dct_psnr(plan, a_planes, b_planes, max_value=0.0, sse=None, host=True, stream=None):
    """SSE (device int64 tensor) and, with host=True, the per-plane PSNRs plus
    the sample-weighted total (a list of nplanes + 1 floats)."""
    if sse is None:
        sse = torch.empty(len(a_planes), dtype=torch.int64, device=a_planes[0].device)
    out = (ctypes.c_double * (len(a_planes) + 1))() if host else None
    _check(load().dct_psnr(plan.handle, _planes(a_planes), _planes(b_planes), len(a_planes),
                           ctypes.c_void_p(sse.data_ptr()), out, float(max_value), _stream_ptr(stream)))
    return sse, (list(out) if host else None)


def make_batch_items(srcs, qualities, coeffs=None, recons=None, chroma=None, qtabs=None):
    """ctypes array of dct_batch_item for lists of planes and per-item settings."""
    n = len(srcs)
    arr = (dct_batch_item * n)()
    # the plan keeps raw device pointers until the next prepare: hold the tensors
    keep = [list(srcs), list(coeffs or []), list(recons or [])]
    for i in range(n):
        it = arr[i]
        it.src = as_plane(srcs[i])
        it.coeffs = coeffs[i].data_ptr() if coeffs is not None and coeffs[i] is not None else None
        if recons is not None and recons[i] is not None:
            it.recon = recons[i].data_ptr()
            it.recon_pitch = recons[i].stride(0)
        it.quality = int(qualities[i])
        it.chroma = int(bool(chroma[i])) if chroma is not None else 0
        if qtabs is not None and qtabs[i] is not None:
            qa = np.ascontiguousarray(np.asarray(qtabs[i], dtype=np.uint16).reshape(64))
            keep.append(qa)
            it.qtab_host = qa.ctypes.data_as(_U16P)
    return arr, keep


def dct_batch_prepare(plan, items, ops, sse=None, shape=None, stream=None):
    arr, keep = items
    sh = dct_launch_shape(*shape) if shape is not None else None
    _check(load().dct_batch_prepare(plan.handle, arr, len(arr), int(ops),
                                    ctypes.c_void_p(sse.data_ptr()) if sse is not None else None,
                                    ctypes.byref(sh) if sh is not None else None, _stream_ptr(stream)))
    plan._keep = (arr, keep, sse)


def dct_batch_launch(plan, stream=None):
    _check(load().dct_batch_launch(plan.handle, _stream_ptr(stream)))


def dct_autotune(plan, stream=None):
    sh = dct_launch_shape()
    ms = ctypes.c_float()
    _check(load().dct_autotune(plan.handle, ctypes.byref(sh), ctypes.byref(ms), _stream_ptr(stream)))
    return (sh.threads_per_cta, sh.ctas_per_sm, sh.tile_blocks, sh.reserved), ms.value


def psnr_list_from_sse(sse_values, shapes, max_value=0.0):
    out = [dct_psnr_from_sse(int(s), h * w, max_value) for s, (h, w) in zip(sse_values, shapes)]
    tot = sum(int(s) for s in sse_values)
    n = sum(h * w for h, w in shapes)
    out.append(dct_psnr_from_sse(tot, n, max_value))
    return out


__all__ = [n for n in dir() if n.startswith("dct_")] + ["Plan", "load", "DctError", "as_plane", "coeff_count",
                                                          "make_batch_items", "STATS_LAYOUT", "STATS_WORDS"]
_ = math  # noqa
