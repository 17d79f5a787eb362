"""Thin ctypes binding of libdctgb (include/dctgb.h) with the same entry-point
names.  It only marshals arguments: torch tensors become device pointers,
sizes and pitches; every step of the codec runs in the library's kernels.
There is no CPU fallback: without the library or a CUDA device the calls
raise.
"""
import contextlib
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
                ("tile_blocks", ctypes.c_int32), ("lanes_per_block", ctypes.c_int32)]


DCT_MLP_INPUTS = 80
DCT_MLP_HIDDEN = 64
DCT_MLP_PARAMS = 9409


class dct_mlp(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("adam_m", ctypes.c_void_p), ("adam_v", ctypes.c_void_p),
                ("feat_mean", ctypes.c_void_p), ("feat_std", ctypes.c_void_p), ("step", ctypes.c_int32),
                ("act_bf16", ctypes.c_int32)]


class dct_rc_summary(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_int32), ("fell_back", ctypes.c_int32), ("unreachable", ctypes.c_int32),
                ("within_tol", ctypes.c_int32), ("passes", ctypes.c_int32), ("gpu_ms", ctypes.c_float)]


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
    "dct_exact_fused": (ctypes.c_int, [_P, ctypes.POINTER(dct_plane), ctypes.c_int, ctypes.c_int, _U16P,
                                       ctypes.c_int, _P, ctypes.POINTER(dct_plane), _P, _P]),
    "dct_rgb_to_yuv420": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(dct_plane),
                                         ctypes.POINTER(dct_plane), ctypes.POINTER(dct_plane), _P]),
    "dct_compress_rgb": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int, _U16P,
                                        ctypes.c_int, _P, _P]),
    "dct_entropy_stats": (ctypes.c_int, [_P, _P, ctypes.POINTER(dct_plane), ctypes.c_int, _P, _P]),
    "dct_entropy_bits": (ctypes.c_double, [ctypes.POINTER(ctypes.c_uint64)]),
    "dct_huffman_bits": (ctypes.c_uint64, [ctypes.POINTER(ctypes.c_uint64)]),
    "dct_psnr": (ctypes.c_int, [_P, ctypes.POINTER(dct_plane), ctypes.POINTER(dct_plane), ctypes.c_int, _P,
                                ctypes.POINTER(ctypes.c_double), ctypes.c_double, _P]),
    "dct_psnr_from_sse": (ctypes.c_double, [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double]),
    "dct_psnr_from_sse_list": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int64),
                                              ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "dct_mlp_labels": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "dct_batch_prepare": (ctypes.c_int, [_P, ctypes.POINTER(dct_batch_item), ctypes.c_int, ctypes.c_uint32, _P,
                                         ctypes.POINTER(dct_launch_shape), _P]),
    "dct_batch_launch": (ctypes.c_int, [_P, _P]),
    "dct_autotune": (ctypes.c_int, [_P, ctypes.POINTER(dct_launch_shape), ctypes.POINTER(ctypes.c_float), _P]),
    "dct_features": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, _P, _P]),
    "dct_mlp_set_norm": (ctypes.c_int, [ctypes.POINTER(dct_mlp), _P, ctypes.c_int, _P]),
    "dct_mlp_forward": (ctypes.c_int, [ctypes.POINTER(dct_mlp), _P, ctypes.c_int, _P, _P, _P]),
    "dct_mlp_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int]),
    "dct_mlp_loss_grad": (ctypes.c_int, [ctypes.POINTER(dct_mlp), _P, _P, _P, ctypes.c_int, _P, _P, _P, _P]),
    "dct_mlp_adam": (ctypes.c_int, [ctypes.POINTER(dct_mlp), _P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, _P]),
    "dct_mlp_train_epoch": (ctypes.c_int, [ctypes.POINTER(dct_mlp), _P, _P, _P, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_float, _P, _P, _P]),
    "dct_rate_control": (ctypes.c_int, [_P, ctypes.POINTER(dct_plane), ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_float), ctypes.POINTER(dct_mlp),
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(dct_rc_summary), _P]),
    "dct_rate_features": (ctypes.c_int, [_P, ctypes.POINTER(dct_plane), ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_float), _P, _P]),
    "dct_batch_run_noalloc": (ctypes.c_int, [ctypes.POINTER(dct_batch_item), ctypes.c_int, ctypes.c_uint32, _P, _P]),
    "dct_int_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float), _P]),
    "dct_debug_fail_alloc": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "dct_last_error": (ctypes.c_char_p, []),
}

_LIBS = {}
_ACTIVE_N = None     # CORDIC count of the library the calls below use (None: the spec's)


def load(build_if_needed=True, n=None):
    """Loads (building first if needed) the in-tree libdctgb.so, or with n
    the same library compiled at CORDIC iteration count n.  Without n it
    returns the library selected by ``cordic_variant`` (default: the spec's)."""
    n = _ACTIVE_N if n is None else n
    key = _build.lib_path(n)
    if key in _LIBS:
        return _LIBS[key]
    path = key
    if build_if_needed and not _build.up_to_date(n):
        path = _build.build(n=n)
    if not os.path.exists(path):
        raise RuntimeError("%s is missing; run paper_1306_1373_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIBS[key] = lib
    return lib


@contextlib.contextmanager
def cordic_variant(n):
    """Within the block every call of this module goes to the library
    compiled at CORDIC iteration count n.  Plans are tied to the library
    that created them: create and use them inside the same block."""
    global _ACTIVE_N
    old = _ACTIVE_N
    lib = load(n=n)
    _ACTIVE_N = n
    try:
        yield lib
    finally:
        _ACTIVE_N = old


def declared_symbols():
    return list(_SIGNATURES)


def _check(status, lib=None):
    if status != DCT_OK:
        raise DctError(status, (lib or load()).dct_last_error().decode())


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


class PlaneArray:
    """A ctypes dct_plane array built once from a list of uint8 CUDA tensors
    (it keeps the tensors alive); pass it wherever a list of planes goes to
    avoid rebuilding the descriptors on every call."""

    def __init__(self, tensors):
        self.tensors = list(tensors)
        n = len(self.tensors)
        self.arr = (dct_plane * n)()
        for i, t in enumerate(self.tensors):
            self.arr[i] = as_plane(t)

    def __len__(self):
        return len(self.tensors)

    def __getitem__(self, i):
        return self.tensors[i]


def _planes(ts):
    if isinstance(ts, PlaneArray):
        return ts.arr
    return (dct_plane * len(ts))(*[as_plane(t) for t in ts])


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
        self.lib = load()          # the library (CORDIC variant) that owns this plan
        desc = dct_plan_desc(int(max_width), int(max_height), int(layout), int(max_batch), 0)
        _check(self.lib.dct_plan_create(ctypes.byref(self.handle), ctypes.byref(desc), _stream_ptr(stream)), self.lib)
        self.layout = layout
        self._keep = None

    def close(self):
        if self.handle:
            _check(self.lib.dct_plan_destroy(self.handle), self.lib)
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
    _check(plan.lib.dct_compress(plan.handle, _planes(planes), len(planes), int(quality), _u16p(qa), n,
                               ctypes.c_void_p(coeffs.data_ptr()),
                               ctypes.c_void_p(stats.data_ptr()) if stats is not None else None,
                               _stream_ptr(stream)), plan.lib)
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
    _check(plan.lib.dct_reconstruct(plan.handle, ctypes.c_void_p(coeffs.data_ptr()), _planes(out_planes),
                                  len(out_planes), int(quality), _u16p(qa), n, refs,
                                  ctypes.c_void_p(sse.data_ptr()) if sse is not None else None,
                                  _stream_ptr(stream)), plan.lib)
    return sse


def dct_codec_fused(plan, planes, quality, qtab=None, coeffs=None, recon_planes=None, sse=None, stream=None):
    """One pass: forward, quantise, dequantise, inverse and SSE.  Returns the
    per-plane SSE tensor (int64)."""
    if sse is None:
        sse = torch.empty(len(planes), dtype=torch.int64, device=planes[0].device)
    _require_cuda(sse, coeffs)
    qa, n = _qtab(qtab)
    _check(plan.lib.dct_codec_fused(plan.handle, _planes(planes), len(planes), int(quality), _u16p(qa), n,
                                  ctypes.c_void_p(coeffs.data_ptr()) if coeffs is not None else None,
                                  _planes(recon_planes) if recon_planes is not None else None,
                                  ctypes.c_void_p(sse.data_ptr()), _stream_ptr(stream)), plan.lib)
    return sse


def dct_exact_fused(plan, planes, quality, qtab=None, coeffs=None, recon_planes=None, sse=None, stream=None):
    """Exact-DCT pipeline (float32, Eq. 6) in one pass; returns the per-plane
    SSE tensor (int64)."""
    if sse is None:
        sse = torch.empty(len(planes), dtype=torch.int64, device=planes[0].device)
    qa, n = _qtab(qtab)
    _check(plan.lib.dct_exact_fused(plan.handle, _planes(planes), len(planes), int(quality), _u16p(qa), n,
                                  ctypes.c_void_p(coeffs.data_ptr()) if coeffs is not None else None,
                                  _planes(recon_planes) if recon_planes is not None else None,
                                  ctypes.c_void_p(sse.data_ptr()), _stream_ptr(stream)), plan.lib)
    return sse


def dct_rgb_to_yuv420(rgb, y=None, cb=None, cr=None, stream=None):
    """(H, W, 3) uint8 CUDA tensor (rows may be padded) -> (Y, Cb, Cr) planes."""
    if rgb.dtype != torch.uint8 or rgb.dim() != 3 or rgb.shape[2] != 3 or rgb.stride(2) != 1 or rgb.stride(1) != 3:
        raise ValueError("rgb must be an (H, W, 3) uint8 tensor with interleaved channels")
    _require_cuda(rgb)
    h, w = rgb.shape[:2]
    ch, cw = (h + 1) // 2, (w + 1) // 2
    y = torch.empty(h, w, dtype=torch.uint8, device=rgb.device) if y is None else y
    cb = torch.empty(ch, cw, dtype=torch.uint8, device=rgb.device) if cb is None else cb
    cr = torch.empty(ch, cw, dtype=torch.uint8, device=rgb.device) if cr is None else cr
    py, pb, pr = as_plane(y), as_plane(cb), as_plane(cr)
    _check(load().dct_rgb_to_yuv420(ctypes.c_void_p(rgb.data_ptr()), w, h, rgb.stride(0), ctypes.byref(py),
                                    ctypes.byref(pb), ctypes.byref(pr), _stream_ptr(stream)))
    return y, cb, cr


def rgb_coeff_count(height, width):
    """int16 codes dct_compress_rgb writes for an RGB frame: Y, Cb, Cr."""
    ch, cw = (height + 1) // 2, (width + 1) // 2
    return coeff_count([(height, width), (ch, cw), (ch, cw)])


def dct_compress_rgb(plan, rgb, quality, qtab=None, coeffs=None, stream=None):
    """(H, W, 3) uint8 CUDA tensor (rows may be padded) -> int16 codes of its
    Y, Cb and Cr planes (4:2:0), converted and coded in one pass."""
    if rgb.dtype != torch.uint8 or rgb.dim() != 3 or rgb.shape[2] != 3 or rgb.stride(2) != 1 or rgb.stride(1) != 3:
        raise ValueError("rgb must be an (H, W, 3) uint8 tensor with interleaved channels")
    _require_cuda(rgb, coeffs)
    h, w = rgb.shape[:2]
    if coeffs is None:
        coeffs = torch.empty(rgb_coeff_count(h, w), dtype=torch.int16, device=rgb.device)
    qa, n = _qtab(qtab)
    _check(plan.lib.dct_compress_rgb(plan.handle, ctypes.c_void_p(rgb.data_ptr()), w, h, rgb.stride(0), int(quality),
                                     _u16p(qa), n, ctypes.c_void_p(coeffs.data_ptr()), _stream_ptr(stream)), plan.lib)
    return coeffs


DCT_ENTROPY_WORDS = 274


def dct_entropy_stats(plan, coeffs, shapes, stream=None):
    """Symbol statistics (device int64 tensor, planes x 274) of coefficients
    laid out for planes of the given (height, width) shapes."""
    n = len(shapes)
    arr = (dct_plane * n)(*[dct_plane(None, w, h, w) for h, w in shapes])
    out = torch.empty(n, DCT_ENTROPY_WORDS, dtype=torch.int64, device=coeffs.device)
    _check(plan.lib.dct_entropy_stats(plan.handle, ctypes.c_void_p(coeffs.data_ptr()), arr, n,
                                    ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), plan.lib)
    return out


def dct_entropy_bits(stats_row):
    """Bits of one plane from its 274 statistics words (host)."""
    a = np.ascontiguousarray(np.asarray(stats_row, dtype=np.uint64))
    return load().dct_entropy_bits(a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))


def dct_huffman_bits(stats_row):
    """Achievable bits of one plane (16-bit length-limited optimal prefix
    codes for its DC and AC symbols) from its 274 statistics words (host)."""
    a = np.ascontiguousarray(np.asarray(stats_row, dtype=np.uint64))
    return int(load().dct_huffman_bits(a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))


def dct_psnr(plan, a_planes, b_planes, max_value=0.0, sse=None, host=True, stream=None):
    """SSE (device int64 tensor) and, with host=True, the per-plane PSNRs plus
    the sample-weighted total (a list of nplanes + 1 floats)."""
    if sse is None:
        sse = torch.empty(len(a_planes), dtype=torch.int64, device=a_planes[0].device)
    out = (ctypes.c_double * (len(a_planes) + 1))() if host else None
    _check(plan.lib.dct_psnr(plan.handle, _planes(a_planes), _planes(b_planes), len(a_planes),
                           ctypes.c_void_p(sse.data_ptr()), out, float(max_value), _stream_ptr(stream)), plan.lib)
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
    _check(plan.lib.dct_batch_prepare(plan.handle, arr, len(arr), int(ops),
                                    ctypes.c_void_p(sse.data_ptr()) if sse is not None else None,
                                    ctypes.byref(sh) if sh is not None else None, _stream_ptr(stream)), plan.lib)
    plan._keep = (arr, keep, sse)


def dct_batch_launch(plan, stream=None):
    _check(plan.lib.dct_batch_launch(plan.handle, _stream_ptr(stream)), plan.lib)


def dct_batch_run_noalloc(items, ops, sse=None, stream=None):
    """One batch of at most 64 items through the allocation-free entry
    point (the work list lives in a fixed array inside the library)."""
    arr, _ = items
    _check(load().dct_batch_run_noalloc(arr, len(arr), int(ops),
                                        ctypes.c_void_p(sse.data_ptr()) if sse is not None else None,
                                        _stream_ptr(stream)))


def dct_int_peak(kind=1, iters=4096, stream=None):
    """Integer issue-rate probe: (ops per clock per SM, Tops/s, ms) for the
    CORDIC micro-rotation in instruction form ``kind`` (0, 1, 2 or 3)."""
    opc, tops, ms = ctypes.c_double(), ctypes.c_double(), ctypes.c_float()
    _check(load().dct_int_peak(int(kind), int(iters), ctypes.byref(opc), ctypes.byref(tops), ctypes.byref(ms),
                               _stream_ptr(stream)))
    return opc.value, tops.value, ms.value


def dct_debug_fail_alloc(nth):
    """Arms (nth >= 1) or disarms (0) the allocation-failure hook of the
    active library; returns the allocation attempts counted so far."""
    att = ctypes.c_int64()
    _check(load().dct_debug_fail_alloc(int(nth), ctypes.byref(att)))
    return att.value


def dct_autotune(plan, stream=None):
    """Times candidate launch shapes for the prepared batch; returns
    ((threads, ctas_per_sm, tile_blocks, lanes_per_block), best ms)."""
    sh = dct_launch_shape()
    ms = ctypes.c_float()
    _check(plan.lib.dct_autotune(plan.handle, ctypes.byref(sh), ctypes.byref(ms), _stream_ptr(stream)), plan.lib)
    return (sh.threads_per_cta, sh.ctas_per_sm, sh.tile_blocks, sh.lanes_per_block), ms.value


def autotune_cached(plan, items, ops, sse=None, cache_path=None, key=None, stream=None):
    """dct_batch_prepare with a launch shape from a JSON cache keyed by
    (GPU name, key); on a miss it runs dct_autotune and stores the result.
    Returns the shape used."""
    import json
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    k = "%s|%s|ops=%d" % (name, key, int(ops))
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except ValueError:
            cache = {}
    if k in cache:
        shape = tuple(cache[k]["shape"])
        dct_batch_prepare(plan, items, ops, sse=sse, shape=shape, stream=stream)
        return shape
    dct_batch_prepare(plan, items, ops, sse=sse, stream=stream)
    shape, ms = dct_autotune(plan, stream=stream)
    cache[k] = {"shape": list(shape), "ms": ms}
    if cache_path:
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return shape


def dct_psnr_from_sse_list(sse_values, sample_counts, max_value=0.0):
    """Per-plane PSNRs and the sample-weighted PSNR over all planes (a list
    of n + 1 floats), from host SSE values and sample counts."""
    n = len(sse_values)
    s = (ctypes.c_uint64 * n)(*[int(v) for v in sse_values])
    c = (ctypes.c_int64 * n)(*[int(v) for v in sample_counts])
    out = (ctypes.c_double * (n + 1))()
    _check(load().dct_psnr_from_sse_list(s, c, n, float(max_value), out))
    return list(out)


def psnr_list_from_sse(sse_values, shapes, max_value=0.0):
    """dct_psnr_from_sse_list for planes of the given (height, width) shapes."""
    return dct_psnr_from_sse_list(sse_values, [h * w for h, w in shapes], max_value)


# ---------------------------------------------------------------------------
# learned rate control
# ---------------------------------------------------------------------------

def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Mlp:
    """Device-resident network 80 -> 64 -> 64 -> 1 (dct_mlp) with its Adam
    state and input normalisation, as torch float32 tensors."""

    def __init__(self, params, act_bf16=True, device="cuda"):
        p = torch.as_tensor(np.asarray(params, dtype=np.float32)).to(device)
        if p.numel() != DCT_MLP_PARAMS:
            raise ValueError("expected %d parameters" % DCT_MLP_PARAMS)
        self.params = p.contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.mean = torch.zeros(DCT_MLP_INPUTS, dtype=torch.float32, device=device)
        self.std = torch.ones(DCT_MLP_INPUTS, dtype=torch.float32, device=device)
        self.c = dct_mlp(self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.mean.data_ptr(),
                         self.std.data_ptr(), 0, 1 if act_bf16 else 0)
        self._ws = None
        self._ws_batch = 0

    @property
    def step(self):
        return self.c.step

    def workspace(self, batch):
        if self._ws is None or self._ws_batch < batch:
            nbytes = load().dct_mlp_workspace_bytes(int(batch)) + 4 * DCT_MLP_PARAMS
            self._ws = torch.empty((nbytes + 3) // 4, dtype=torch.float32, device=self.params.device)
            self._ws_batch = batch
        return self._ws

    def set_norm(self, feats, stream=None):
        _check(load().dct_mlp_set_norm(ctypes.byref(self.c), _vp(feats), int(feats.shape[0]), _stream_ptr(stream)))

    def forward(self, feats, stream=None):
        n = int(feats.shape[0])
        y = torch.empty(n, dtype=torch.float32, device=feats.device)
        q = torch.empty(n, dtype=torch.int32, device=feats.device)
        _check(load().dct_mlp_forward(ctypes.byref(self.c), _vp(feats), n, _vp(y), _vp(q), _stream_ptr(stream)))
        return y, q

    def loss_grad(self, feats, labels, index, stream=None):
        grad = torch.empty(DCT_MLP_PARAMS, dtype=torch.float32, device=feats.device)
        loss = torch.empty(1, dtype=torch.float32, device=feats.device)
        ws = self.workspace(int(index.numel()))
        _check(load().dct_mlp_loss_grad(ctypes.byref(self.c), _vp(feats), _vp(labels), _vp(index), int(index.numel()),
                                        _vp(grad), _vp(loss), _vp(ws), _stream_ptr(stream)))
        return loss, grad

    def adam(self, grad, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _check(load().dct_mlp_adam(ctypes.byref(self.c), _vp(grad), float(lr), float(beta1), float(beta2), float(eps),
                                   _stream_ptr(stream)))

    def train_epoch(self, feats, labels, order, batch=256, lr=1e-3, stream=None):
        n = int(order.numel())
        losses = torch.empty((n + batch - 1) // batch, dtype=torch.float32, device=feats.device)
        ws = self.workspace(batch)
        _check(load().dct_mlp_train_epoch(ctypes.byref(self.c), _vp(feats), _vp(labels), _vp(order), n, int(batch),
                                          float(lr), _vp(losses), _vp(ws), _stream_ptr(stream)))
        return losses


def dct_mlp_labels(quality, stream=None):
    """Device float32 training targets (Q - 1) / 99 of a device int32 tensor of qualities."""
    _require_cuda(quality)
    q = quality.to(torch.int32).contiguous()
    out = torch.empty(q.numel(), dtype=torch.float32, device=q.device)
    _check(load().dct_mlp_labels(_vp(q), int(q.numel()), _vp(out), _stream_ptr(stream)))
    return out


def dct_features(stats, width, height, target, stream=None):
    n = int(width.numel())
    out = torch.empty(n, DCT_MLP_INPUTS, dtype=torch.float32, device=stats.device)
    _check(load().dct_features(_vp(stats), _vp(width), _vp(height), _vp(target), n, _vp(out), _stream_ptr(stream)))
    return out


def dct_rate_features(plan, planes, planes_per_frame, targets, stream=None):
    """Features (n, 80) of every frame's plane 0; planes frame-major (a list
    of tensors or a PlaneArray)."""
    nf = len(planes) // planes_per_frame
    t = (ctypes.c_float * nf)(*[float(v) for v in targets])
    out = torch.empty(nf, DCT_MLP_INPUTS, dtype=torch.float32, device=planes[0].device)
    _check(plan.lib.dct_rate_features(plan.handle, _planes(planes), int(planes_per_frame), nf, t, _vp(out),
                                    _stream_ptr(stream)), plan.lib)
    return out


def dct_rate_control(plan, planes, planes_per_frame, targets, net=None, stream=None):
    """Quality per frame for the target PSNRs (bisection when net is None).
    Returns a dict of numpy arrays and the summary."""
    nf = len(planes) // planes_per_frame
    t = (ctypes.c_float * nf)(*[float(v) for v in targets])
    q = np.zeros(nf, dtype=np.int32)
    sse = np.zeros(nf, dtype=np.uint64)
    fell = np.zeros(nf, dtype=np.uint8)
    summ = dct_rc_summary()
    _check(plan.lib.dct_rate_control(plan.handle, _planes(planes), int(planes_per_frame), nf, t,
                                   ctypes.byref(net.c) if net is not None else None,
                                   q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   sse.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                   fell.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.byref(summ),
                                   _stream_ptr(stream)), plan.lib)
    return dict(quality=q, sse=sse, fell_back=fell,
                summary={f: getattr(summ, f) for f, _ in dct_rc_summary._fields_})


__all__ = [n for n in dir() if n.startswith("dct_")] + ["Plan", "Mlp", "PlaneArray", "load", "DctError", "as_plane", "coeff_count",
                                                          "make_batch_items", "STATS_LAYOUT", "STATS_WORDS"]
_ = math  # noqa
