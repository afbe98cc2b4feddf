"""Thin Python binding of the C ABI in include/sfmm.h (argument marshalling only).

Every computation runs in the CUDA kernels of libsfmm.so; this module only
converts Python/torch arguments to plain pointers and sizes and turns status
codes into exceptions.  There is no fallback: if the library is missing the
import of this module fails with instructions to build it.

Names follow the C ABI: sfmm_create -> Handle(...), sfmm_m2l_batch ->
m2l_batch(...), and so on.  Device arrays are passed as torch tensors (or raw
integer device addresses); `stream` defaults to torch's current stream.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsfmm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)

F32, F64 = 0, 1
M2M, M2L, L2L = 0, 1, 2
OPS = {"m2m": M2M, "m2l": M2L, "l2l": L2L}

STATUS = {
    0: "SFMM_OK", 1: "SFMM_ERR_ARG", 2: "SFMM_ERR_ORDER", 3: "SFMM_ERR_NOMEM",
    4: "SFMM_ERR_CUDA", 5: "SFMM_ERR_TIMEOUT", 6: "SFMM_ERR_UNSUPPORTED", 7: "SFMM_ERR_DEVICE",
}

_vp, _i, _ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
_dp = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "sfmm_status_string": (ctypes.c_char_p, [_i]),
    "sfmm_create": (_i, [_i, _i, ctypes.POINTER(_vp)]),
    "sfmm_destroy": (_i, [_vp]),
    "sfmm_get_info": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "sfmm_m2m_batch": (_i, [_vp, _vp, _vp, _vp, _i, _i, _ll, _i, _vp]),
    "sfmm_m2l_batch": (_i, [_vp, _vp, _vp, _vp, _i, _i, _ll, _i, _vp]),
    "sfmm_l2l_batch": (_i, [_vp, _vp, _vp, _vp, _i, _i, _ll, _i, _vp]),
    "sfmm_translate_lists": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _i, _i, _ll, _i, _vp]),
    "sfmm_p2m_boxes": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _ll, _vp]),
    "sfmm_p2l_boxes": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _ll, _vp]),
    "sfmm_sync_status": (_i, [_vp, _vp, ctypes.POINTER(_i)]),
    "sfmm_translate_batch_noalloc": (_i, [_vp, _i, _vp, _vp, _vp, _i, _i, _ll, _i, _vp]),
    "sfmm_translate_lists_multi": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp, _i, _vp]),
    "sfmm_translate_pass": (_i, [_vp, _vp, _i, _vp]),
    "sfmm_set_policy": (_i, [_vp, _i, _i, _i, _i, _i]),
    "sfmm_reserve_scratch": (_i, [_vp, _i]),
    "sfmm_grid_create": (_i, [_vp, _i, _i, ctypes.POINTER(_vp)]),
    "sfmm_grid_m2l": (_i, [_vp, ctypes.c_double, _vp, _vp, _i, _vp]),
    "sfmm_grid_destroy": (_i, [_vp]),
    "sfmm_grid_inject_timeout": (_i, [_vp, _ll]),
    "sfmm_host_swap_matrices": (_i, [_i, _dp, _dp]),
    "sfmm_host_ztranslate": (_i, [_i, _i, _i, _dp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class SfmmError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = _lib.sfmm_status_string(code).decode()
        super().__init__(f"{what}: {msg}" if what else msg)


def _check(code, what):
    if code != 0:
        raise SfmmError(code, what)


def status_string(code):
    return _lib.sfmm_status_string(int(code)).decode()


def _addr(x):
    """Device address of a torch tensor, or an integer address as is."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Handle:
    """sfmm_create / sfmm_destroy: tables for orders <= P_max on the current device."""

    def __init__(self, P_max, dtype="f64"):
        self.dtype_code = {"f64": F64, "f32": F32, F64: F64, F32: F32}[dtype]
        self.P_max = int(P_max)
        h = _vp()
        _check(_lib.sfmm_create(self.P_max, self.dtype_code, ctypes.byref(h)), "sfmm_create")
        self._h = h

    @property
    def ptr(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.sfmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        p, d = _i(), _i()
        _check(_lib.sfmm_get_info(self._h, ctypes.byref(p), ctypes.byref(d)), "sfmm_get_info")
        return p.value, d.value

    def sync_status(self, stream=None):
        v = _i()
        code = _lib.sfmm_sync_status(self._h, _stream(stream), ctypes.byref(v))
        if code not in (0, 7):
            _check(code, "sfmm_sync_status")
        return v.value


def _batch(fn, h, inp, out, shift, p_in, p_out, count, accumulate, stream):
    _check(fn(h.ptr, _addr(inp), _addr(out), _addr(shift), int(p_in), int(p_out), int(count),
              int(bool(accumulate)), _stream(stream)), fn.__name__)


def m2m_batch(h, inp, out, shift, p_in, p_out, count, accumulate=False, stream=None):
    """sfmm_m2m_batch: inp/out are device arrays of `count` solid pointers (int64)."""
    _batch(_lib.sfmm_m2m_batch, h, inp, out, shift, p_in, p_out, count, accumulate, stream)


def m2l_batch(h, inp, out, shift, p_in, p_out, count, accumulate=False, stream=None):
    """sfmm_m2l_batch: inp/out are device arrays of `count` solid pointers (int64)."""
    _batch(_lib.sfmm_m2l_batch, h, inp, out, shift, p_in, p_out, count, accumulate, stream)


def l2l_batch(h, inp, out, shift, p_in, p_out, count, accumulate=False, stream=None):
    """sfmm_l2l_batch: inp/out are device arrays of `count` solid pointers (int64)."""
    _batch(_lib.sfmm_l2l_batch, h, inp, out, shift, p_in, p_out, count, accumulate, stream)


def translate_batch(op, h, *args, **kw):
    {"m2m": m2m_batch, "m2l": m2l_batch, "l2l": l2l_batch}[op](h, *args, **kw)


def translate_batch_noalloc(h, op, inp, out, shift, p_in, p_out, count, accumulate=False,
                            stream=None):
    """sfmm_translate_batch_noalloc: like the *_batch calls, for callers that
    cannot allocate device memory (scratch is a fixed array in the library)."""
    _check(_lib.sfmm_translate_batch_noalloc(h.ptr, OPS.get(op, op), _addr(inp), _addr(out),
                                             _addr(shift), int(p_in), int(p_out), int(count),
                                             int(bool(accumulate)), _stream(stream)),
           "sfmm_translate_batch_noalloc")


def translate_lists(h, op, src, shift, offsets, out, p_in, p_out, n_targets,
                    accumulate=False, stream=None):
    """sfmm_translate_lists: target-major CSR lists (offsets: int64, n_targets+1)."""
    _check(_lib.sfmm_translate_lists(h.ptr, OPS.get(op, op), _addr(src), _addr(shift),
                                     _addr(offsets), _addr(out), int(p_in), int(p_out),
                                     int(n_targets), int(bool(accumulate)), _stream(stream)),
           "sfmm_translate_lists")


class ListClass(ctypes.Structure):
    """sfmm_list_class: one (op, p_in, p_out) class of a multi-class lists call."""
    _fields_ = [("op", ctypes.c_int), ("p_in", ctypes.c_int), ("p_out", ctypes.c_int),
                ("lanes_per_target", ctypes.c_int), ("target_begin", ctypes.c_longlong),
                ("target_end", ctypes.c_longlong)]


MAX_CLASSES = 256
POLICY = {"auto": 0, "unrolled": 1, "shared": 2, "global": 3, "wide": 4}
# Orders p_in = p_out with fully unrolled kernels in libsfmm.so (one unit per
# order and real type, listed in csrc/sfmm_unrolled_registry.cu); AUTO takes
# them for these orders, SFMM_POLICY_UNROLLED accepts only these.
UNROLLED_ORDERS = (1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12)


def translate_lists_multi(h, classes, src, shift, offsets, out, accumulate=False, stream=None):
    """sfmm_translate_lists_multi: classes = [(op, p_in, p_out, target_begin,
    target_end[, lanes_per_target])] (lanes_per_target 0 = the default)."""
    arr = (ListClass * len(classes))()
    for k, cl in enumerate(classes):
        op, pi, po, tb, te = cl[:5]
        lanes = int(cl[5]) if len(cl) > 5 else 0
        arr[k] = ListClass(OPS.get(op, op), int(pi), int(po), lanes, int(tb), int(te))
    _check(_lib.sfmm_translate_lists_multi(h.ptr, ctypes.cast(arr, _vp), len(classes), _addr(src),
                                           _addr(shift), _addr(offsets), _addr(out),
                                           int(bool(accumulate)), _stream(stream)),
           "sfmm_translate_lists_multi")


class PassClass(ctypes.Structure):
    """sfmm_pass_class (include/sfmm.h)."""
    _fields_ = [("op", _i), ("p_in", _i), ("p_out", _i), ("lanes_per_target", _i),
                ("phase", _i), ("accumulate", _i), ("n_targets", _ll),
                ("src", _vp), ("shift", _vp), ("offsets", _vp), ("out", _vp)]


MAX_PASS_CLASSES = 320
MAX_PASS_PHASES = 64


def pass_classes(classes):
    """Pack (op, p_in, p_out, lanes, phase, accumulate, n_targets, src, shift,
    offsets, out) tuples (arrays as tensors or addresses) into the C array."""
    arr = (PassClass * len(classes))()
    for k, (op, pi, po, g, ph, acc, nt, src, shift, offs, out) in enumerate(classes):
        arr[k] = PassClass(OPS.get(op, op), int(pi), int(po), int(g), int(ph), int(bool(acc)), int(nt),
                           _addr(src), _addr(shift), _addr(offs), _addr(out))
    return arr


def translate_pass(h, classes, stream=None):
    """sfmm_translate_pass: a whole pass of phased classes in one launch.
    `classes` is the packed array of pass_classes()."""
    _check(_lib.sfmm_translate_pass(h.ptr, ctypes.cast(classes, _vp), len(classes), _stream(stream)),
           "sfmm_translate_pass")


def set_policy(h, op, p_in, p_out, policy="auto", warps=0):
    """sfmm_set_policy: kernel variant and warps per block for (op, p_in, p_out)."""
    _check(_lib.sfmm_set_policy(h.ptr, OPS.get(op, op), int(p_in), int(p_out),
                                POLICY.get(policy, policy), int(warps)), "sfmm_set_policy")


def reserve_scratch(h, p_in_max):
    """sfmm_reserve_scratch: global scratch for inputs up to order p_in_max."""
    _check(_lib.sfmm_reserve_scratch(h.ptr, int(p_in_max)), "sfmm_reserve_scratch")


class Grid:
    """sfmm_grid_create / sfmm_grid_m2l / sfmm_grid_destroy: tensor-core M2L of one
    uniform octree level (P = 16)."""

    def __init__(self, h, P, nside):
        g = _vp()
        _check(_lib.sfmm_grid_create(h.ptr, int(P), int(nside), ctypes.byref(g)), "sfmm_grid_create")
        self._g, self.P, self.nside = g, P, nside

    def m2l(self, box_size, M, L, accumulate=False, stream=None):
        _check(_lib.sfmm_grid_m2l(self._g, float(box_size), _addr(M), _addr(L),
                                  int(bool(accumulate)), _stream(stream)), "sfmm_grid_m2l")

    def inject_timeout(self, after_chunks):
        """sfmm_grid_inject_timeout: fault injection for the time-out path (tests)."""
        _check(_lib.sfmm_grid_inject_timeout(self._g, int(after_chunks)), "sfmm_grid_inject_timeout")

    def close(self):
        if getattr(self, "_g", None):
            _lib.sfmm_grid_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def p2m_boxes(h, P, points, q, offsets, centres, out, n_boxes, stream=None):
    _check(_lib.sfmm_p2m_boxes(h.ptr, int(P), _addr(points), _addr(q), _addr(offsets),
                               _addr(centres), _addr(out), int(n_boxes), _stream(stream)),
           "sfmm_p2m_boxes")


def p2l_boxes(h, P, points, q, offsets, centres, out, n_boxes, stream=None):
    _check(_lib.sfmm_p2l_boxes(h.ptr, int(P), _addr(points), _addr(q), _addr(offsets),
                               _addr(centres), _addr(out), int(n_boxes), _stream(stream)),
           "sfmm_p2l_boxes")


def host_swap_matrices(n):
    """sfmm_host_swap_matrices: dense F_n, G_n (numpy, (n+1)x(n+1))."""
    import numpy as np
    F = np.zeros((n + 1, n + 1))
    G = np.zeros((n + 1, n + 1))
    _check(_lib.sfmm_host_swap_matrices(int(n), F.ctypes.data_as(_dp), G.ctypes.data_as(_dp)),
           "sfmm_host_swap_matrices")
    return F, G


def host_ztranslate(op, P, m):
    """sfmm_host_ztranslate: dense z-axis translation block (numpy, (P-m)x(P-m))."""
    import numpy as np
    T = np.zeros((P - m, P - m))
    _check(_lib.sfmm_host_ztranslate(OPS.get(op, op), int(P), int(m), T.ctypes.data_as(_dp)),
           "sfmm_host_ztranslate")
    return T


def solid_size(P):
    return P * (P + 1)


def pointer_array(base, stride_elems, index):
    """Device int64 array of addresses base + index*stride (torch, on base's device)."""
    import torch
    idx = index if isinstance(index, torch.Tensor) else torch.as_tensor(index)
    idx = idx.to(device=base.device, dtype=torch.int64)
    return idx * (stride_elems * base.element_size()) + base.data_ptr()
