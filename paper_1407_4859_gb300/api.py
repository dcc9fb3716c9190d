"""Thin Python binding of libadha.so: builds the C structs, passes raw pointers, checks status.

PyTorch provides device memory and streams only; every byte the library moves or computes is
moved or computed by its CUDA kernels.  Function names follow the C ABI (adha_remap, ...).
"""
import ctypes

import torch

from . import _lib
from ._lib import adha_schema, adha_layout, adha_section, OPS, check

DTYPE_SIZE = {0: 4, 1: 8, 2: 4, 3: 2}


def _i32_array(xs):
    return (ctypes.c_int32 * max(1, len(xs)))(*xs)


class Schema:
    """Field types of a record (adha_dtype codes: f32=0, f64=1, i32=2, bf16=3)."""

    def __init__(self, dtypes):
        self.dtypes = [int(d) for d in dtypes]
        self._arr = _i32_array(self.dtypes)
        self.c = adha_schema(len(self.dtypes), self._arr)

    @property
    def F(self):
        return len(self.dtypes)


class Layout:
    """An ordered list of field groups (each group one array of C structs)."""

    def __init__(self, groups):
        self.groups = [list(map(int, g)) for g in groups]
        self._len = _i32_array([len(g) for g in self.groups])
        self._fields = _i32_array([f for g in self.groups for f in g])
        self.c = adha_layout(len(self.groups), self._len, self._fields)

    def key(self):
        return tuple(tuple(g) for g in self.groups)

    def __eq__(self, other):
        return isinstance(other, Layout) and self.key() == other.key()

    def __hash__(self):
        return hash(self.key())

    def __repr__(self):
        return "Layout(%r)" % (self.groups,)

    @staticmethod
    def aos(F):
        return Layout([list(range(F))])

    @staticmethod
    def soa(F):
        return Layout([[f] for f in range(F)])


def adha_version():
    return _lib.load().adha_version().decode()


def adha_layout_strides(schema, layout):
    """(group strides, field offsets) in bytes."""
    st = (ctypes.c_int32 * len(layout.groups))()
    off = (ctypes.c_int32 * schema.F)()
    check(_lib.load().adha_layout_strides(ctypes.byref(schema.c), ctypes.byref(layout.c), st, off),
          "adha_layout_strides")
    return list(st), list(off)


def _ptrs(bufs):
    arr = (ctypes.c_void_p * max(1, len(bufs)))()
    for k, b in enumerate(bufs):
        arr[k] = b.data_ptr() if isinstance(b, torch.Tensor) else int(b)
    return arr


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def alloc_layout(schema, layout, n, device="cuda"):
    """One uint8 tensor per group, n * stride bytes each (torch's allocator aligns to 512 bytes)."""
    strides, _ = adha_layout_strides(schema, layout)
    return [torch.empty(n * s, dtype=torch.uint8, device=device) for s in strides]


def c_section(sec, perm=None):
    """adha_section from a synth.Section (perm: device int32 tensor for gather sections)."""
    s = adha_section()
    s.op = OPS[sec.op]
    for k, a in enumerate(sec.args):
        s.arg[k] = int(a)
    for k, p in enumerate(sec.params):
        s.fparam[k] = float(p)
    s.read_mask = sum(1 << f for f in sec.read)
    s.write_mask = sum(1 << f for f in sec.write)
    s.read_at_perm_mask = sum(1 << f for f in sec.read_at_perm)
    s.perm = perm.data_ptr() if (perm is not None and sec.op == "gather") else None
    return s


def adha_remap(schema, n, src_layout, src_bufs, dst_layout, dst_bufs, stream=None):
    check(_lib.load().adha_remap(ctypes.byref(schema.c), int(n), ctypes.byref(src_layout.c), _ptrs(src_bufs),
                                 ctypes.byref(dst_layout.c), _ptrs(dst_bufs), _stream_ptr(stream)), "adha_remap")


def adha_run_section(schema, n, layout, bufs, section, save=None, stream=None):
    """section: an adha_section (see c_section)."""
    check(_lib.load().adha_run_section(ctypes.byref(schema.c), int(n), ctypes.byref(layout.c), _ptrs(bufs),
                                       ctypes.byref(section), None if save is None else save.data_ptr(),
                                       _stream_ptr(stream)), "adha_run_section")


def adha_section_backward(schema, n, layout, state_bufs, grad_bufs, section, save, stream=None):
    check(_lib.load().adha_section_backward(ctypes.byref(schema.c), int(n), ctypes.byref(layout.c),
                                            _ptrs(state_bufs), _ptrs(grad_bufs), ctypes.byref(section),
                                            save.data_ptr(), _stream_ptr(stream)), "adha_section_backward")


def adha_device_status(stream=None):
    v = ctypes.c_int32(0)
    check(_lib.load().adha_device_status(_stream_ptr(stream), ctypes.byref(v)), "adha_device_status")
    return v.value


def remap(schema, n, src_layout, src_bufs, dst_layout, stream=None):
    """Remap into freshly allocated buffers of dst_layout; returns them."""
    dst = alloc_layout(schema, dst_layout, n, device=src_bufs[0].device)
    adha_remap(schema, n, src_layout, src_bufs, dst_layout, dst, stream)
    return dst
