"""ctypes front end of adha_oracle.c (TEST INFRASTRUCTURE ONLY; see the package docstring)."""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adha_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SIZE = {0: 4, 1: 8, 2: 4, 3: 2}
NP = {0: np.float32, 1: np.float64, 2: np.int32, 3: np.uint16}
OPS = dict(madd3=1, xorshift=2, add=3, mix=4, drift=5, bin=6, ke=7, flags=8, gather=9, kick=10,
           axpb=11, mul=12, tanh=13, assign=14, reduce=15)

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64


def build(force=False):
    """Compile liboracle.so (plain C, no FMA contraction, no fast math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_group_layout.argtypes = [_P, _P, _I, _P]
            lib.oracle_layout_info.argtypes = [_I, _P, _I, _P, _P, _P, _P, _P]
            lib.oracle_remap.argtypes = [_I64, _I, _P, _I, _P, _P, _P, _I, _P, _P, _P]
            lib.oracle_tanhf.restype = ctypes.c_float
            lib.oracle_tanhf.argtypes = [ctypes.c_float]
            lib.oracle_tanhf_n.argtypes = [_P, _P, _I64]
            lib.oracle_tanh_coeffs.argtypes = [_P, _P]
            lib.oracle_section.argtypes = [_I, _P, _P, ctypes.c_uint64, ctypes.c_uint64, _I, _P, _P, _I64, _P]
            lib.oracle_chain_grad.argtypes = [_I, _P, _P, _P, _I, _P, _P, _P, _I64]
            lib.oracle_kmeans_assign.argtypes = [_I, _P, _I, _I, _P, _P, _I64]
            lib.oracle_kmeans_reduce.argtypes = [_I, _P, _I, _I, _P, _I64, _P]
            lib.oracle_section_range.argtypes = [_I, _P, _P, ctypes.c_uint64, ctypes.c_uint64, _I, _P, _P, _I64,
                                                 _I64, _P]
            lib.oracle_kmeans_assign_range.argtypes = [_I, _P, _I, _I, _P, _P, _I64, _I64]
            lib.oracle_kmeans_reduce_range.argtypes = [_I, _P, _I, _I, _P, _I64, _I64, _P]
            _lib = lib
    return _lib


def _i32(xs):
    return np.ascontiguousarray(np.asarray(xs, dtype=np.int32))


def aos(F):
    return [list(range(F))]


def soa(F):
    return [[f] for f in range(F)]


def canon(groups):
    """Canonical form of a grouping: fields ascending in a group, groups ordered by their first field."""
    return sorted((sorted(g) for g in groups), key=lambda g: g[0])


def group_layout(dtypes, fields):
    """(offsets, struct size) of one group: natural alignment, size rounded to the largest alignment."""
    f = _i32(fields)
    off = np.zeros(len(fields), dtype=np.int32)
    s = _get().oracle_group_layout(_i32(dtypes).ctypes.data, f.ctypes.data, len(fields), off.ctypes.data)
    return off.tolist(), int(s)


def layout_info(dtypes, groups):
    """(strides per group, group of each field, offset of each field) of a layout."""
    F = len(dtypes)
    lens = _i32([len(g) for g in groups])
    flat = _i32([f for g in groups for f in g])
    stride = np.zeros(len(groups), dtype=np.int32)
    gof = np.zeros(F, dtype=np.int32)
    oof = np.zeros(F, dtype=np.int32)
    d = _i32(dtypes)
    rc = _get().oracle_layout_info(F, d.ctypes.data, len(groups), lens.ctypes.data, flat.ctypes.data,
                                   stride.ctypes.data, gof.ctypes.data, oof.ctypes.data)
    if rc != 0:
        raise ValueError("not a layout of %d fields: %r" % (F, groups))
    return stride.tolist(), gof.tolist(), oof.tolist()


def _ptrs(bufs):
    arr = (ctypes.c_void_p * max(1, len(bufs)))()
    for k, b in enumerate(bufs):
        assert b.flags.c_contiguous
        arr[k] = b.ctypes.data
    return arr


def remap(n, dtypes, src_groups, src_bufs, dst_groups):
    """Byte remap of n records from src_groups (buffers src_bufs) to new buffers in dst_groups."""
    F = len(dtypes)
    d_stride, _, _ = layout_info(dtypes, dst_groups)
    dst = [np.empty(n * s, dtype=np.uint8) for s in d_stride]
    sl, sf = _i32([len(g) for g in src_groups]), _i32([f for g in src_groups for f in g])
    dl, df = _i32([len(g) for g in dst_groups]), _i32([f for g in dst_groups for f in g])
    srcb = [np.ascontiguousarray(b).view(np.uint8).reshape(-1) for b in src_bufs]
    rc = _get().oracle_remap(n, F, _i32(dtypes).ctypes.data, len(src_groups), sl.ctypes.data, sf.ctypes.data,
                             _ptrs(srcb), len(dst_groups), dl.ctypes.data, df.ctypes.data, _ptrs(dst))
    if rc != 0:
        raise ValueError("bad layout")
    return dst


def to_fields(n, dtypes, groups, bufs):
    """Decode a layout's group buffers into one numpy array per field (via a remap to SoA)."""
    F = len(dtypes)
    out = remap(n, dtypes, groups, bufs, soa(F))
    return [out[f].view(NP[dtypes[f]]) for f in range(F)]


def from_fields(n, dtypes, groups, fields):
    """Encode field arrays into the group buffers of a layout (via a remap from SoA)."""
    F = len(dtypes)
    src = [np.ascontiguousarray(fields[f], dtype=NP[dtypes[f]]).view(np.uint8) for f in range(F)]
    return remap(n, dtypes, soa(F), src, groups)


def tanhf(x):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    y = np.empty_like(x)
    _get().oracle_tanhf_n(x.ctypes.data, y.ctypes.data, x.size)
    return y


def tanh_coeffs():
    p = np.zeros(13, dtype=np.float32)
    q = np.zeros(13, dtype=np.float32)
    k = _get().oracle_tanh_coeffs(p.ctypes.data, q.ctypes.data)
    return k, p, q


def _mask(s):
    m = 0
    for f in s:
        m |= 1 << f
    return m


def kmeans_features(sec, dtypes):
    """(feature field ids ascending, membership field, K) of an assign or reduce section: the
    features are its fp32 read fields; args = (membership field, K)."""
    feats = sorted(f for f in sec.read if dtypes[f] == 0)
    return feats, int(sec.args[0]), int(sec.args[1])


def kmeans_assign(sec, dtypes, fields):
    """The assign section in place (membership field written); centroids from sec.table, K x d."""
    feats, mf, K = kmeans_features(sec, dtypes)
    n = fields[0].shape[0]
    cent = np.ascontiguousarray(np.asarray(sec.table, dtype=np.float32))
    assert cent.size == K * len(feats)
    rc = _get().oracle_kmeans_assign(len(feats), _i32(feats).ctypes.data, mf, K, cent.ctypes.data, _ptrs(fields), n)
    if rc != 0:
        raise ValueError("bad assign section")


def kmeans_reduce(sec, dtypes, fields):
    """The reduce section: int64 array of K rows [count, fixed-point sum of each feature]."""
    feats, mf, K = kmeans_features(sec, dtypes)
    n = fields[0].shape[0]
    out = np.zeros((K, len(feats) + 1), dtype=np.int64)
    rc = _get().oracle_kmeans_reduce(len(feats), _i32(feats).ctypes.data, mf, K, _ptrs(fields), n, out.ctypes.data)
    if rc != 0:
        raise ValueError("bad reduce section")
    return out


def section(sec, dtypes, fields, perm=None):
    """Run one section (a synth.Section) in place on field arrays (list of numpy arrays); a reduce
    section returns its sums (kmeans_reduce) and changes no field."""
    if sec.op == "assign":
        return kmeans_assign(sec, dtypes, fields)
    if sec.op == "reduce":
        return kmeans_reduce(sec, dtypes, fields)
    n = fields[0].shape[0]
    args = _i32(list(sec.args) + [0] * (8 - len(sec.args)))
    par = np.ascontiguousarray(np.asarray(list(sec.params) + [0.0] * (4 - len(sec.params)), dtype=np.float32))
    for a in fields:
        assert a.flags.c_contiguous and a.shape[0] == n
    pp = None
    if sec.op == "gather":
        pp = np.ascontiguousarray(perm, dtype=np.int32)
        assert pp.shape[0] == n and (n == 0 or (pp.min() >= 0 and pp.max() < n))
        pp = pp.ctypes.data
    rc = _get().oracle_section(OPS[sec.op], args.ctypes.data, par.ctypes.data, _mask(sec.read),
                               _mask(sec.write), len(dtypes), _i32(dtypes).ctypes.data, _ptrs(fields), n, pp)
    if rc != 0:
        raise ValueError("unknown op %r" % sec.op)


def chain_grad(sections, fields, c):
    """Final state (in place in `fields`, fp32 arrays) and dL/d(input) of an axpb/mul/tanh chain."""
    n = fields[0].shape[0]
    F = len(fields)
    ops = _i32([OPS[s.op] for s in sections])
    args = []
    par = []
    for s in sections:
        if s.op == "mul":
            args += [s.args[0], s.args[1], s.args[2]]
        else:
            args += [s.args[0], 0, s.args[1]]
        par += list(s.params) if s.op == "axpb" else [0.0, 0.0]
    args = _i32(args)
    par = np.ascontiguousarray(np.asarray(par, dtype=np.float32))
    cc = np.ascontiguousarray(np.asarray(c, dtype=np.float32))
    grads = [np.empty(n, dtype=np.float32) for _ in range(F)]
    rc = _get().oracle_chain_grad(len(sections), ops.ctypes.data, args.ctypes.data, par.ctypes.data, F,
                                  _ptrs(fields), cc.ctypes.data, _ptrs(grads), n)
    if rc != 0:
        raise ValueError("chain_grad failed")
    return grads


def chain_grad_threads(sections, fields, c, threads=1):
    """chain_grad() split over `threads` host threads by record range: every record's forward and
    reverse pass is independent of the others, so each range runs the same per-record code on
    slices of the arrays (bit-identical to one call; ctypes releases the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor
    n = fields[0].shape[0]
    for a in fields:
        assert a.flags.c_contiguous and a.shape[0] == n and a.dtype == np.float32
    F = len(fields)
    ops = _i32([OPS[s.op] for s in sections])
    args, par = [], []
    for s in sections:
        args += [s.args[0], s.args[1], s.args[2]] if s.op == "mul" else [s.args[0], 0, s.args[1]]
        par += list(s.params) if s.op == "axpb" else [0.0, 0.0]
    args = _i32(args)
    par = np.ascontiguousarray(np.asarray(par, dtype=np.float32))
    cc = np.ascontiguousarray(np.asarray(c, dtype=np.float32))
    grads = [np.empty(n, dtype=np.float32) for _ in range(F)]
    lib = _get()

    def work(r):
        i0, i1 = r
        return lib.oracle_chain_grad(len(sections), ops.ctypes.data, args.ctypes.data, par.ctypes.data, F,
                                     _ptrs([a[i0:i1] for a in fields]), cc.ctypes.data,
                                     _ptrs([g[i0:i1] for g in grads]), i1 - i0)
    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        if any(ex.map(work, _ranges(n, threads))):
            raise ValueError("chain_grad failed")
    return grads


def _ranges(n, threads):
    step = (n + threads - 1) // max(1, threads)
    return [(i0, min(n, i0 + step)) for i0 in range(0, n, max(1, step))]


def section_threads(sec, dtypes, fields, perm=None, threads=1):
    """section() split over `threads` host threads by record range (the per-record code is the
    same, so the result is bit-identical; ctypes releases the interpreter lock during each call).
    A reduce section's partial sums of the ranges are added (exact: integers)."""
    from concurrent.futures import ThreadPoolExecutor
    n = fields[0].shape[0]
    for a in fields:
        assert a.flags.c_contiguous and a.shape[0] == n
    fa = _ptrs(fields)
    dt = _i32(dtypes)
    lib = _get()
    if sec.op in ("assign", "reduce"):
        feats, mf, K = kmeans_features(sec, dtypes)
        fe = _i32(feats)
        if sec.op == "assign":
            cent = np.ascontiguousarray(np.asarray(sec.table, dtype=np.float32))
            work = lambda r: lib.oracle_kmeans_assign_range(len(feats), fe.ctypes.data, mf, K, cent.ctypes.data, fa,
                                                            r[0], r[1])
        else:
            parts = []

            def work(r):
                out = np.zeros((K, len(feats) + 1), dtype=np.int64)
                rc = lib.oracle_kmeans_reduce_range(len(feats), fe.ctypes.data, mf, K, fa, r[0], r[1], out.ctypes.data)
                parts.append(out)
                return rc
    else:
        args = _i32(list(sec.args) + [0] * (8 - len(sec.args)))
        par = np.ascontiguousarray(np.asarray(list(sec.params) + [0.0] * (4 - len(sec.params)), dtype=np.float32))
        pp = np.ascontiguousarray(perm, dtype=np.int32).ctypes.data if sec.op == "gather" else None
        work = lambda r: lib.oracle_section_range(OPS[sec.op], args.ctypes.data, par.ctypes.data, _mask(sec.read),
                                                  _mask(sec.write), len(dtypes), dt.ctypes.data, fa, r[0], r[1], pp)
    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        rcs = list(ex.map(work, _ranges(n, threads)))
    if any(rcs):
        raise ValueError("oracle section %r failed" % sec.op)
    if sec.op == "reduce":
        return sum(parts) if parts else np.zeros((kmeans_features(sec, dtypes)[2], 1), dtype=np.int64)
    return None


def remap_threads(n, dtypes, src_groups, src_bufs, dst_groups, threads=1):
    """remap() split over host threads by record range (each range a slice of every buffer)."""
    from concurrent.futures import ThreadPoolExecutor
    s_stride, _, _ = layout_info(dtypes, src_groups)
    d_stride, _, _ = layout_info(dtypes, dst_groups)
    dst = [np.empty(n * st, dtype=np.uint8) for st in d_stride]
    srcb = [np.ascontiguousarray(b).view(np.uint8).reshape(-1) for b in src_bufs]
    F = len(dtypes)
    sl, sf = _i32([len(g) for g in src_groups]), _i32([f for g in src_groups for f in g])
    dl, df = _i32([len(g) for g in dst_groups]), _i32([f for g in dst_groups for f in g])
    dt = _i32(dtypes)
    lib = _get()

    def work(r):
        i0, i1 = r
        sp = _ptrs([b[i0 * st:i1 * st] for b, st in zip(srcb, s_stride)])
        dp = _ptrs([b[i0 * st:i1 * st] for b, st in zip(dst, d_stride)])
        return lib.oracle_remap(i1 - i0, F, dt.ctypes.data, len(src_groups), sl.ctypes.data, sf.ctypes.data, sp,
                                len(dst_groups), dl.ctypes.data, df.ctypes.data, dp)
    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        if any(ex.map(work, _ranges(n, threads))):
            raise ValueError("bad layout")
    return dst
