"""Thin Python binding of libadha.so: builds the C structs, passes raw pointers, checks status.

PyTorch provides device memory and streams only; every byte the library moves or computes is
moved or computed by its CUDA kernels.  Function names follow the C ABI (adha_remap, ...).
"""
import ctypes

import torch

from . import _lib
from ._lib import (adha_schema, adha_layout, adha_section, adha_plan_opts, adha_layout_set, adha_cost_table,
                   adha_plan, OPS, check)

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


def c_section(sec, perm=None, aux=None):
    """adha_section from a synth.Section (perm: device int32 tensor for gather sections; aux: device
    tensor with an assign section's centroids or for a reduce section's sums)."""
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
    s.aux = aux.data_ptr() if aux is not None else None
    return s


def adha_remap(schema, n, src_layout, src_bufs, dst_layout, dst_bufs, stream=None):
    check(_lib.load().adha_remap(ctypes.byref(schema.c), int(n), ctypes.byref(src_layout.c), _ptrs(src_bufs),
                                 ctypes.byref(dst_layout.c), _ptrs(dst_bufs), _stream_ptr(stream)), "adha_remap")


def adha_run_section(schema, n, layout, bufs, section, save=None, stream=None):
    """section: an adha_section (see c_section)."""
    check(_lib.load().adha_run_section(ctypes.byref(schema.c), int(n), ctypes.byref(layout.c), _ptrs(bufs),
                                       ctypes.byref(section), None if save is None else save.data_ptr(),
                                       _stream_ptr(stream)), "adha_run_section")


def adha_run_sections_fused(schema, n, layout, bufs, sections, stream=None):
    """sections: a Sections (or list of synth.Section / adha_section) run fused in one pass."""
    secs = sections if isinstance(sections, Sections) else Sections(sections)
    check(_lib.load().adha_run_sections_fused(ctypes.byref(schema.c), int(n), ctypes.byref(layout.c), _ptrs(bufs),
                                              secs.arr, len(secs), _stream_ptr(stream)), "adha_run_sections_fused")


def adha_section_backward(schema, n, layout, state_bufs, grad_bufs, section, save, stream=None):
    check(_lib.load().adha_section_backward(ctypes.byref(schema.c), int(n), ctypes.byref(layout.c),
                                            _ptrs(state_bufs), _ptrs(grad_bufs), ctypes.byref(section),
                                            save.data_ptr(), _stream_ptr(stream)), "adha_section_backward")


def adha_tune_override(chunk_records=0):
    check(_lib.load().adha_tune_override(int(chunk_records)), "adha_tune_override")


def adha_tune_writeback(mode=0):
    check(_lib.load().adha_tune_writeback(int(mode)), "adha_tune_writeback")


def adha_tune_section_buffers(buffers=0):
    check(_lib.load().adha_tune_section_buffers(int(buffers)), "adha_tune_section_buffers")


def adha_tune_fused_jit(mode=0):
    check(_lib.load().adha_tune_fused_jit(int(mode)), "adha_tune_fused_jit")


def adha_tune_section_jit(mode=0):
    check(_lib.load().adha_tune_section_jit(int(mode)), "adha_tune_section_jit")


def adha_tune_fused_buffers(buffers=0):
    check(_lib.load().adha_tune_fused_buffers(int(buffers)), "adha_tune_fused_buffers")


def adha_fused_jit_build(schema, n, layout, sections, chunk_records=0, buffers=0, load=False):
    """The specialised kernel's CUDA source for the fused run `sections` (compiled; loaded into the
    process's cache when `load`, which needs the GPU)."""
    secs = sections if isinstance(sections, Sections) else Sections(sections)
    cap = 1 << 20
    buf = ctypes.create_string_buffer(cap)
    n_src = ctypes.c_size_t(0)
    check(_lib.load().adha_fused_jit_build(ctypes.byref(schema.c), int(n), ctypes.byref(layout.c), secs.arr, len(secs),
                                           int(chunk_records), int(buffers), int(bool(load)), buf, cap,
                                           ctypes.byref(n_src)), "adha_fused_jit_build")
    assert n_src.value < cap, "source longer than the buffer"
    return buf.value.decode()


def adha_jit_available():
    return bool(_lib.load().adha_jit_available())


def adha_jit_log():
    n = ctypes.c_size_t(0)
    check(_lib.load().adha_jit_log(None, 0, ctypes.byref(n)), "adha_jit_log")
    buf = ctypes.create_string_buffer(n.value + 1)
    check(_lib.load().adha_jit_log(buf, n.value + 1, None), "adha_jit_log")
    return buf.value.decode(errors="replace")


def adha_tune_remap_direct(mode=0):
    check(_lib.load().adha_tune_remap_direct(int(mode)), "adha_tune_remap_direct")


def adha_tune_remap_pieces(mode=0):
    check(_lib.load().adha_tune_remap_pieces(int(mode)), "adha_tune_remap_pieces")


def adha_tune_clear():
    check(_lib.load().adha_tune_clear(), "adha_tune_clear")


def adha_tune_export():
    need = ctypes.c_size_t(0)
    check(_lib.load().adha_tune_export(None, 0, ctypes.byref(need)), "adha_tune_export")
    buf = ctypes.create_string_buffer(need.value)
    check(_lib.load().adha_tune_export(buf, need.value, ctypes.byref(need)), "adha_tune_export")
    return buf.value.decode()


def adha_tune_import(text):
    check(_lib.load().adha_tune_import(text.encode()), "adha_tune_import")


def remap(schema, n, src_layout, src_bufs, dst_layout, stream=None):
    """Remap into freshly allocated buffers of dst_layout; returns them."""
    dst = alloc_layout(schema, dst_layout, n, device=src_bufs[0].device)
    adha_remap(schema, n, src_layout, src_bufs, dst_layout, dst, stream)
    return dst


# ------------------------------------------------------------------ planning, measuring, running

class PlanOpts:
    """adha_plan_opts: ODS struct-size limits, window length, candidate cap, return to input, and the
    longest run of sections PDL may fuse (fuse_window <= 1: none)."""

    def __init__(self, caps=(16, 32, 64, 128, 256, 0), max_window=0, include_aos_soa=True, max_candidates=0,
                 return_to_input=False, fuse_window=0):
        self._caps = _i32_array(list(caps))
        self.c = adha_plan_opts(len(caps), self._caps, int(max_window), int(bool(include_aos_soa)),
                                int(max_candidates), int(bool(return_to_input)), int(fuse_window))


class Sections:
    """A contiguous adha_section array (keeps the tensors it points to alive).  An assign section's
    centroids (its synth table) are uploaded to the device; a reduce section gets an int64 device
    tensor of K rows x (features + 1) for its result, in self.outputs[k] (unless aux[k] is given)."""

    def __init__(self, secs, perm=None, aux=None):
        self.src = list(secs)
        self.perm = perm
        self.aux = dict(aux or {})
        self.outputs = {}
        self.arr = (adha_section * len(self.src))()
        for k, s in enumerate(self.src):
            if isinstance(s, adha_section):
                self.arr[k] = s
                continue
            if k not in self.aux and torch.cuda.is_available():
                if s.op == "assign":
                    self.aux[k] = torch.tensor(s.table, dtype=torch.float32, device="cuda")
                elif s.op == "reduce":
                    self.aux[k] = torch.zeros((int(s.args[1]), len(s.read)), dtype=torch.int64, device="cuda")
            if s.op == "reduce" and k in self.aux:
                self.outputs[k] = self.aux[k]
            self.arr[k] = c_section(s, perm, self.aux.get(k))

    def __len__(self):
        return len(self.src)


class LayoutSet:
    """A library-owned adha_layout_set (freed with adha_free)."""

    def __init__(self, ptr):
        self.ptr = ptr

    @property
    def layouts(self):
        s = self.ptr.contents
        F = s.n_fields
        out = []
        for l in range(s.n_layouts):
            groups, p = [], 0
            for g in range(s.n_groups[l]):
                n = s.group_len[l * F + g]
                groups.append([s.fields[l * F + p + j] for j in range(n)])
                p += n
            out.append(Layout(groups))
        return out

    def __len__(self):
        return self.ptr.contents.n_layouts

    def __del__(self):
        if getattr(self, "ptr", None) is not None and _lib._lib is not None:
            _lib._lib.adha_free(ctypes.cast(self.ptr, ctypes.c_void_p))
            self.ptr = None


class CostTable:
    """A library-owned adha_cost_table; section_ns[k][l] and remap_ns[a][b] in nanoseconds."""

    def __init__(self, ptr):
        self.ptr = ptr

    @property
    def section_ns(self):
        t = self.ptr.contents
        return [[t.section_ns[k * t.n_layouts + l] for l in range(t.n_layouts)] for k in range(t.n_sections)]

    @property
    def remap_ns(self):
        t = self.ptr.contents
        L = t.n_layouts + 1
        return [[t.remap_ns[a * L + b] for b in range(L)] for a in range(L)]

    @property
    def max_window(self):
        return self.ptr.contents.max_window

    @property
    def fused_ns(self):
        """{(k, m): [ns per layout]} for the runs of m >= 2 sections starting at k (inf: not fusable)."""
        t = self.ptr.contents
        W, L = t.max_window, t.n_layouts
        out = {}
        for k in range(t.n_sections):
            for m in range(2, W + 1):
                if k + m <= t.n_sections:
                    out[(k, m)] = [t.fused_ns[(k * W + m - 1) * L + l] for l in range(L)]
        return out

    def set(self, section_ns, remap_ns, fused_ns=None):
        t = self.ptr.contents
        for k, row in enumerate(section_ns):
            for l, v in enumerate(row):
                t.section_ns[k * t.n_layouts + l] = float(v)
        for a, row in enumerate(remap_ns):
            for b, v in enumerate(row):
                t.remap_ns[a * (t.n_layouts + 1) + b] = float(v)
        for (k, m), row in (fused_ns or {}).items():
            for l, v in enumerate(row):
                t.fused_ns[(k * t.max_window + m - 1) * t.n_layouts + l] = float(v)

    def __del__(self):
        if getattr(self, "ptr", None) is not None and _lib._lib is not None:
            _lib._lib.adha_free(ctypes.cast(self.ptr, ctypes.c_void_p))
            self.ptr = None


def adha_ods(schema, sections, cap_bytes=0):
    secs = sections if isinstance(sections, Sections) else Sections(sections)
    ng = ctypes.c_int32(0)
    gl = (ctypes.c_int32 * schema.F)()
    fl = (ctypes.c_int32 * schema.F)()
    check(_lib.load().adha_ods(ctypes.byref(schema.c), secs.arr, len(secs), int(cap_bytes), ctypes.byref(ng), gl, fl),
          "adha_ods")
    groups, p = [], 0
    for g in range(ng.value):
        groups.append([fl[p + j] for j in range(gl[g])])
        p += gl[g]
    return Layout(groups)


def adha_plan_sections(schema, sections, opts=None):
    secs = sections if isinstance(sections, Sections) else Sections(sections)
    opts = opts or PlanOpts()
    out = ctypes.POINTER(adha_layout_set)()
    check(_lib.load().adha_plan_sections(ctypes.byref(schema.c), secs.arr, len(secs), ctypes.byref(opts.c),
                                         ctypes.byref(out)), "adha_plan_sections")
    return LayoutSet(out)


def adha_layout_set_create(F, layouts):
    arr = (adha_layout * len(layouts))(*[l.c for l in layouts])
    out = ctypes.POINTER(adha_layout_set)()
    check(_lib.load().adha_layout_set_create(F, len(layouts), arr, ctypes.byref(out)), "adha_layout_set_create")
    return LayoutSet(out)


def adha_cost_table_create(n_sections, n_layouts, max_window=0):
    out = ctypes.POINTER(adha_cost_table)()
    check(_lib.load().adha_cost_table_create_fused(n_sections, n_layouts, int(max_window), ctypes.byref(out)),
          "adha_cost_table_create_fused")
    return CostTable(out)


def adha_pdl_solve(costs, return_to_input=False):
    S = costs.ptr.contents.n_sections
    seq = (ctypes.c_int32 * S)()
    tot = ctypes.c_double(0)
    check(_lib.load().adha_pdl_solve(costs.ptr, int(bool(return_to_input)), seq, ctypes.byref(tot)), "adha_pdl_solve")
    return tot.value, list(seq)


def adha_pdl_solve_fused(costs, return_to_input=False, max_window=0):
    """(total ns, layout per section, window length per section: the run length at its first section, 0 inside)."""
    S = costs.ptr.contents.n_sections
    seq = (ctypes.c_int32 * S)()
    win = (ctypes.c_int32 * S)()
    tot = ctypes.c_double(0)
    check(_lib.load().adha_pdl_solve_fused(costs.ptr, int(bool(return_to_input)), int(max_window), seq, win,
                                           ctypes.byref(tot)), "adha_pdl_solve_fused")
    return tot.value, list(seq), list(win)


def adha_pdl_solve_devices(tables, transfer_ns, input_device=0, return_to_input=False):
    """PDL over (layout, device): tables = one CostTable per device, transfer_ns[a][b][l] the time to
    move layout l (l = n_layouts: the input layout) from device a to device b.  Returns (total ns,
    [(layout, device)] per section)."""
    D = len(tables)
    S, L = tables[0].ptr.contents.n_sections, tables[0].ptr.contents.n_layouts
    arr = (ctypes.POINTER(adha_cost_table) * D)(*[t.ptr for t in tables])
    flat = [float(transfer_ns[a][b][l]) for a in range(D) for b in range(D) for l in range(L + 1)]
    xf = (ctypes.c_double * len(flat))(*flat)
    lay, dev = (ctypes.c_int32 * S)(), (ctypes.c_int32 * S)()
    tot = ctypes.c_double(0)
    check(_lib.load().adha_pdl_solve_devices(D, arr, xf, int(input_device), int(bool(return_to_input)), lay, dev,
                                             ctypes.byref(tot)), "adha_pdl_solve_devices")
    return tot.value, [(lay[k], dev[k]) for k in range(S)]


SCFG_KINDS = {"sec": 0, "seq": 1, "branch": 2, "loop": 3}


def adha_pdl_solve_scfg(costs, tree, return_to_input=False):
    """PDL over a region tree of nested lists: ["sec", k], ["seq", [regions]],
    ["branch", [regions], [weights]], ["loop", region, trips].  Returns (expected cost,
    {id(region): layout}) with a layout for every section, merge point and loop header."""
    order = []

    def walk(t):
        order.append(t)
        kids = t[1] if t[0] in ("seq", "branch") else ([t[1]] if t[0] == "loop" else [])
        for c in kids:
            walk(c)
    walk(tree)
    index = {id(t): i for i, t in enumerate(order)}
    keep = []
    nodes = (_lib.adha_scfg_node * len(order))()
    for i, t in enumerate(order):
        kids = t[1] if t[0] in ("seq", "branch") else ([t[1]] if t[0] == "loop" else [])
        ch = _i32_array([index[id(c)] for c in kids])
        w = (ctypes.c_double * max(1, len(kids)))(*(t[2] if t[0] == "branch" else []))
        keep += [ch, w]
        nodes[i] = _lib.adha_scfg_node(SCFG_KINDS[t[0]], int(t[1]) if t[0] == "sec" else 0, len(kids), ch, w,
                                       float(t[2]) if t[0] == "loop" else 0.0)
    lay = (ctypes.c_int32 * len(order))()
    tot = ctypes.c_double(0)
    check(_lib.load().adha_pdl_solve_scfg(costs.ptr, len(order), nodes, 0, int(bool(return_to_input)), lay,
                                          ctypes.byref(tot)), "adha_pdl_solve_scfg")
    return tot.value, {id(t): lay[i] for i, t in enumerate(order) if t[0] != "seq"}


def adha_measure_workspace_bytes(schema, n, in_layout, candidates, flags=0):
    return _lib.load().adha_measure_workspace_bytes_for(ctypes.byref(schema.c), int(n), ctypes.byref(in_layout.c),
                                                        candidates.ptr, int(flags))


ADHA_MEASURE_AUTOTUNE = 1
ADHA_MEASURE_DIFFERENTIABLE = 2


def adha_measure(schema, n, in_layout, in_bufs, sections, candidates, reps=2, workspace=None, stream=None,
                 autotune=False, fuse_window=0, differentiable=False):
    """Cost table of every section in every candidate and every remap between candidates (and, with
    fuse_window >= 2, of every run of 2..fuse_window sections that may be fused; with differentiable,
    of a forward + backward step)."""
    secs = sections if isinstance(sections, Sections) else Sections(sections)
    flags = ((ADHA_MEASURE_AUTOTUNE if autotune else 0) | (ADHA_MEASURE_DIFFERENTIABLE if differentiable else 0)
             | (int(fuse_window) << 8))
    need = adha_measure_workspace_bytes(schema, n, in_layout, candidates, flags)
    ws = workspace if workspace is not None else torch.empty(need, dtype=torch.uint8, device=in_bufs[0].device)
    out = ctypes.POINTER(adha_cost_table)()
    check(_lib.load().adha_measure(ctypes.byref(schema.c), int(n), ctypes.byref(in_layout.c), _ptrs(in_bufs),
                                   secs.arr, len(secs), candidates.ptr, int(reps), flags,
                                   ws.data_ptr(), ws.numel(),
                                   _stream_ptr(stream), ctypes.byref(out)), "adha_measure")
    return CostTable(out)


def adha_program_workspace_bytes(schema, n, in_layout, candidates):
    return _lib.load().adha_program_workspace_bytes(ctypes.byref(schema.c), int(n), ctypes.byref(in_layout.c),
                                                    candidates.ptr)


def _fix_plan(plan, fixed, windows):
    plan.fixed = 0
    if fixed is not None:
        plan.fixed = 1
        for k, l in enumerate(fixed):
            plan.layout_of_section[k] = int(l)
        for k in range(len(fixed)):
            plan.window_len[k] = int(windows[k]) if windows is not None else 0


def adha_run_program(schema, n, in_layout, in_bufs, sections, candidates, costs=None, opts=None, workspace=None,
                     fixed=None, stream=None, plan=None, windows=None):
    """Runs the program; returns the adha_plan (layout per section, fused windows, final buffers'
    pointers).  fixed: a layout per section; windows: with fixed, the run length at each run's
    first section and 0 inside (None: every section alone)."""
    secs = sections if isinstance(sections, Sections) else Sections(sections)
    opts = opts or PlanOpts()
    if plan is None:
        plan = adha_plan()
    _fix_plan(plan, fixed, windows)
    check(_lib.load().adha_run_program(ctypes.byref(schema.c), int(n), ctypes.byref(in_layout.c), _ptrs(in_bufs),
                                       secs.arr, len(secs), candidates.ptr, costs.ptr if costs is not None else None,
                                       ctypes.byref(opts.c), workspace.data_ptr() if workspace is not None else None,
                                       workspace.numel() if workspace is not None else 0, _stream_ptr(stream),
                                       ctypes.byref(plan)), "adha_run_program")
    return plan


def adha_program_host_workspace_bytes(schema, n, in_layout, candidates, n_slices):
    return _lib.load().adha_program_host_workspace_bytes(ctypes.byref(schema.c), int(n), ctypes.byref(in_layout.c),
                                                         candidates.ptr, int(n_slices))


def adha_run_program_host(schema, n, in_layout, host_in, sections, candidates, host_out, costs=None, opts=None,
                          workspace=None, n_slices=8, fixed=None, stream=None, plan=None, windows=None):
    """Runs the program on host buffers (pinned CPU tensors), writing the result into host_out
    (CPU tensors in the plan's final layout); returns the adha_plan."""
    secs = sections if isinstance(sections, Sections) else Sections(sections)
    opts = opts or PlanOpts()
    if plan is None:
        plan = adha_plan()
    _fix_plan(plan, fixed, windows)
    check(_lib.load().adha_run_program_host(ctypes.byref(schema.c), int(n), ctypes.byref(in_layout.c), _ptrs(host_in),
                                            secs.arr, len(secs), candidates.ptr,
                                            costs.ptr if costs is not None else None, ctypes.byref(opts.c),
                                            _ptrs(host_out), int(n_slices), workspace.data_ptr(), workspace.numel(),
                                            _stream_ptr(stream), ctypes.byref(plan)), "adha_run_program_host")
    return plan


def final_buffers(plan, schema, n, candidates, in_layout, workspace_views=None):
    """(layout, list of uint8 device tensors viewing the result's groups) of a finished program."""
    layouts = candidates.layouts
    lay = layouts[plan.final_layout] if plan.final_layout >= 0 else in_layout
    strides, _ = adha_layout_strides(schema, lay)
    out = []
    for g, st in enumerate(strides):
        out.append(_view_device(plan.final_ptrs[g], n * st))
    return lay, out


def _view_device(ptr, nbytes):
    """A uint8 CUDA tensor aliasing nbytes at ptr (memory owned elsewhere)."""
    class _Cuda:
        __cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                    "version": 3, "strides": None}
    return torch.as_tensor(_Cuda(), device="cuda")


KINDS = {0: "remap", 1: "section", 2: "section_backward", 3: "batched_remap", 4: "fused", 5: "gather_probe",
         6: "section_specialised"}


def adha_gather_probe(table, perm, out, rec_bytes=16, stream=None):
    """out[i] = table[perm[i]] for every i (device tensors; elements of rec_bytes bytes)."""
    n = perm.numel()
    check(_lib.load().adha_gather_probe(table.data_ptr(), perm.data_ptr(), out.data_ptr(), int(n), int(rec_bytes),
                                        _stream_ptr(stream)), "adha_gather_probe")
OP_NAMES = {v: k for k, v in OPS.items()}


def adha_profile_start(max_records=4096):
    check(_lib.load().adha_profile_start(int(max_records)), "adha_profile_start")


def adha_profile_stop(max_records=4096):
    """List of dicts (kind, op, bytes, ms) of the launches recorded since adha_profile_start."""
    recs = (_lib.adha_launch_record * max_records)()
    n = ctypes.c_int32(0)
    check(_lib.load().adha_profile_stop(recs, max_records, ctypes.byref(n)), "adha_profile_stop")
    return [dict(kind=KINDS.get(recs[k].kind, recs[k].kind),
                 op=recs[k].op if recs[k].kind in (4, 5) else OP_NAMES.get(recs[k].op, recs[k].op),
                 bytes=recs[k].bytes, ms=recs[k].ms) for k in range(min(n.value, max_records))]


# ------------------------------------------------------------------ batched remap

ADHA_BATCHED_AUTOTUNE = 1
ADHA_BATCHED_TWO_BUFFERS = 2


def remap_descs(arrays):
    """(adha_remap_desc array, objects to keep alive) for a list of array dicts with keys schema,
    n, src, src_bufs, dst, dst_bufs."""
    keep = []
    descs = (_lib.adha_remap_desc * max(1, len(arrays)))()
    for k, a in enumerate(arrays):
        sp, dp = _ptrs(a["src_bufs"]), _ptrs(a["dst_bufs"])
        keep += [a["schema"], a["src"], a["dst"], sp, dp]
        descs[k] = _lib.adha_remap_desc(ctypes.pointer(a["schema"].c), int(a["n"]), ctypes.pointer(a["src"].c),
                                        sp, ctypes.pointer(a["dst"].c), dp)
    return descs, keep


def adha_workspace_bytes(arrays):
    """Device workspace bytes adha_remap_batched needs for these arrays."""
    descs, _keep = remap_descs(arrays)
    out = ctypes.c_size_t(0)
    check(_lib.load().adha_workspace_bytes(len(arrays), descs, ctypes.byref(out)), "adha_workspace_bytes")
    return out.value


def adha_remap_batched(arrays, workspace, stream=None):
    """All arrays remapped in one persistent launch, descriptors placed in `workspace` (a device
    uint8 tensor of at least adha_workspace_bytes(arrays) bytes)."""
    descs, _keep = remap_descs(arrays)
    check(_lib.load().adha_remap_batched(len(arrays), descs, workspace.data_ptr(), workspace.numel(),
                                         _stream_ptr(stream)), "adha_remap_batched")


class Batched:
    """A prepared batched remap (adha_batched_create); arrays: list of dicts with keys
    schema (Schema), n, src (Layout), src_bufs, dst (Layout), dst_bufs.  ctas: force that many
    CTAs per SM (1..8; 0 = the library's choice); buffers: input chunk buffers per warp (1 or 2)."""

    def __init__(self, arrays, autotune=False, stream=None, ctas=0, buffers=1):
        descs, self._keep = remap_descs(arrays)
        self.ptr = ctypes.c_void_p()
        flags = ((ADHA_BATCHED_AUTOTUNE if autotune else 0) | (ADHA_BATCHED_TWO_BUFFERS if buffers == 2 else 0)
                 | (int(ctas) << 4))
        check(_lib.load().adha_batched_create(len(arrays), descs, flags, _stream_ptr(stream), ctypes.byref(self.ptr)),
              "adha_batched_create")
        self.workspace = None

    @property
    def info(self):
        """(CTAs per SM, shared bytes per warp, work units per launch) the plan chose."""
        k, r, u = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
        check(_lib.load().adha_batched_info(self.ptr, ctypes.byref(k), ctypes.byref(r), ctypes.byref(u)),
              "adha_batched_info")
        return k.value, r.value, u.value

    @property
    def workspace_bytes(self):
        return _lib.load().adha_batched_workspace_bytes(self.ptr)

    @property
    def bytes(self):
        return _lib.load().adha_batched_bytes(self.ptr)

    def upload(self, workspace=None, stream=None):
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        check(_lib.load().adha_batched_upload(self.ptr, workspace.data_ptr(), workspace.numel(), _stream_ptr(stream)),
              "adha_batched_upload")
        return workspace

    def launch(self, stream=None):
        check(_lib.load().adha_batched_launch(self.ptr, self.workspace.data_ptr(), _stream_ptr(stream)),
              "adha_batched_launch")

    def capture(self, stream=None):
        check(_lib.load().adha_batched_graph(self.ptr, self.workspace.data_ptr(), _stream_ptr(stream)),
              "adha_batched_graph")

    def graph_launch(self, stream=None):
        check(_lib.load().adha_batched_graph_launch(self.ptr, _stream_ptr(stream)), "adha_batched_graph_launch")

    def __del__(self):
        if getattr(self, "ptr", None) and _lib._lib is not None:
            _lib._lib.adha_batched_destroy(self.ptr)
            self.ptr = None
