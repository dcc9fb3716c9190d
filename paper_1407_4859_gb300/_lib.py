"""ctypes declarations of libadha.so (include/adha.h).  Loading fails loudly if the library is missing."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libadha.so")

ADHA_OK, ADHA_EINVAL, ADHA_ENOMEM, ADHA_ECUDA, ADHA_ETIMEOUT, ADHA_ENOTIMPL = 0, -1, -2, -3, -4, -5
CODES = {-1: "ADHA_EINVAL", -2: "ADHA_ENOMEM", -3: "ADHA_ECUDA", -4: "ADHA_ETIMEOUT", -5: "ADHA_ENOTIMPL"}
OPS = dict(madd3=1, xorshift=2, add=3, mix=4, drift=5, bin=6, ke=7, flags=8, gather=9, kick=10,
           axpb=11, mul=12, tanh=13, assign=14, reduce=15)

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_PP = ctypes.POINTER(ctypes.c_void_p)


class adha_schema(ctypes.Structure):
    _fields_ = [("n_fields", _I32), ("dtype", ctypes.POINTER(_I32))]


class adha_layout(ctypes.Structure):
    _fields_ = [("n_groups", _I32), ("group_len", ctypes.POINTER(_I32)), ("fields", ctypes.POINTER(_I32))]


class adha_section(ctypes.Structure):
    _fields_ = [("op", _I32), ("arg", _I32 * 8), ("fparam", ctypes.c_float * 4), ("read_mask", ctypes.c_uint64),
                ("write_mask", ctypes.c_uint64), ("read_at_perm_mask", ctypes.c_uint64), ("perm", _P), ("aux", _P)]


class adha_plan_opts(ctypes.Structure):
    _fields_ = [("n_caps", _I32), ("caps", ctypes.POINTER(_I32)), ("max_window", _I32), ("include_aos_soa", _I32),
                ("max_candidates", _I32), ("return_to_input", _I32), ("fuse_window", _I32)]


class adha_layout_set(ctypes.Structure):
    _fields_ = [("n_fields", _I32), ("n_layouts", _I32), ("n_groups", ctypes.POINTER(_I32)),
                ("group_len", ctypes.POINTER(_I32)), ("fields", ctypes.POINTER(_I32))]


class adha_cost_table(ctypes.Structure):
    _fields_ = [("n_sections", _I32), ("n_layouts", _I32), ("section_ns", ctypes.POINTER(ctypes.c_double)),
                ("remap_ns", ctypes.POINTER(ctypes.c_double)), ("max_window", _I32),
                ("fused_ns", ctypes.POINTER(ctypes.c_double))]


MAX_SECTIONS = 256
MAX_FIELDS = 64
MAX_FUSED = 16


class adha_plan(ctypes.Structure):
    _fields_ = [("fixed", _I32), ("n_sections", _I32), ("layout_of_section", _I32 * MAX_SECTIONS),
                ("model_ns", ctypes.c_double), ("n_remaps", _I32), ("n_launches", _I32), ("final_layout", _I32),
                ("final_n_groups", _I32), ("final_ptrs", _P * MAX_FIELDS), ("window_len", _I32 * MAX_SECTIONS)]


class adha_launch_record(ctypes.Structure):
    _fields_ = [("kind", _I32), ("op", _I32), ("bytes", ctypes.c_double), ("ms", ctypes.c_double)]


class adha_remap_desc(ctypes.Structure):
    _fields_ = [("schema", ctypes.POINTER(adha_schema)), ("n", _I64), ("src", ctypes.POINTER(adha_layout)),
                ("src_ptrs", _PP), ("dst", ctypes.POINTER(adha_layout)), ("dst_ptrs", _PP)]


class adha_scfg_node(ctypes.Structure):
    _fields_ = [("kind", _I32), ("section", _I32), ("n_children", _I32), ("children", ctypes.POINTER(_I32)),
                ("weights", ctypes.POINTER(ctypes.c_double)), ("trips", ctypes.c_double)]


class AdhaError(RuntimeError):
    def __init__(self, code, fn, msg):
        super().__init__("%s failed with %s: %s" % (fn, CODES.get(code, code), msg))
        self.code = code


_lib = None

# name -> (restype, argtypes)
SIGNATURES = {
    "adha_version": (ctypes.c_char_p, []),
    "adha_last_error": (ctypes.c_char_p, []),
    "adha_free": (None, [_P]),
    "adha_layout_strides": (ctypes.c_int, [ctypes.POINTER(adha_schema), ctypes.POINTER(adha_layout),
                                           ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "adha_remap": (ctypes.c_int, [ctypes.POINTER(adha_schema), _I64, ctypes.POINTER(adha_layout), _PP,
                                  ctypes.POINTER(adha_layout), _PP, _P]),
    "adha_run_section": (ctypes.c_int, [ctypes.POINTER(adha_schema), _I64, ctypes.POINTER(adha_layout), _PP,
                                        ctypes.POINTER(adha_section), _P, _P]),
    "adha_run_sections_fused": (ctypes.c_int, [ctypes.POINTER(adha_schema), _I64, ctypes.POINTER(adha_layout), _PP,
                                               ctypes.POINTER(adha_section), _I32, _P]),
    "adha_section_backward": (ctypes.c_int, [ctypes.POINTER(adha_schema), _I64, ctypes.POINTER(adha_layout), _PP,
                                             _PP, ctypes.POINTER(adha_section), _P, _P]),
    "adha_tune_override": (ctypes.c_int, [_I32]),
    "adha_batched_create": (ctypes.c_int, [_I32, ctypes.POINTER(adha_remap_desc), _I32, _P, ctypes.POINTER(_P)]),
    "adha_batched_workspace_bytes": (ctypes.c_size_t, [_P]),
    "adha_batched_upload": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "adha_batched_launch": (ctypes.c_int, [_P, _P, _P]),
    "adha_batched_graph": (ctypes.c_int, [_P, _P, _P]),
    "adha_batched_graph_launch": (ctypes.c_int, [_P, _P]),
    "adha_batched_bytes": (ctypes.c_double, [_P]),
    "adha_batched_destroy": (None, [_P]),
    "adha_remap_batched_noalloc": (ctypes.c_int, [_I32, ctypes.POINTER(adha_remap_desc), _P]),
    "adha_remap_batched": (ctypes.c_int, [_I32, ctypes.POINTER(adha_remap_desc), _P, ctypes.c_size_t, _P]),
    "adha_workspace_bytes": (ctypes.c_int, [_I32, ctypes.POINTER(adha_remap_desc), ctypes.POINTER(ctypes.c_size_t)]),
    "adha_batched_info": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
    "adha_gather_probe": (ctypes.c_int, [_P, _P, _P, _I64, _I32, _P]),
    "adha_pdl_solve_devices": (ctypes.c_int, [_I32, ctypes.POINTER(ctypes.POINTER(adha_cost_table)),
                                              ctypes.POINTER(ctypes.c_double), _I32, _I32, ctypes.POINTER(_I32),
                                              ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_double)]),
    "adha_pdl_solve_scfg": (ctypes.c_int, [ctypes.POINTER(adha_cost_table), _I32, ctypes.POINTER(adha_scfg_node), _I32,
                                           _I32, ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_double)]),
    "adha_tune_writeback": (ctypes.c_int, [_I32]),
    "adha_tune_section_buffers": (ctypes.c_int, [_I32]),
    "adha_tune_fused_jit": (ctypes.c_int, [_I32]),
    "adha_tune_fused_buffers": (ctypes.c_int, [_I32]),
    "adha_tune_section_jit": (ctypes.c_int, [_I32]),
    "adha_fused_jit_build": (ctypes.c_int, [ctypes.POINTER(adha_schema), _I64, ctypes.POINTER(adha_layout),
                                            ctypes.POINTER(adha_section), _I32, _I32, _I32, _I32, ctypes.c_char_p,
                                            ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "adha_jit_available": (ctypes.c_int, []),
    "adha_jit_log": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "adha_tune_remap_direct": (ctypes.c_int, [_I32]),
    "adha_tune_remap_pieces": (ctypes.c_int, [_I32]),
    "adha_tune_clear": (ctypes.c_int, []),
    "adha_tune_export": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "adha_tune_import": (ctypes.c_int, [ctypes.c_char_p]),
    "adha_profile_start": (ctypes.c_int, [_I32]),
    "adha_profile_stop": (ctypes.c_int, [ctypes.POINTER(adha_launch_record), _I32, ctypes.POINTER(_I32)]),
    "adha_ods": (ctypes.c_int, [ctypes.POINTER(adha_schema), ctypes.POINTER(adha_section), _I32, _I32,
                                ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "adha_plan_sections": (ctypes.c_int, [ctypes.POINTER(adha_schema), ctypes.POINTER(adha_section), _I32,
                                          ctypes.POINTER(adha_plan_opts), ctypes.POINTER(ctypes.POINTER(adha_layout_set))]),
    "adha_layout_set_create": (ctypes.c_int, [_I32, _I32, ctypes.POINTER(adha_layout),
                                              ctypes.POINTER(ctypes.POINTER(adha_layout_set))]),
    "adha_cost_table_create": (ctypes.c_int, [_I32, _I32, ctypes.POINTER(ctypes.POINTER(adha_cost_table))]),
    "adha_cost_table_create_fused": (ctypes.c_int, [_I32, _I32, _I32, ctypes.POINTER(ctypes.POINTER(adha_cost_table))]),
    "adha_pdl_solve": (ctypes.c_int, [ctypes.POINTER(adha_cost_table), _I32, ctypes.POINTER(_I32),
                                      ctypes.POINTER(ctypes.c_double)]),
    "adha_pdl_solve_fused": (ctypes.c_int, [ctypes.POINTER(adha_cost_table), _I32, _I32, ctypes.POINTER(_I32),
                                            ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_double)]),
    "adha_measure_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(adha_schema), _I64, ctypes.POINTER(adha_layout),
                                                       ctypes.POINTER(adha_layout_set)]),
    "adha_measure_workspace_bytes_for": (ctypes.c_size_t, [ctypes.POINTER(adha_schema), _I64,
                                                           ctypes.POINTER(adha_layout), ctypes.POINTER(adha_layout_set),
                                                           _I32]),
    "adha_measure": (ctypes.c_int, [ctypes.POINTER(adha_schema), _I64, ctypes.POINTER(adha_layout), _PP,
                                    ctypes.POINTER(adha_section), _I32, ctypes.POINTER(adha_layout_set), _I32, _I32,
                                    _P, ctypes.c_size_t, _P, ctypes.POINTER(ctypes.POINTER(adha_cost_table))]),
    "adha_program_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(adha_schema), _I64, ctypes.POINTER(adha_layout),
                                                       ctypes.POINTER(adha_layout_set)]),
    "adha_program_host_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(adha_schema), _I64, ctypes.POINTER(adha_layout),
                                                            ctypes.POINTER(adha_layout_set), _I32]),
    "adha_run_program_host": (ctypes.c_int, [ctypes.POINTER(adha_schema), _I64, ctypes.POINTER(adha_layout), _PP,
                                             ctypes.POINTER(adha_section), _I32, ctypes.POINTER(adha_layout_set),
                                             ctypes.POINTER(adha_cost_table), ctypes.POINTER(adha_plan_opts), _PP, _I32,
                                             _P, ctypes.c_size_t, _P, ctypes.POINTER(adha_plan)]),
    "adha_run_program": (ctypes.c_int, [ctypes.POINTER(adha_schema), _I64, ctypes.POINTER(adha_layout), _PP,
                                        ctypes.POINTER(adha_section), _I32, ctypes.POINTER(adha_layout_set),
                                        ctypes.POINTER(adha_cost_table), ctypes.POINTER(adha_plan_opts), _P,
                                        ctypes.c_size_t, _P, ctypes.POINTER(adha_plan)]),
}


def load():
    """The loaded libadha.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libadha.so is not built (%s): run __graft_entry__.build() or "
                              "python -m paper_1407_4859_gb300.build" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(rc, fn):
    if rc != 0:
        raise AdhaError(rc, fn, load().adha_last_error().decode())
    return rc
