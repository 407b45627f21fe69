"""ctypes binding of libcg_growth.so: the C ABI of include/cg_growth.h, same names.

Argument marshalling only.  Every step of the growth runs in the library's CUDA kernels; there
is no CPU fallback.  Importing this module loads the library and raises if it is missing.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcg_growth.so")

CG_OK = 0
CG_TRUNC_RADIUS = 1
CG_TRUNC_MEMCAP = 2
CG_TRUNC_ABOVE = 3
CG_EINVAL = -1
CG_ENOTCLOSED = -2
CG_ENOMEM = -3
CG_ECUDA = -4
CG_EDEVICE = -5
CG_ETIMEOUT = -6
CG_ETOOBIG = -7

CG_STRATEGY_AUTO = 0
CG_STRATEGY_HASH = 1
CG_STRATEGY_SORT = 2
CG_STRATEGY_BITMAP = 3
CG_STRATEGY_SWEEP = 4
CG_OPT_BATCH_WAVE_L2 = 6
CG_OPT_BATCH_VISITED = 7
CG_OPT_GRAPH = 8
CG_OPT_BATCH_ACTIVE = 10
CG_OPT_UNIT = 11

CG_OPT_STRATEGY = 1
CG_OPT_STOP_ABOVE = 2
CG_OPT_KEEP_LAST = 3
CG_OPT_GRID = 4
CG_OPT_ILP = 5
CG_OPT_SWEEP_ORDER = 9
CG_NOALLOC_MAX_STATES = 1 << 20
CG_NOALLOC_MAX_GENS = 256
CG_SERVER_SOLO_STATES = 1 << 24

# Every symbol include/cg_growth.h declares: name -> (restype, argtypes)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

class cg_growth_stats(ctypes.Structure):
    _fields_ = [("kernel_ms", ctypes.c_double), ("launches", ctypes.c_int), ("rounds", ctypes.c_int),
                ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64),
                ("state_capacity", ctypes.c_uint64), ("table_slots", ctypes.c_uint64),
                ("strategy_used", ctypes.c_int), ("probe_variant", ctypes.c_int),
                ("switched_to_sort", ctypes.c_int), ("sort_from", ctypes.c_int)]


SIGNATURES = {
    "cg_set_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, _vp]),
    "cg_growth_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _u8p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_uint64, ctypes.POINTER(_vp)]),
    "cg_growth_set_option": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int64]),
    "cg_growth_set_start": (ctypes.c_int, [_vp, _u8p]),
    "cg_growth_run": (ctypes.c_int, [_vp, _vp, _u64p, ctypes.c_int, _ip]),
    "cg_growth_last_layer": (ctypes.c_int, [_vp, _u64p, ctypes.c_uint64, _u64p]),
    "cg_growth_group_order": (ctypes.c_uint64, [_vp]),
    "cg_growth_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(cg_growth_stats)]),
    "cg_growth_destroy": (ctypes.c_int, [_vp]),
    "cg_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "cg_last_error_detail": (ctypes.c_char_p, []),
    "cg_growth_key_width": (ctypes.c_int, [_vp]),
    "cg_growth_key_words": (ctypes.c_int, [_vp]),
    "cg_batch_create": (ctypes.c_int, [ctypes.c_int, _ip, _ip, _u8p, _u64p, _ip, _ip, ctypes.c_uint64,
                                       ctypes.POINTER(_vp)]),
    "cg_batch_run": (ctypes.c_int, [_vp, _vp, _u64p, ctypes.c_int, _ip, _ip]),
    "cg_batch_destroy": (ctypes.c_int, [_vp]),
    "cg_batch_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(cg_growth_stats)]),
    "cg_batch_set_wave_l2": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "cg_batch_set_option": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int64]),
    "cg_server_create": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.POINTER(_vp)]),
    "cg_server_submit": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _u8p, ctypes.c_int, ctypes.c_int, _u64p]),
    "cg_server_predict": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _u8p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_uint64, _u64p, _u64p, _u64p, _ip]),
    "cg_server_step": (ctypes.c_int, [_vp, _vp, _ip, _ip]),
    "cg_server_finished": (ctypes.c_int, [_vp, _u64p, ctypes.c_int, _ip]),
    "cg_server_result": (ctypes.c_int, [_vp, ctypes.c_uint64, _u64p, ctypes.c_int, _ip, _ip]),
    "cg_server_load": (ctypes.c_int, [_vp, _ip, _ip, _u64p]),
    "cg_server_destroy": (ctypes.c_int, [_vp]),
    "cg_growth_run_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _u8p, ctypes.c_int, ctypes.c_int,
                                             _vp, _u64p, ctypes.c_int, _ip]),
    "cg_expand": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _u8p, _vp, ctypes.c_uint64, _vp, _vp]),
    "cg_hash_insert": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp, ctypes.c_uint64, _vp, _vp, _vp]),
    "cg_hash_clear": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp]),
    "cg_shard_owner": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int]),
    "cg_shard_expand": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _u8p, _vp, ctypes.c_uint64, ctypes.c_int,
                                       _vp, ctypes.c_uint64, _u64p, _vp]),
    "cg_perm_rank": (ctypes.c_int, [ctypes.c_int, _vp, ctypes.c_uint64, _vp, _vp]),
    "cg_perm_unrank": (ctypes.c_int, [ctypes.c_int, _vp, ctypes.c_uint64, _vp, _vp]),
    "cg_sort_unique_scratch_bytes": (ctypes.c_size_t, [ctypes.c_uint64]),
    "cg_sort_unique": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_int, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "cg_set_difference": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp, ctypes.c_uint64, _vp, ctypes.c_uint64,
                                         _vp, _vp, _vp, ctypes.c_size_t, _vp]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -m paper_2509_19162_gb300.builder); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class CgError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        detail = lib.cg_last_error_detail().decode() if code in (-3, -4) else ""
        super().__init__(f"{where}: {strerror(code)} (code {code})" + (f" [{detail}]" if detail else ""))


def strerror(code: int) -> str:
    return lib.cg_strerror(int(code)).decode()


def check(code: int, where: str) -> int:
    if code < 0:
        raise CgError(code, where)
    return code


# Same names as the C ABI, for callers that want the raw entry points.
def _export(name):
    return getattr(lib, name)


cg_set_allocator = _export("cg_set_allocator")
cg_growth_create = _export("cg_growth_create")
cg_growth_set_option = _export("cg_growth_set_option")
cg_growth_set_start = _export("cg_growth_set_start")
cg_growth_run = _export("cg_growth_run")
cg_growth_last_layer = _export("cg_growth_last_layer")
cg_growth_group_order = _export("cg_growth_group_order")
cg_growth_get_stats = _export("cg_growth_get_stats")
cg_growth_destroy = _export("cg_growth_destroy")
cg_strerror = _export("cg_strerror")
cg_last_error_detail = _export("cg_last_error_detail")
cg_growth_key_width = _export("cg_growth_key_width")
cg_growth_key_words = _export("cg_growth_key_words")
cg_batch_create = _export("cg_batch_create")
cg_batch_run = _export("cg_batch_run")
cg_batch_destroy = _export("cg_batch_destroy")
cg_batch_get_stats = _export("cg_batch_get_stats")
cg_batch_set_wave_l2 = _export("cg_batch_set_wave_l2")
cg_batch_set_option = _export("cg_batch_set_option")
cg_perm_rank = _export("cg_perm_rank")
cg_perm_unrank = _export("cg_perm_unrank")
cg_server_create = _export("cg_server_create")
cg_server_submit = _export("cg_server_submit")
cg_server_predict = _export("cg_server_predict")
cg_server_step = _export("cg_server_step")
cg_server_finished = _export("cg_server_finished")
cg_server_result = _export("cg_server_result")
cg_server_load = _export("cg_server_load")
cg_server_destroy = _export("cg_server_destroy")
cg_growth_run_noalloc = _export("cg_growth_run_noalloc")
cg_expand = _export("cg_expand")
cg_hash_insert = _export("cg_hash_insert")
cg_hash_clear = _export("cg_hash_clear")
cg_shard_owner = _export("cg_shard_owner")
cg_shard_expand = _export("cg_shard_expand")
cg_sort_unique_scratch_bytes = _export("cg_sort_unique_scratch_bytes")
cg_sort_unique = _export("cg_sort_unique")
cg_set_difference = _export("cg_set_difference")
