"""ctypes declarations of the C ABI in include/bp4m.h (argument marshalling only)."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbp4m.so")

BP4M_OK = 0
BP4M_ETIMEOUT = -4
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "EUNSUPPORTED", -4: "ETIMEOUT", -5: "ECUDA"}

ROTATED = 0
UNROTATED = 1
MEMORY_Z = 0
CODE_CAPACITY = 0
CIRCUIT = 1
PRIOR_P = 0
PRIOR_2P3 = 1
FP64 = 0
FP32 = 1
FP16 = 2
BF16 = 3
DEC_BP4M = 0
DEC_BP4MF = 1
DEC_BBP4MF = 2
EXPORT_W, EXPORT_L, EXPORT_PARITY, EXPORT_EDGES, EXPORT_THRESH = range(5)


class Code(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int), ("d", ctypes.c_int), ("rounds", ctypes.c_int),
                ("basis", ctypes.c_int)]


class Noise(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("p", ctypes.c_double), ("prior_conv", ctypes.c_int),
                ("pair_through_boundary", ctypes.c_int)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("early_exit", ctypes.c_int), ("decoder", ctypes.c_int),
                ("alpha", ctypes.c_double), ("type", ctypes.c_int), ("forced", ctypes.c_int),
                ("stream_cluster", ctypes.c_int), ("tile_form", ctypes.c_int)]


class Counts(ctypes.Structure):
    _fields_ = [("shots", ctypes.c_uint64), ("fail", ctypes.c_uint64 * 3),
                ("unconverged", ctypes.c_uint64 * 2), ("forced_output", ctypes.c_uint64 * 2),
                ("conv_fail", ctypes.c_uint64 * 2), ("iterations", ctypes.c_uint64),
                ("msg_updates", ctypes.c_uint64), ("defects", ctypes.c_uint64),
                ("forced_runs", ctypes.c_uint64), ("forced_rounds", ctypes.c_uint64),
                ("unconverged_any", ctypes.c_uint64), ("conv_fail_any", ctypes.c_uint64)]


class GraphInfo(ctypes.Structure):
    _fields_ = [("n_types", ctypes.c_int), ("n_det", ctypes.c_int * 2), ("n_words", ctypes.c_int * 2),
                ("n_edges", ctypes.c_int * 2), ("n_units", ctypes.c_int), ("model", ctypes.c_int),
                ("d", ctypes.c_int), ("rounds", ctypes.c_int), ("p", ctypes.c_double),
                ("table_bytes", ctypes.c_int64), ("mean_defects", ctypes.c_double * 2)]


class Edge(ctypes.Structure):
    _fields_ = [("u", ctypes.c_int32), ("v", ctypes.c_int32), ("obs", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("q", ctypes.c_double)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 11), ("ms", ctypes.c_double * 11),
                ("msg_updates", ctypes.c_uint64 * 11), ("shots", ctypes.c_uint64 * 11)]


PROFILE_SLOTS = ["classify", "tier1", "tier2", "tier3", "tier4", "tier5", "tier6", "tier7", "global", "sample",
                 "count"]


class Trace(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_void_p), ("partner", ctypes.c_void_p), ("defects", ctypes.c_void_p),
                ("flags", ctypes.c_void_p), ("s_cap", ctypes.c_int)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("batch_shots", ctypes.c_int64), ("slot", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_int64), ("merged_requests", ctypes.c_int64), ("shots", ctypes.c_int64),
                ("evictions", ctypes.c_int64), ("max_inflight_batches", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class MultiInfo(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_int), ("plan_ms", ctypes.c_double * 3), ("runs", ctypes.c_int64),
                ("graph_replays", ctypes.c_int64), ("msg_updates", ctypes.c_uint64),
                ("stream_cluster", ctypes.c_int), ("stream_ms", ctypes.c_double * 2)]


_P = ctypes.c_void_p
SIGNATURES = {
    "bp4m_build_graph": (ctypes.c_int, [ctypes.POINTER(Code), ctypes.POINTER(Noise), ctypes.POINTER(_P)]),
    "bp4m_graph_info": (ctypes.c_int, [_P, ctypes.POINTER(GraphInfo)]),
    "bp4m_graph_export": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_size_t]),
    "bp4m_sample": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                   _P, _P, _P]),
    "bp4m_decode_batch": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(Opts),
                                         _P, _P, _P, _P]),
    "bp4m_decode_trace": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(Opts),
                                         _P, ctypes.POINTER(Trace), _P]),
    "bp4m_sample_and_decode": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64,
                                              ctypes.c_int, ctypes.POINTER(Opts), ctypes.POINTER(Counts), _P]),
    "bp4m_sample_and_decode_range": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint64,
                                                    ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(Opts),
                                                    ctypes.POINTER(Counts), _P]),
    "bp4m_decode_bbp4mf": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(Opts), _P, _P, _P]),
    "bp4m_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "bp4m_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(Profile)]),
    "bp4m_free_graph": (None, [_P]),
    "bp4m_probe_mufu": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P]),
    "bp4m_server_create": (_P, [ctypes.c_int, ctypes.c_int64, ctypes.c_int64]),
    "bp4m_server_add_graph": (ctypes.c_int, [_P, _P]),
    "bp4m_server_submit": (ctypes.c_int64, [_P, ctypes.c_int, _P, ctypes.c_int64, ctypes.c_int,
                                            ctypes.POINTER(Opts), _P, _P]),
    "bp4m_server_wait": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(RequestInfo)]),
    "bp4m_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    "bp4m_server_destroy": (ctypes.c_int, [_P]),
    "bp4m_multi_create": (_P, [ctypes.c_int, _P, _P, _P, ctypes.c_int, ctypes.POINTER(Opts), ctypes.c_int,
                               ctypes.c_int]),
    "bp4m_multi_run": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "bp4m_multi_info": (ctypes.c_int, [_P, ctypes.POINTER(MultiInfo)]),
    "bp4m_multi_destroy": (None, [_P]),
    "bp4m_last_error": (ctypes.c_char_p, []),
    "bp4m_version": (ctypes.c_char_p, []),
}

_lib = None


def load():
    """Loads libbp4m.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libbp4m.so is not built: run `python -c \"import __graft_entry__ as g; g.build()\"` "
                           "or `python -m paper_2603_05381_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class Bp4mError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "error"), code, msg))
        self.code = code


def check(rc):
    if rc != BP4M_OK:
        raise Bp4mError(rc, load().bp4m_last_error().decode(errors="replace"))
    return rc
