"""ctypes loader of libtdprobe.so, the issue-rate probe that checks the sweep
kernel's derived roofline peak (SMs x 128 lanes x SM clock) by measurement.
It is a measurement aid for the benchmark, kept out of the depth library; see
csrc/td_issue_rate.h for the call."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdprobe.so")

TD_ISSUE_FFMA, TD_ISSUE_FFMA2, TD_ISSUE_INT, TD_ISSUE_MIXED = 0, 1, 2, 3
ISSUE_KINDS = {"ffma": TD_ISSUE_FFMA, "ffma2": TD_ISSUE_FFMA2, "int": TD_ISSUE_INT, "mixed": TD_ISSUE_MIXED}

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libtdprobe.so is not built: run `python -m paper_1409_3901_gb300.build`")
        _lib = ctypes.CDLL(LIB_PATH)
        _lib.td_issue_rate.restype = ctypes.c_int
        _lib.td_issue_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_float)]
    return _lib


def issue_rate(kind, device=0):
    """(lane operations per second, launch ms) of td_issue_rate for one kind
    ("ffma", "ffma2", "int", "mixed")."""
    rate, ms = ctypes.c_double(), ctypes.c_float()
    rc = lib().td_issue_rate(device, ISSUE_KINDS[kind], ctypes.byref(rate), ctypes.byref(ms))
    if rc != 0:
        raise RuntimeError("td_issue_rate(%s) failed: %d" % (kind, rc))
    return rate.value, ms.value
