"""The C-ABI library loads and exports every symbol the headers under
include/ declare; host-side argument checks (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tukey_depth.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


def _declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"\b(td_[a-z_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def tukey():
    from paper_1409_3901_gb300 import build
    build.build()
    from paper_1409_3901_gb300 import tukey as t
    return t


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ["td_create", "td_destroy", "td_depth", "td_depth_batched", "td_stream_create",
              "td_stream_submit", "td_stream_poll", "td_stream_wait", "td_stream_destroy",
              "td_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(tukey):
    lib = ctypes.CDLL(tukey.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert sorted(tukey.EXPORTED) == _declared_functions()


def test_coord_limits_and_strerror(tukey):
    lim = [tukey.td_coord_limit(p) for p in range(0, 8)]
    assert lim[0] == 0 and lim[7] == 0
    assert lim[1] == lim[2] == lim[3] == 2 ** 22 - 1
    # every exact intermediate fits: d * max|minor| * M < 2^62
    assert 4 * 2 * lim[4] ** 3 < 2 ** 62
    assert 5 * 3 ** 1.5 * lim[5] ** 4 < 2 ** 62
    assert 6 * 16 * lim[6] ** 5 < 2 ** 62
    for code in range(-8, 1):
        assert tukey.td_strerror(code)
    assert tukey.td_strerror(-99) == b"unknown error"


def test_autotune_arguments_rejected_without_device(tukey):
    assert tukey.td_autotune(None, 4, 100, None) == tukey.TD_ERR_INVALID
    assert tukey.td_set_tuned(None, 4, 5, 64) == tukey.TD_ERR_INVALID


def test_null_and_bad_arguments_rejected_without_device(tukey):
    assert tukey.td_create(None, 0, None) == tukey.TD_ERR_INVALID
    assert tukey.td_depth(None, None, 1, 1, None, 0, None, None) == tukey.TD_ERR_INVALID
    assert tukey.td_destroy(None) == tukey.TD_ERR_INVALID
    assert tukey.td_stream_create(None, 0, None) == tukey.TD_ERR_INVALID
    done = ctypes.c_int()
    assert tukey.td_stream_poll(None, 1, ctypes.byref(done)) == tukey.TD_ERR_INVALID


def test_probe_library_is_separate(tukey):
    """The issue-rate probe lives in libtdprobe.so, not in the depth library,
    and rejects bad arguments without a device."""
    from paper_1409_3901_gb300 import probe
    assert not hasattr(ctypes.CDLL(tukey.LIB_PATH), "td_issue_rate")
    lib = probe.lib()
    rate = ctypes.c_double()
    assert lib.td_issue_rate(0, 0, None, None) == tukey.TD_ERR_INVALID
    assert lib.td_issue_rate(0, 4, ctypes.byref(rate), None) == tukey.TD_ERR_INVALID
    assert lib.td_issue_rate(0, -1, ctypes.byref(rate), None) == tukey.TD_ERR_INVALID


def test_create_reports_missing_device(tukey):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    ptr = ctypes.c_void_p()
    rc = tukey.td_create(ctypes.byref(ptr), 0, None)
    assert rc in (tukey.TD_ERR_CUDA, tukey.TD_ERR_OOM)
    assert not ptr.value
    from paper_1409_3901_gb300 import probe
    rate = ctypes.c_double()
    assert probe.lib().td_issue_rate(0, 0, ctypes.byref(rate), None) == tukey.TD_ERR_CUDA


def test_structs_match_header_layout(tukey, tmp_path):
    """Every field offset and struct size of the binding against the header,
    as the C compiler lays them out."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"td_options": tukey.td_options, "td_dataset": tukey.td_dataset, "td_stats": tukey.td_stats,
               "td_tune_result": tukey.td_tune_result}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tukey_depth.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-I", inc, str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        a, b, c = line.split()
        got[(a, b)] = int(c)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_workload_generators_are_deterministic():
    from paper_1409_3901_gb300 import workloads as W
    a, b = W.w1(), W.w1()
    assert a.checksum() == b.checksum()
    d = W.w2()
    assert d.X.shape == (1000, 4) and d.Zq.shape == (64, 4)
    assert np.abs(d.X).max() <= 127
    d4 = W.w4()
    # the copied rows and the hyperplane rows are present
    uniq = np.unique(d4.X, axis=0)
    assert len(uniq) <= 200 - 15
    a_, c_ = d4.meta["hyperplane_a"], d4.meta["hyperplane_c"]
    on = (d4.X @ np.array(a_) == c_).sum()
    assert on >= 10


def test_algorithm_option_validation(tukey):
    """Algorithm 3 runs in the filtered form on unsharded calls only; unknown
    algorithms are rejected before any device work."""
    bad = [tukey.options(algorithm=3),
           tukey.options(algorithm=tukey.TD_ALG_ADIA, mode=tukey.TD_MODE_PLAIN_EXACT),
           tukey.options(algorithm=tukey.TD_ALG_ADIA, shard_index=0, shard_count=2)]
    for o in bad:
        ptr = ctypes.c_void_p()
        assert tukey.td_create(ctypes.byref(ptr), 0, ctypes.byref(o)) == tukey.TD_ERR_INVALID
        assert not ptr.value
    assert tukey.td_set_options(None, ctypes.byref(bad[0])) == tukey.TD_ERR_INVALID


def test_critical_form_not_served_by_streams(tukey):
    """TD_ALG_CRITICAL is accepted by td_create's validation; the stream API
    refuses it (checked without a device: td_create fails first on CPU)."""
    o = tukey.options(algorithm=tukey.TD_ALG_CRITICAL)
    ptr = ctypes.c_void_p()
    rc = tukey.td_create(ctypes.byref(ptr), 0, ctypes.byref(o))
    assert rc != tukey.TD_ERR_INVALID
    if ptr.value:
        tukey.td_destroy(ptr)


def test_missing_library_fails_loudly(tukey, monkeypatch):
    """No fallback: without the built library the binding raises."""
    monkeypatch.setattr(tukey, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libtukeydepth.so"))
    with pytest.raises(tukey.LibraryMissing):
        tukey._load()


def test_smoke_needs_a_device():
    """smoke() runs the kernels on cuda:0 and refuses to run without one."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    import __graft_entry__
    with pytest.raises(AssertionError):
        __graft_entry__.smoke()
