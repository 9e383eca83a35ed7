"""The debug build (libswept_debug.so: device-side index checks, include/swept.h
"Debug build").

CPU: the debug build compiles, its library reports that the checks are on
(the release library that they are off), and it exports the same symbols.

GPU: every kernel family and execution mode runs under the checks with no check
failing and results equal to the oracle (tests/debug_cases.py, in a child
process because a process loads one build), and the recording path reports a
failing check: swept_debug_probe checks i < bound for i < n and so fails for
i >= bound, where the copy it skips was in range anyway.
"""
import ctypes
import os
import subprocess
import sys

import pytest

from paper_1612_02495_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(code, timeout=900):
    env = dict(os.environ, SWEPT_DEBUG="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=timeout)


@pytest.fixture(scope="module")
def debug_lib():
    return libbuild.build(debug=True)


def test_debug_library_reports_checks_on(debug_lib):
    assert os.path.basename(debug_lib) == "libswept_debug.so"
    # release library: checks off, nothing to read
    rel = ctypes.CDLL(libbuild.build())
    en, chk, idx = ctypes.c_int32(-1), ctypes.c_int32(-1), ctypes.c_int64(-1)
    rel.swept_debug_status.restype = ctypes.c_int
    assert rel.swept_debug_status(ctypes.byref(en), ctypes.byref(chk), ctypes.byref(idx)) == 0
    assert (en.value, chk.value, idx.value) == (0, 0, 0)
    # debug library: checks on (reading the records needs a device)
    r = _child("import ctypes; from paper_1612_02495_gb300 import swept as S; "
               "en = ctypes.c_int32(-1); st = S.swept_debug_status(ctypes.byref(en), None, None); "
               "print(S.LIB_PATH, en.value, st)")
    assert r.returncode == 0, r.stderr
    path, en_v, st = r.stdout.split()
    assert os.path.basename(path) == "libswept_debug.so" and en_v == "1"
    assert int(st) in (0, 3)  # SWEPT_OK with a device, SWEPT_ECUDA without one


def test_debug_library_exports_the_release_symbols(debug_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", debug_lib], capture_output=True, text=True).stdout
    rel = subprocess.run(["nm", "-D", "--defined-only", libbuild.build()], capture_output=True, text=True).stdout
    names = lambda t: {ln.split()[-1] for ln in t.splitlines() if " T " in ln and ln.split()[-1].startswith(
        ("swept", "classic"))}
    assert names(rel) and names(out) == names(rel)


@pytest.mark.gpu
def test_debug_build_runs_every_mode_clean(debug_lib):
    r = _child("import runpy; runpy.run_path('tests/debug_cases.py', run_name='__main__')", timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "all clean" in r.stdout, r.stdout[-3000:]


@pytest.mark.gpu
def test_debug_probe_reports_a_failing_check(debug_lib):
    code = (
        "import torch; from paper_1612_02495_gb300 import swept as S\n"
        "buf = torch.arange(1000, dtype=torch.float64, device='cuda'); ref = buf.clone()\n"
        "assert S.debug_status() == (True, None)\n"
        "assert S.swept_debug_probe(S.ctypes.c_void_p(buf.data_ptr()), 1000, 600, None) == S.SWEPT_OK\n"
        "en, rec = S.debug_status()\n"
        "assert en and rec is not None and rec[0] == 'probe' and 600 <= rec[1] < 1000, rec\n"
        "assert S.debug_status() == (True, None)  # cleared\n"
        "assert S.swept_debug_probe(S.ctypes.c_void_p(buf.data_ptr()), 1000, 1000, None) == S.SWEPT_OK\n"
        "assert S.debug_status() == (True, None)\n"
        "assert torch.equal(buf, ref)\n"
        "assert S.swept_debug_probe(None, 10, 11, None) == S.SWEPT_EINVAL\n"
        "print('probe ok')\n")
    r = _child(code)
    assert r.returncode == 0 and "probe ok" in r.stdout, r.stdout + r.stderr
