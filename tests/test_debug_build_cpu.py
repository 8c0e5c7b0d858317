"""The bounds-checked build of the library (-DZC_DEBUG) on the CPU: it
compiles for sm_103a, loads, exports every declared function, says it is the
checked build, and a process that sets ZC_LIBRARY=debug loads it instead of
the release library.  (Its GPU run is tests/test_gpu_debug_build.py.)"""
import ctypes
import os
import subprocess
import sys

from paper_2308_05199_gb300 import build as zbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "tests"))
from test_lib_cpu import declared_functions  # noqa: E402


def test_debug_library_builds_and_exports_everything():
    path = zbuild.build(debug=True)
    assert path == zbuild.DEBUG_LIB and os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.zc_version.restype = ctypes.c_char_p
    assert b"bounds-checked" in lib.zc_version()
    rel = ctypes.CDLL(zbuild.build())
    rel.zc_version.restype = ctypes.c_char_p
    assert b"bounds-checked" not in rel.zc_version()


def test_environment_selects_the_debug_library():
    code = ("from paper_2308_05199_gb300 import zc; print(zc.lib_path()); print(zc.zc_version())")
    env = dict(os.environ, ZC_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    path, ver = r.stdout.split("\n")[:2]
    assert path == zbuild.DEBUG_LIB and "bounds-checked" in ver
