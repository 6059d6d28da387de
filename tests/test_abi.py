"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(mvn_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_14892_gb300 import mvn
    return mvn.LIB_PATH


def test_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_2405_14892_gb300 import mvn
    assert set(mvn.SIGNATURES) == _declared()
    mvn.lib()  # sets argtypes for every symbol


def test_library_is_sm103a_only(libpath):
    import subprocess
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", libpath],
                         capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    archs = set(re.findall(r"sm_(\d+a?)", out.stdout))
    assert archs == {"103a"}, archs


def test_null_context_is_an_argument_error(libpath):
    from paper_2405_14892_gb300 import mvn
    lib = mvn.lib()
    assert lib.mvn_sov(None, 1, None, None, None, 1, None, 0, None, None) == mvn.MVN_ERR_ARG
    assert lib.mvn_destroy(None) == mvn.MVN_ERR_ARG
    assert lib.mvn_last_error(None) == b"null context"


def _zero_args(argtypes):
    vals = []
    for t in argtypes:
        if t is ctypes.c_double:
            vals.append(0.0)
        elif t in (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64):
            vals.append(0)
        else:
            vals.append(None)  # every pointer, handle and string argument NULL
    return vals


def test_every_entry_point_rejects_null_handles(libpath):
    """Each exported call, given NULL for its context/graph/TLR handle (and every other
    pointer), returns the error the header's conventions state without reaching CUDA (this host
    has no GPU, so a call that reached CUDA would report MVN_ERR_CUDA instead)."""
    from paper_2405_14892_gb300 import mvn
    lib = mvn.lib()
    special = {"mvn_last_error": b"null context", "mvn_launch_count": -1,
               "mvn_graph_kernels": 0, "mvn_graph_destroy": mvn.MVN_OK}
    got = {}
    for name, (_, argtypes) in mvn.SIGNATURES.items():
        got[name] = getattr(lib, name)(*_zero_args(argtypes))
    want = {name: special.get(name, mvn.MVN_ERR_ARG) for name in mvn.SIGNATURES}
    assert got == want
