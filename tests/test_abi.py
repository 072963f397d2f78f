"""The C-ABI library loads and exports every entry point include/darm.h
declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "darm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(darm_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 15
    missing = [name for name in declared if not hasattr(lib, name)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_the_header():
    import paper_2107_05681_gb300 as darm
    assert sorted(darm.EXPORTED) == _declared()


def test_status_strings_and_uninitialised_calls():
    import subprocess
    import sys
    import paper_2107_05681_gb300 as darm
    assert darm.status_str(darm.OK) == "DARM_OK"
    assert darm.status_str(darm.ERR_NOT_POW2) == "DARM_ERR_NOT_POW2"
    assert darm.status_str(12345) == "DARM_ERR_UNKNOWN"
    # before darm_sort_init every sorting call is refused on the host (in a
    # fresh process: other tests may have initialised this one)
    code = ("import paper_2107_05681_gb300 as d; "
            "assert d.lib.darm_bitonic_sort(None, None, 16, 0, 1, None) == d.ERR_NOT_INIT; "
            "assert d.lib.darm_oddeven_sort_block(None, None, 16, 1, None) == d.ERR_NOT_INIT; "
            "assert d.lib.darm_launch_count() == 0")
    subprocess.run([sys.executable, "-c", code], cwd=ROOT, check=True)
