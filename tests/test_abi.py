"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h (no compute calls: these run without a GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(mnbab_\w+)\s*\(", txt):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2205_00263_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mnbab_create", "mnbab_load_network", "mnbab_set_property", "mnbab_set_mnc",
              "mnbab_bound_batch", "mnbab_optimize", "mnbab_score_branches", "mnbab_bab_step",
              "mnbab_get_verdict", "mnbab_export_params"):
        assert n in names


def test_boundary_calls_cite_the_paper():
    """Each call of the method's boundary is documented with the passage that
    defines it: the comment text between the previous declaration and its
    own (its group heading included) names a section or appendix."""
    txt = open(os.path.join(ROOT, "include", "mnbab.h")).read()
    decl = [(m.start(), m.group(1)) for m in
            re.finditer(r"\nmnbab_status\s+(mnbab_\w+)\s*\(", txt)]
    prev_end = {}
    for k, (pos, name) in enumerate(decl):
        start = txt.index(";", decl[k - 1][0]) if k else 0
        prev_end[name] = txt[start:pos]
    for name in ("mnbab_load_network", "mnbab_set_property", "mnbab_set_mnc",
                 "mnbab_bound_batch", "mnbab_deeppoly_batch", "mnbab_bound_grad",
                 "mnbab_optimize", "mnbab_score_branches", "mnbab_bab_step",
                 "mnbab_get_verdict", "mnbab_get_root_bounds", "mnbab_node_root",
                 "mnbab_optimize_intermediate", "mnbab_attack", "mnbab_set_branching"):
        assert re.search(r"Sec\. \d|App\. [A-Z]", prev_end[name]), name


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T mnbab_" in l}
    assert _declared() <= exported


def test_binding_covers_every_symbol(lib_path):
    from paper_2205_00263_gb300 import _lib
    assert set(_lib.SIGNATURES) == _declared()
    _lib.load()


def test_build_targets_sm_103a():
    from paper_2205_00263_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_create_without_device_fails_cleanly(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2205_00263_gb300 import Context, MnbabError
    with pytest.raises(MnbabError):
        Context(device=0)
