"""The C-ABI library: it builds, loads without a GPU, and exports every entry
point ``include/rbf.h`` declares.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(rbf_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1305_5179_b300 import build
    build.build()
    import paper_1305_5179_b300 as rbf
    return rbf.lib()


def test_header_declares_the_paper_entry_points():
    names = declared_functions()
    for must in ("rbf_build_centers", "rbf_solve", "rbf_eval_grid", "rbf_matvec", "rbf_plan_create",
                 "rbf_schwarz_setup", "rbf_schwarz_apply", "rbf_residual", "rbf_count_pairs"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_binding_covers_header():
    import paper_1305_5179_b300 as rbf
    assert sorted(rbf.EXPORTS) == declared_functions()


def test_host_only_calls(lib):
    assert lib.rbf_version() == 1
    assert lib.rbf_status_string(0) == b"RBF_OK"
    assert lib.rbf_status_string(7) == b"RBF_ERR_NOT_SPD"
    # invalid arguments are rejected on the host, before any device work
    assert lib.rbf_ctx_create(None, 0) == 1
    assert lib.rbf_plan_destroy(None) == 0
    assert lib.rbf_matvec(None, None, None, None) == 1


def test_struct_layouts_match_header():
    """ctypes mirrors of the C structs have the C sizes (checked by compiling a probe)."""
    import subprocess
    import tempfile
    import paper_1305_5179_b300 as rbf
    src = """
#include <stdio.h>
#include "rbf.h"
#include "rbf_probe.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(rbf_plan_params), sizeof(rbf_plan_info), sizeof(rbf_schwarz_params),
         sizeof(rbf_solve_params), sizeof(rbf_report), sizeof(rbf_grid), sizeof(rbf_probe_result));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = list(map(int, subprocess.check_output([exe]).split()))
    mine = [ctypes.sizeof(t) for t in (rbf.PlanParams, rbf.PlanInfo, rbf.SchwarzParams, rbf.SolveParams,
                                       rbf.Report, rbf.Grid, rbf.ProbeResult)]
    assert sizes == mine


def test_no_gpu_means_loud_failure(lib):
    """Without a device the context cannot be created: the binding raises instead of falling back."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1305_5179_b300 as rbf
    with pytest.raises(rbf.RbfError):
        rbf.Context(0)
