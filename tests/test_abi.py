"""Host-side checks of the C ABI (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cpapr.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cpapr_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2307_03276_gb300 import build, cpapr
    build.build()
    return cpapr.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("cpapr_create", "cpapr_phi", "cpapr_mttkrp", "cpapr_mu_solve", "cpapr_batch_mu_solve",
                 "cpapr_destroy", "cpapr_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in cpapr.h but not exported"


def test_binding_names_match_header(lib):
    from paper_2307_03276_gb300 import cpapr
    for name in declared_functions():
        assert hasattr(cpapr, name), f"binding lacks {name}"


def test_default_options_and_version(lib):
    from paper_2307_03276_gb300 import cpapr
    o = cpapr.cpapr_default_options()
    assert o.precision == 0 and o.eps == 1e-10 and o.kappa == 0.01 and o.kappa_tol == 1e-10
    assert "sm_103a" in cpapr.cpapr_version()


def test_ctypes_structs_match_c_layout(tmp_path):
    """The binding's struct mirrors have the C compiler's sizes and offsets."""
    import subprocess
    from paper_2307_03276_gb300 import cpapr
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "cpapr.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(cpapr_options),"
        " offsetof(cpapr_options, stream), offsetof(cpapr_options, profile), sizeof(cpapr_result),"
        " offsetof(cpapr_result, loglik), sizeof(cpapr_info), offsetof(cpapr_info, device_bytes),"
        " offsetof(cpapr_options, l2_persist), offsetof(cpapr_info, l2_window_bytes));"
        "printf(\"%zu\\n\", offsetof(cpapr_options, tune_cache));return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(cpapr.Options), cpapr.Options.stream.offset, cpapr.Options.profile.offset,
            ctypes.sizeof(cpapr.Result), cpapr.Result.loglik.offset, ctypes.sizeof(cpapr.Info),
            cpapr.Info.device_bytes.offset, cpapr.Options.l2_persist.offset, cpapr.Info.l2_window_bytes.offset,
            cpapr.Options.tune_cache.offset]
    assert got == want


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    """Argument checks run on the host first, so these fail cleanly without a device."""
    import numpy as np
    from paper_2307_03276_gb300 import cpapr
    idx = np.zeros((3, 4), dtype=np.int64)
    vals = np.ones(4)
    with pytest.raises(cpapr.CpaprError) as e:
        cpapr.cpapr_create([3, 3], idx[:2], vals, 0)
    assert e.value.status == 1
    with pytest.raises(cpapr.CpaprError) as e:
        cpapr.cpapr_create([3, 0, 3], idx, vals, 2)
    assert e.value.status == 2
    with pytest.raises(cpapr.CpaprError) as e:
        cpapr.cpapr_create([3] * 9, np.zeros((9, 4), dtype=np.int64), vals, 2)
    assert e.value.status == 1
    with pytest.raises(cpapr.CpaprError) as e:
        cpapr.cpapr_create([3, 3, 3], idx, vals, 2, cpapr.cpapr_default_options(rank_lanes=3))
    assert e.value.status == 1
    with pytest.raises(cpapr.CpaprError) as e:
        cpapr.cpapr_create([3, 3, 3], idx, vals, 2, cpapr.cpapr_default_options(l2_persist=2))
    assert e.value.status == 1
    with pytest.raises(cpapr.CpaprError) as e:
        cpapr.cpapr_create([3, 3, 3], idx, vals, 2, cpapr.cpapr_default_options(fp64_dot=3))
    assert e.value.status == 1
