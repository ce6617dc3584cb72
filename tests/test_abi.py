"""The C-ABI library loads here (no GPU needed) and exports every entry point
that include/ni.h declares; the binding's structs match the header's sizes."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(files=("ni.h", "ni_cnn.h")):
    names = set()
    for f in files:
        txt = open(os.path.join(ROOT, "include", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(ni_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2510_11508_gb300 import build, ni
    build.build()
    return ni.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    from paper_2510_11508_gb300 import ni
    assert sorted(ni.EXPORTS) == _declared(("ni.h",))


def test_config_default_is_host_only(lib):
    from paper_2510_11508_gb300 import ni
    cfg = ni.default_config(512, 612)
    assert (cfg.H, cfg.W, cfg.T, cfg.freq_merging, cfg.connectivity) == (512, 612, 15, 5, 4)
    assert cfg.L == 1e-5 and cfg.U == 1e-3 and cfg.dE_max == 1e-3
    assert lib.ni_status_string(4) == b"NI_ERR_NOT_CONVERGED"


def test_struct_layout_matches_header(lib, tmp_path):
    """Compile a tiny C program against include/ni.h and compare sizeof/offsets
    with the ctypes mirrors of the binding."""
    import shutil
    import subprocess
    from paper_2510_11508_gb300 import ni
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "l.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ni.h"\nint main(){'
                   'printf("%zu %zu %zu %zu %zu\\n", sizeof(ni_config), sizeof(ni_stats),'
                   ' offsetof(ni_config, cg_rtol), offsetof(ni_stats, energy), offsetof(ni_config, fill_kernels));}')
    exe = tmp_path / "l"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    exp = [C.sizeof(ni.Config), C.sizeof(ni.Stats), ni.Config.cg_rtol.offset,
           ni.Stats.energy.offset, ni.Config.fill_kernels.offset]
    assert [int(v) for v in out] == exp


def test_no_oracle_in_product_path():
    """The package never imports the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2510_11508_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "oracle" not in txt.replace("oracles", ""), f


@pytest.mark.parametrize("field,value", [
    ("H", 0), ("connectivity", 6), ("connectivity", 0),
    ("connectivity", 8),   # 8-connectivity needs batched = 0 (the default is 1)
    ("T", 0), ("T", 1000), ("precision", 2), ("precond", 2),
    ("mg_omega", 1.0), ("mg_correction", 4.0), ("ctas_per_sm", 9), ("fill_kernels", 2), ("scale_solver", 3), ("bini_residual", 2), ("learned_weights", 1),
    ("mg_coarse_sweeps", 100), ("cg_maxit", 0), ("n_fill_irls", 0), ("dE_max", -1.0),
])
def test_invalid_config_rejected_before_any_device_call(lib, field, value):
    """ni_create validates the whole config on the host and returns
    NI_ERR_INVALID_ARG (no device is touched, so this runs without a GPU)."""
    from paper_2510_11508_gb300 import ni
    cfg = ni.default_config(64, 64)
    setattr(cfg, field, type(getattr(cfg, field))(value))
    h = C.c_void_p()
    assert lib.ni_create(C.byref(cfg), C.byref(h)) == 1   # NI_ERR_INVALID_ARG
    assert not h.value


def test_warm_start_needs_the_batched_fill(lib):
    from paper_2510_11508_gb300 import ni
    cfg = ni.default_config(64, 64)
    cfg.warm_start, cfg.batched = 1, 0
    h = C.c_void_p()
    assert lib.ni_create(C.byref(cfg), C.byref(h)) == 1
