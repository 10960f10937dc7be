"""The C-ABI library builds, loads and exports every symbol of include/lbm.h;
argument validation that happens before any CUDA call works without a GPU."""
import ctypes

import pytest

import paper_1303_0625_gb300 as G
from paper_1303_0625_gb300 import lbm as L


def test_library_exports_every_header_symbol():
    lib = L.load()
    names = L.header_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} declared in lbm.h but not exported"
        assert n in L._SIGNATURES, f"{n} has no Python binding"


def test_config_default_and_struct_layout():
    c = L.lbm_config_default()
    assert (c.nx, c.ny, c.precision, c.refill, c.force_ring) == (64, 64, L.LBM_FP32_DEV, 1, 256)


def test_struct_layout_matches_header(tmp_path):
    """ctypes mirrors of lbm_config / lbm_disk have the C sizes and offsets."""
    import os
    import subprocess
    src = tmp_path / "layout.c"
    fields_c = [f for f, _ in L.lbm_config._fields_]
    fields_d = [f for f, _ in L.lbm_disk._fields_]
    body = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm.h"', "int main(void){",
            'printf("%zu %zu\\n", sizeof(lbm_config), sizeof(lbm_disk));']
    body += [f'printf("%zu\\n", offsetof(lbm_config, {f}));' for f in fields_c]
    body += [f'printf("%zu\\n", offsetof(lbm_disk, {f}));' for f in fields_d]
    body += ["return 0;}"]
    src.write_text("\n".join(body))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(os.path.dirname(L._build.PKG), "include"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    vals = list(map(int, out))
    assert vals[:2] == [ctypes.sizeof(L.lbm_config), ctypes.sizeof(L.lbm_disk)]
    offs = [getattr(L.lbm_config, f).offset for f in fields_c] + \
           [getattr(L.lbm_disk, f).offset for f in fields_d]
    assert vals[2:] == offs


def test_unet_config_layout_matches_header(tmp_path):
    import os
    import subprocess
    src = tmp_path / "layout_nn.c"
    fields = [f for f, _ in L.lbm_unet_config._fields_]
    body = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm_nn.h"', "int main(void){",
            'printf("%zu\\n", sizeof(lbm_unet_config));']
    body += [f'printf("%zu\\n", offsetof(lbm_unet_config, {f}));' for f in fields]
    body += ["return 0;}"]
    src.write_text("\n".join(body))
    exe = tmp_path / "layout_nn"
    subprocess.run(["gcc", "-I", os.path.join(os.path.dirname(L._build.PKG), "include"),
                    str(src), "-o", str(exe)], check=True)
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                        check=True).stdout.split()))
    assert vals == [ctypes.sizeof(L.lbm_unet_config)] + \
        [getattr(L.lbm_unet_config, f).offset for f in fields]


@pytest.mark.parametrize("field,value", [("tau", 0.5), ("tau", 0.2), ("nx", 3), ("precision", 7),
                                         ("refill", 0), ("force_ring", 0), ("motion_cme", 2), ("relative_changes", -1), ("collision", 2), ("boundary", 2),
                                         ("bc_y", 2)])
def test_create_rejects_invalid_config_without_touching_the_gpu(field, value):
    c = L.make_config(32, 32, 0.8)
    setattr(c, field, value)
    with pytest.raises(L.LBMError) as e:
        L.lbm_create(c)
    assert e.value.status == L.LBM_EINVAL
    assert L.lbm_last_error(None)


def test_status_strings():
    assert L.lbm_status_string(L.LBM_OK) == "ok"
    assert "unstable" in L.lbm_status_string(L.LBM_EUNSTABLE)


def test_product_path_has_no_oracle_dependency():
    """The package must not import, call or build anything under oracle/."""
    import os
    import re
    pkg = os.path.dirname(G.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(root, f)).read()
                assert not re.search(r"\boracle\b", text), f"{f} mentions the oracle"
