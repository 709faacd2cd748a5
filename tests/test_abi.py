"""The C-ABI library builds for sm_103a, loads, and exports every function include/sfft.h declares.

No compute call is made (no GPU here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sfft.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(sfft_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1201_2501_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sfft_plan_create", "sfft_execute", "sfft_plan_destroy", "sfft_hash_to_bins",
                     "sfft_exact_decode", "sfft_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(sfft_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_loads_and_covers_the_header(built_lib):
    from paper_1201_2501_gb300 import sfft

    L = sfft.lib()
    for name in declared_functions():
        assert hasattr(L, name)
        assert name in sfft.EXPORTED, f"binding lacks {name}"
    assert sfft.sfft_status_str(sfft.SFFT_OK) == "ok"


def test_params_default_and_struct_layout(built_lib):
    from paper_1201_2501_gb300 import sfft

    p = sfft.sfft_params_default(1 << 22, 64, sfft.SFFT_EXACT)
    assert p.n == 1 << 22 and p.k == 64 and p.mode == 0 and p.precision == 0
    assert p.thr == 0.5 and p.alpha0 == 0.5 and p.bins_per_k == 4.0 and p.z_cap == 256
    # every test parameter field exists in the C struct under the same name
    from tests.common import FIELDS_DEFAULT

    for f in FIELDS_DEFAULT:
        assert hasattr(p, f)



def test_binding_struct_layouts_match_the_header(tmp_path):
    """sizeof and every field offset of the ctypes mirrors equal the C compiler's for include/sfft.h."""
    import ctypes

    from paper_1201_2501_gb300 import sfft

    mirrors = {"sfft_params": sfft.SfftParams, "sfft_request": sfft.SfftRequest,
               "sfft_server_config": sfft.SfftServerConfig, "sfft_job": sfft.SfftJob,
               "sfft_job_result": sfft.SfftJobResult, "sfft_server_stats": sfft.SfftServerStats,
               "sfft_tune_entry": sfft.SfftTuneEntry}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sfft.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, f, v = line.split()
        got[(cname, f)] = int(v)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_server_create_without_a_device_fails_cleanly(built_lib):
    """With no CUDA device the server reports SFFT_ERR_CUDA and hands out no handle."""
    import ctypes

    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_1201_2501_gb300 import sfft

    h = ctypes.c_void_p(123)
    st = sfft.lib().sfft_server_create(None, ctypes.byref(h))
    assert st == sfft.SFFT_ERR_CUDA
    assert not h.value
    assert sfft.lib().sfft_server_destroy(None) == sfft.SFFT_OK
