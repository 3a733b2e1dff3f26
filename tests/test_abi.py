"""The C-ABI library loads without a GPU and exports every call include/im_gb300.h declares."""
import re
import subprocess
from pathlib import Path

import pytest

import paper_2311_07554_gb300 as im
from paper_2311_07554_gb300 import _native
from paper_2311_07554_gb300 import build as cuda_build

ROOT = Path(__file__).resolve().parent.parent
HEADER = ROOT / "include" / "im_gb300.h"


def _declared():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(im_[a-z_]+)\s*\(", text)))


def _defines():
    return {k: int(v) for k, v in re.findall(r"#define\s+(IM_[A-Z_]+)\s+\(?(-?\d+)\)?", HEADER.read_text())}


@pytest.fixture(scope="module")
def libpath():
    return cuda_build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("im_create", "im_build_sketches", "im_select_seeds", "im_spread", "im_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", str(libpath)], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b[TW]\s+(im_\w+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binds_every_symbol(libpath):
    L = im.lib()
    for name in _declared():
        assert hasattr(L, name)
    assert L.im_kernel_count() > 10
    assert L.im_kernel_name(0).decode() == "pack_edges"


def test_error_codes_match_binding():
    d = _defines()
    assert d["IM_OK"] == _native.IM_OK
    assert d["IM_EINVAL"] == _native.IM_EINVAL
    assert d["IM_ENOMEM"] == _native.IM_ENOMEM
    assert d["IM_ECUDA"] == _native.IM_ECUDA
    assert d["IM_ESTATE"] == _native.IM_ESTATE
    assert d["IM_ETIMEOUT"] == _native.IM_ETIMEOUT
    assert d["IM_EDEVICE"] == _native.IM_EDEVICE
    assert d["IM_PTR_HOST"] == _native.IM_PTR_HOST and d["IM_PTR_DEVICE"] == _native.IM_PTR_DEVICE


def test_argument_errors_need_no_gpu(libpath):
    # rejected before any CUDA call
    with pytest.raises(im.IMError) as e:
        im.im_create(0, __import__("numpy").zeros(0, "uint32"), __import__("numpy").zeros(0, "uint32"))
    assert e.value.code == _native.IM_EINVAL
    with pytest.raises(im.IMError) as e:
        im.im_autotune(None, 64, 1, 0.05, 0.1, 5)
    assert e.value.code == _native.IM_EINVAL


def test_product_package_never_imports_the_oracle():
    pkg = ROOT / "paper_2311_07554_gb300"
    for f in list(pkg.rglob("*.py")) + list(pkg.rglob("*.cu")) + list(pkg.rglob("*.cuh")):
        t = f.read_text()
        assert "import oracle" not in t and "from oracle" not in t and "im_oracle" not in t, f


@pytest.mark.parametrize("name", ["im_stats", "im_instance", "im_request", "im_tuning", "im_model_stats", "im_batch_schedule"])
def test_struct_layouts_match_the_header(tmp_path, name):
    """The binding's ctypes structs have the header's sizes and field offsets (a C compiler
    reads the header)."""
    import ctypes
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    st = getattr(_native, name)
    fields = [f for f, _ in st._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', f'#include "{HEADER}"', "int main(void) {",
             f'    printf("%zu\\n", sizeof({name}));']
    lines += [f'    printf("%zu\\n", offsetof({name}, {f}));' for f in fields]
    lines += ["    return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-o", str(exe), str(src)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(st)] + [getattr(st, f).offset for f in fields]
    assert got == want
