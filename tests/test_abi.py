"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/pic.h; the Python structures match the C layouts. No GPU
work is done here."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in ("pic.h", "unet.h")]


def declared_functions():
    names = set()
    for hdr in HEADERS:
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b((?:pic|unet)_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2606_05893_gb300 import _build
    try:
        _build.nvcc()
    except RuntimeError:
        pytest.skip("no CUDA toolkit")
    _build.build()
    try:
        import paper_2606_05893_gb300 as pkg
        return pkg.load_library()
    except OSError as e:  # no CUDA runtime on this host
        pytest.skip(f"cannot load the CUDA runtime: {e}")


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"pic_create", "pic_inject", "pic_step", "pic_moments", "pic_destroy"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    import paper_2606_05893_gb300 as pkg
    assert set(pkg.EXPORTED) == set(names)


def test_version_and_null_handle_errors(lib):
    import paper_2606_05893_gb300 as pkg
    assert "sm_103a" in pkg.pic_version()
    assert lib.pic_step(None, 1) == pkg.PIC_EINVAL
    assert lib.pic_destroy(None) == pkg.PIC_OK
    assert b"null" in lib.pic_last_error(None)


def test_struct_layouts_match_header(tmp_path):
    import paper_2606_05893_gb300 as pkg
    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "pic.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(pic_species), sizeof(pic_xsec),"
        " sizeof(pic_instance_cfg), sizeof(pic_moments_t), offsetof(pic_instance_cfg, warm_start),"
        " offsetof(pic_moments_t, next_pid)); return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(v) for v in out]
    want = [C.sizeof(pkg.pic_species), C.sizeof(pkg.pic_xsec), C.sizeof(pkg.pic_instance_cfg),
            C.sizeof(pkg.pic_moments_t), pkg.pic_instance_cfg.warm_start.offset, pkg.pic_moments_t.next_pid.offset]
    assert got == want


def test_invalid_configuration_is_rejected_without_gpu_work(lib):
    import paper_2606_05893_gb300 as pkg
    cfg = pkg.pic_instance_cfg()
    cfg.nx = 0  # invalid grid: rejected before any device call
    h = C.c_void_p()
    st = lib.pic_create(C.byref(cfg), 1, None, C.byref(h))
    assert st == pkg.PIC_EINVAL
    assert not h.value


def test_allocator_argument_checks(lib):
    # pic_set_allocator touches no device: exactly one function is refused, both or
    # neither are taken (and neither restores cudaMalloc / cudaFree)
    import paper_2606_05893_gb300 as pkg
    keep = pkg.ALLOC_FN(lambda n, ctx: None)
    assert lib.pic_set_allocator(C.cast(keep, C.c_void_p), None, None) == pkg.PIC_EINVAL
    assert "both" in pkg.pic_last_error(None)
    with pytest.raises(ValueError):
        pkg.pic_set_allocator(lambda n: 0, None)
    pkg.pic_set_allocator(lambda n: 0, lambda p: None)
    pkg.pic_set_allocator()
    assert lib.pic_set_allocator(None, None, None) == pkg.PIC_OK
