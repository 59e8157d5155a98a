"""C ABI checks that need no GPU: the library builds, loads and exports every
function include/sf.h declares; the binding covers exactly those; invalid
configurations are rejected on the host before any CUDA call."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sf.h")


@pytest.fixture(scope="module")
def libsf():
    from paper_1507_04941_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sf_[a-z_0-9]+)\s*\(", text)))


def test_header_compiles_as_plain_c(tmp_path):
    src = tmp_path / "use.c"
    src.write_text('#include "sf.h"\nint main(void){ sf_config c; (void)c; return 0; }\n')
    res = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                          "-fsyntax-only", str(src)], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr


def test_every_declared_symbol_is_exported(libsf):
    handle, path = libsf
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(handle, n), f"{n} declared in sf.h but not exported by {path}"
    dyn = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sf_\w+)", dyn))
    assert set(names) <= exported


def test_binding_covers_exactly_the_header():
    from paper_1507_04941_gb300 import sf
    assert sorted(sf.SIGNATURES) == declared_functions()


def test_status_strings(libsf):
    from paper_1507_04941_gb300 import sf
    lib = sf.lib()
    for code, name in enumerate(["SF_OK", "SF_EINVAL", "SF_ENOMEM", "SF_EBUDGET", "SF_ECUDA",
                                 "SF_ETIMEOUT", "SF_ESTATE", "SF_EJIT", "SF_ECANCELED"]):
        assert lib.sf_status_str(code).decode() == name


def _cfg(sf, **kw):
    bank = kw.pop("bank", ((1.0, 2.0),))
    specs = (sf.FilterSpec * max(1, len(bank)))(*[sf.FilterSpec(a, b) for a, b in bank])
    vals = dict(nx=16, ny=16, nz=32, n_filters=len(bank), filters=specs, truncation=3.0, wx=8,
                wy=8, wz=32, k=4.0, storage=0, stats_fp64=0, device=-1)
    vals.update(kw)
    return sf.Config(**vals), specs


@pytest.mark.parametrize("bad", [dict(nx=0), dict(ny=0), dict(nz=-3), dict(nx=2 ** 31 + 1),
                                 dict(n_filters=0), dict(truncation=0.0),
                                 dict(wx=0), dict(storage=7), dict(stats_fp64=2), dict(std_ddof=2),
                                 dict(bank=((-1.0, 2.0),)), dict(bank=((1.0, 40.0),)),
                                 dict(filters=None)])
def test_invalid_config_rejected_on_host(libsf, bad):
    from paper_1507_04941_gb300 import sf
    lib = sf.lib()
    cfg, _keep = _cfg(sf, **bad)
    h = ctypes.c_void_p()
    st = lib.sf_create(ctypes.byref(cfg), ctypes.byref(h))
    assert st == sf.SF_EINVAL
    assert not h.value
    assert lib.sf_last_error(None).decode()


@pytest.mark.parametrize("dims", [(0, 4, 8), (4, 0, 8), (4, 4, 0), (4, 4, -1), (2 ** 31 + 1, 1, 1)])
def test_batch_with_an_empty_or_oversized_cube_rejected_on_host(libsf, dims):
    """An empty cube (a zero extent) has no windows: a batch holding one is
    refused before any device work, as is an extent above 2^31."""
    from paper_1507_04941_gb300 import sf
    lib = sf.lib()
    cfg, _keep = _cfg(sf)
    arr = (ctypes.c_int64 * 6)(16, 16, 32, *dims)
    h = ctypes.c_void_p()
    assert lib.sf_create_batch(ctypes.byref(cfg), 2, arr, ctypes.byref(h)) == sf.SF_EINVAL
    assert not h.value
    assert "dimensions" in lib.sf_last_error(None).decode()


def test_create_without_gpu_reports_cuda_error(libsf):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1507_04941_gb300 import sf
    lib = sf.lib()
    cfg, _keep = _cfg(sf)
    h = ctypes.c_void_p()
    assert lib.sf_create(ctypes.byref(cfg), ctypes.byref(h)) == sf.SF_ECUDA
    assert not h.value


def test_null_arguments(libsf):
    from paper_1507_04941_gb300 import sf
    lib = sf.lib()
    h = ctypes.c_void_p()
    assert lib.sf_create(None, ctypes.byref(h)) == sf.SF_EINVAL
    assert lib.sf_destroy(None) == sf.SF_OK
    assert lib.sf_detect(None, None, None, None, None, None) == sf.SF_EINVAL
    assert lib.sf_mask_words(None, None) == sf.SF_EINVAL


def test_server_invalid_arguments(libsf):
    from paper_1507_04941_gb300 import sf
    lib = sf.lib()
    cfg, _keep = _cfg(sf)
    h = ctypes.c_void_p()
    assert lib.sf_server_create(ctypes.byref(cfg), 0, 4, ctypes.byref(h)) == sf.SF_EINVAL
    assert lib.sf_server_create(ctypes.byref(cfg), 10 ** 9, 0, ctypes.byref(h)) == sf.SF_EINVAL
    assert lib.sf_server_create(None, 10 ** 9, 4, ctypes.byref(h)) == sf.SF_EINVAL
    assert lib.sf_server_destroy(None) == sf.SF_OK
    n = ctypes.c_int32()
    assert lib.sf_server_poll(None, None, None, None, 0, 0, ctypes.byref(n)) == sf.SF_EINVAL


@pytest.mark.parametrize("section,bad", [(0, {}), (12, {}), (-8, {}), (16, dict(wx=0)),
                                         (16, dict(bank=((float("nan"), 2.0),))),
                                         (16, dict(filters=None)), (16, dict(truncation=0.0))])
def test_sectioned_arguments_rejected_on_host(libsf, section, bad):
    """A section must be a positive multiple of wx (wx = 8 here); the bank is
    checked before any device work."""
    from paper_1507_04941_gb300 import sf
    lib = sf.lib()
    cfg, _keep = _cfg(sf, **bad)
    h = ctypes.c_void_p()
    assert lib.sf_create_sectioned(ctypes.byref(cfg), section, ctypes.byref(h)) == sf.SF_EINVAL
    assert not h.value
    assert lib.sf_create_sectioned(None, 16, ctypes.byref(h)) == sf.SF_EINVAL


def test_no_fallback_without_the_library(tmp_path):
    """Without libsf.so every entry point raises: there is no CPU path."""
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_1507_04941_gb300 import sf\n"
        "sf.library_path = lambda: %r\n"
        "sf._lib = None\n"
        "try:\n"
        "    sf.lib()\n"
        "except RuntimeError as e:\n"
        "    print('raised', 'not built' in str(e))\n"
        "else:\n"
        "    print('loaded')\n"
    ) % (ROOT, str(tmp_path / "missing" / "libsf.so"))
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert res.stdout.strip() == "raised True", res.stdout + res.stderr
