"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/lbm.h declares; the binding's structs match the header's sizes.
No compute calls (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1111_0922_gb300 import build, lbm

    build.build()
    return lbm.load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)) - {"lbm_alloc_fn", "lbm_free_fn"})


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("lbm_create", "lbm_set_geometry", "lbm_step", "lbm_macroscopics", "lbm_destroy"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1111_0922_gb300 import lbm

    for name in _declared():
        assert hasattr(lib, name), name
        assert name in lbm.SIGNATURES, "binding lacks %s" % name


def _c_layout(tmp_path, struct, fields):
    """sizeof and offsetof of a header struct as the C compiler lays it out."""
    import subprocess

    src = tmp_path / "layout.c"
    body = "".join('printf("%%zu\\n", offsetof(%s, %s));' % (struct, f) for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\n'
                   'int main(void) { printf("%%zu\\n", sizeof(%s)); %s return 0; }\n' % (struct, body))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.parametrize("name", ["lbm_config", "lbm_info", "lbm_batch_config", "lbm_batch_info"])
def test_struct_layouts_match_header(lib, tmp_path, name):
    """Every ctypes struct of the binding has the size and field offsets the
    C compiler gives the header's struct."""
    from paper_1111_0922_gb300 import lbm

    cls = getattr(lbm, name)
    fields = [f[0] for f in cls._fields_]
    size, offs = _c_layout(tmp_path, name, fields)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offs


def test_host_only_calls(lib):
    """Calls that need no device: defaults, status strings, argument checks."""
    from paper_1111_0922_gb300 import lbm

    cfg = lbm.lbm_config_default()
    assert (cfg.nx, cfg.variant, cfg.precision) == (32, lbm.LBM_AA, lbm.LBM_F32)
    assert lib.lbm_status_string(lbm.LBM_ERR_STATE) == b"invalid state"
    bad = lbm.lbm_config_default()
    bad.omega = 2.5
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_create(bad)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    bad = lbm.lbm_config_default()
    bad.periodic[1] = 1
    bad.ny = 1
    with pytest.raises(lbm.LBMError):
        lbm.lbm_create(bad)
    for variant, layout in ((lbm.LBM_AA, lbm.LBM_SOA), (lbm.LBM_OS_PULL, lbm.LBM_AOS)):
        bad = lbm.lbm_config_default()
        bad.variant, bad.layout, bad.store_hint = variant, layout, 1
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_create(bad)
        assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    bad = lbm.lbm_config_default()
    bad.swap_schedule = 3
    with pytest.raises(lbm.LBMError):
        lbm.lbm_create(bad)
    bad = lbm.lbm_config_default()
    bad.pair_z = 3
    with pytest.raises(lbm.LBMError):
        lbm.lbm_create(bad)
    assert lib.lbm_destroy(None) == 0


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1111_0922_gb300 import lbm

    with pytest.raises(RuntimeError):
        lbm.load.__wrapped__ if hasattr(lbm.load, "__wrapped__") else None
        saved = lbm._lib
        lbm._lib = None
        try:
            lbm.load(str(tmp_path / "missing.so"))
        finally:
            lbm._lib = saved
