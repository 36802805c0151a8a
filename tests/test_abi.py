"""Host-side tests of the C ABI (no GPU needed): the library builds, loads and exports
every entry point include/pft.h declares, and argument validation fails cleanly
before any device work."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "pft.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pft_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1204_5434_gb300 import build
    build.build()
    from paper_1204_5434_gb300 import pft
    return pft._lib()


def test_header_declares_expected_api():
    names = _declared()
    for must in ("pft_create", "pft_destroy", "pft_set_fields", "pft_solve", "pft_get_observables",
                 "pft_get_densities", "pft_field_step", "pft_gradients", "pft_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1204_5434_gb300 import pft
    assert sorted(pft.exported_symbols()) == _declared()


def test_shape_and_argument_validation(lib):
    from paper_1204_5434_gb300 import pft
    with pytest.raises(pft.PftError) as e:
        pft.pft_create((10, 8, 8), (1, 1, 1), 10, 0.5, 10, 1)
    assert e.value.status == pft.PFT_ERR_SHAPE
    with pytest.raises(pft.PftError) as e:
        pft.pft_create((8, 8, 8), (1, -1, 1), 10, 0.5, 10, 1)
    assert e.value.status == pft.PFT_ERR_ARG
    with pytest.raises(pft.PftError) as e:
        pft.pft_create((8, 8, 8), (1, 1, 1), 0, 0.5, 10, 1)
    assert e.value.status == pft.PFT_ERR_ARG
    with pytest.raises(pft.PftError) as e:
        pft.pft_create((8, 8, 8), (1, 1, 1), 10, 1.5, 10, 1)
    assert e.value.status == pft.PFT_ERR_ARG
    with pytest.raises(pft.PftError) as e:
        pft.pft_create((8, 8, 8), (1, 1, 1), 10, 0.5, 10, 1, precision=7)
    assert e.value.status == pft.PFT_ERR_ARG
    with pytest.raises(pft.PftError) as e:
        pft.pft_create((8, 8, 8), (1, 1, 1), 10, 0.5, 10, 1, scheme=5)
    assert e.value.status == pft.PFT_ERR_ARG
    with pytest.raises(pft.PftError) as e:
        pft.pft_create((8, 8, 8), (1, 1, 1), 10, 0.5, 10, 1, checkpoint=-1)
    assert e.value.status == pft.PFT_ERR_ARG
    with pytest.raises(pft.PftError) as e:
        pft.pft_create((8, 8, 8), (1, 1, 1), 10, 0.5, 10, 1, checkpoint=3, scheme=pft.PFT_SCHEME_RQM4)
    assert e.value.status == pft.PFT_ERR_UNSUPPORTED
    with pytest.raises(pft.PftError) as e:
        pft.pft_create((64, 64, 64), (1, 1, 1), 10, 0.5, 10, 1, precision=pft.PFT_FP32_MIXED, march=2)
    assert e.value.status == pft.PFT_ERR_ARG


def test_status_strings(lib):
    from paper_1204_5434_gb300 import pft
    for s in range(10):
        assert pft.pft_status_string(s).startswith("PFT_")


_LAYOUT_PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "pft.h"
#define S(T) printf(#T " size %zu\n", sizeof(T));
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  S(pft_grid) F(pft_grid, L)
  S(pft_chain) F(pft_chain, fA)
  S(pft_model) F(pft_model, C) F(pft_model, kind) F(pft_model, arch) F(pft_model, B)
  S(pft_opts) F(pft_opts, use_graph) F(pft_opts, stream) F(pft_opts, seed) F(pft_opts, instance)
  F(pft_opts, march) F(pft_opts, scheme) F(pft_opts, checkpoint)
  F(pft_opts, autotune)
  S(pft_obs) F(pft_obs, lnQ) F(pft_obs, H) F(pft_obs, h) F(pft_obs, phiA_mean) F(pft_obs, phiB_mean)
  F(pft_obs, force_p_rms) F(pft_obs, force_m_rms) F(pft_obs, fA_eff) F(pft_obs, NsA) F(pft_obs, step)
  S(pft_instance_desc) F(pft_instance_desc, chain) F(pft_instance_desc, model) F(pft_instance_desc, seed)
  S(pft_profile)
  return 0;
}
"""


def test_binding_struct_layouts_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets that a C
    compiler gives the header's declarations."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1204_5434_gb300 import pft
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_PROBE)
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            key, val = line.rsplit(" ", 1)
            got[key] = int(val)
    import ctypes as ct
    for key, val in got.items():
        if key.endswith(" size"):
            name = key[:-5]
            assert ct.sizeof(getattr(pft, name)) == val, key
        else:
            name, field = key.split(".")
            assert getattr(getattr(pft, name), field).offset == val, key
