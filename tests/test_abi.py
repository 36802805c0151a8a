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


def test_status_strings(lib):
    from paper_1204_5434_gb300 import pft
    for s in range(10):
        assert pft.pft_status_string(s).startswith("PFT_")
