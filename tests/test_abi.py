"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/gakco.h declares; argument validation
that happens before any device work."""

import ctypes
import os
import re

import pytest

import paper_1704_07468_gb300 as pkg
from paper_1704_07468_gb300 import build as lib_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gakco.h")


@pytest.fixture(scope="module")
def lib():
    lib_build.build()
    return pkg.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gakco_\w+)\s*\(", text)))


def test_header_declares_the_interface():
    names = declared_functions()
    for required in ("gakco_create", "gakco_destroy", "gakco_gram",
                     "gakco_gram_device", "gakco_gram_batch_device",
                     "gakco_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_library_is_built_for_sm103a():
    # The build pins one target; the flag must name compute_103a / sm_103a.
    assert "arch=compute_103a,code=sm_103a" in lib_build.ARCH


@pytest.mark.parametrize("sigma,g,k", [(1, 5, 3), (256, 5, 3), (4, 5, 0),
                                       (4, 5, 6), (4, 0, 0), (36, 12, 2),
                                       (4, 33, 5), (4, 20, 2)])
def test_create_rejects_invalid_parameters(lib, sigma, g, k):
    h = ctypes.c_void_p()
    rc = lib.gakco_create(sigma, g, k, ctypes.byref(h))
    assert rc == -1 and not h.value


def test_null_context_is_rejected(lib):
    assert lib.gakco_gram(None, None, None, 0, None, None, None) == -1
    assert lib.gakco_set_option(None, 1, 0) == -1
    lib.gakco_destroy(None)  # no-op


def test_option_and_stat_numbers_match_the_header():
    """The binding's option and statistic keys are the header's values."""
    text = open(HEADER).read()
    opts = {m.group(1).lower(): int(m.group(2))
            for m in re.finditer(r"#define GAKCO_OPT_(\w+)\s+(\d+)", text)}
    stats = {m.group(1).lower(): int(m.group(2))
             for m in re.finditer(r"#define GAKCO_STAT_(\w+)\s+(\d+)", text)}
    assert opts == pkg.OPT
    assert stats == pkg.STAT
