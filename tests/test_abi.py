"""CPU checks of the C ABI: the library loads, exports every symbol the header
declares, and rejects bad configurations with error codes (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2211_16278_gb300 as pkg
from paper_2211_16278_gb300 import bblock as bbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bblock.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bblock_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return pkg.load()


def test_header_declares_the_binding_symbols():
    assert declared_symbols() == sorted(bbm.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(bbm.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(raw, name), f"{name} missing from {bbm.LIB_PATH}"


def test_config_struct_matches_header():
    text = open(HEADER).read()
    body = re.search(r"typedef struct \{([^}]*)\} bblock_config;", text, re.S).group(1)
    fields = re.findall(r"int\s+(\w+);", re.sub(r"/\*.*?\*/", "", body, flags=re.S))
    assert fields == [f for f, _ in bbm.bblock_config._fields_]
    body = re.search(r"typedef struct \{([^}]*)\} bblock_job;", text, re.S).group(1)
    names = re.findall(r"(\w+)[,;]", re.sub(r"/\*.*?\*/", "", body, flags=re.S))
    assert names == [f for f, _ in bbm.bblock_job._fields_]


@pytest.mark.parametrize("cfg", [
    dict(L=0, n_ev=1, max_ndil=1),
    dict(L=2, n_ev=25, max_ndil=1),         # n_ev > 3 L^3
    dict(L=2, n_ev=4, max_ndil=0),
    dict(L=2, n_ev=4, max_ndil=300),
    dict(L=2, n_ev=4, max_ndil=8, precision=7),
    dict(L=2, n_ev=4, max_ndil=8, precision=2, bf16_products=4),
])
def test_create_rejects_bad_config_before_touching_a_device(lib, cfg):
    c = bbm.bblock_config(cfg["L"], cfg["n_ev"], cfg["max_ndil"], cfg.get("precision", 0),
                          cfg.get("bf16_products", 6), 0)
    h = ctypes.c_void_p()
    assert lib.bblock_create(ctypes.byref(h), ctypes.byref(c)) == -1
    assert not h.value


def test_null_arguments_are_rejected(lib):
    assert lib.bblock_create(None, None) == -1
    assert lib.bblock_status(None) == -1
    lib.bblock_destroy(None)  # no-op
    assert lib.bblock_last_launch_count(None) == 0


def header_defines(prefix):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {m.group(1): int(m.group(2))
            for m in re.finditer(rf"#define\s+{prefix}(\w+)\s+\(?(-?\d+)\)?", text)}


def test_binding_options_and_precisions_match_header():
    """The binding's option and precision names map to the header's values, one for one."""
    opts = {k.lower(): v for k, v in header_defines("BBLOCK_OPT_").items()}
    assert opts == bbm.OPTIONS
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    enum = re.search(r"typedef enum \{([^}]*)\} bblock_precision;", text, re.S).group(1)
    precisions = {m.group(1).lower(): int(m.group(2))
                  for m in re.finditer(r"BBLOCK_(\w+)\s*=\s*(\d+)", enum)}
    assert precisions == {"fp64": 0, "tf32x3": 1, "bf16_split": 2, "df64": 3, "fp16x3": 4,
                          "ozaki": 5}
    for name in ("fp64", "tf32x3", "df64", "fp16x3", "ozaki"):
        assert bbm.PRECISIONS[name] == precisions[name]
    assert bbm.PRECISIONS["bf16"] == precisions["bf16_split"]
