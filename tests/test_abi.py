"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point that
include/*.h declares; the Python binding names exactly those entry points. No compute calls."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(gmp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_2010_14244_gb300 import build

    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("gmp_create", "gmp_load_graph", "gmp_set_signals", "gmp_set_densities", "gmp_solve",
              "gmp_solve_batch", "gmp_batch_launch", "gmp_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = C.CDLL(built)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(built):
    from paper_2010_14244_gb300 import gmacop

    assert set(gmacop.SIGNATURES) == _declared()
    gmacop.lib()  # binds every signature


def test_strerror_without_gpu(built):
    from paper_2010_14244_gb300 import gmacop

    L = gmacop.lib()
    assert L.gmp_strerror(0) == b"ok"
    assert L.gmp_strerror(gmacop.ERR_NO_ROUTE) == b"no route found"
    assert L.gmp_strerror(12345) == b"unknown error"


def test_context_fails_loudly_without_gpu(built):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2010_14244_gb300 import gmacop

    with pytest.raises(gmacop.GmpError):
        gmacop.Context(0)


def test_built_for_sm_103a():
    from paper_2010_14244_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_header_constants_match_binding_and_oracle():
    """Every GMP_FLAG_*, GMP_MODE_* and GMP_TAU_* value of the header equals the binding's constant of the
    same name, and the flag bits both sides of the parity tests use mean the same on the oracle."""
    from oracle import oracle as orc
    from paper_2010_14244_gb300 import gmacop

    text = "".join(open(h).read() for h in glob.glob(os.path.join(ROOT, "include", "*.h")))
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define GMP_((?:FLAG|MODE|TAU)_\w+) (\d+)u?", text)}
    assert {"FLAG_RANDOM_TAU", "FLAG_REPULSIVE", "FLAG_UNIT_DEPOSIT", "FLAG_EVAP_UNUSED", "FLAG_EXACT_H"} <= set(consts)
    for name, v in consts.items():
        assert getattr(gmacop, name) == v, name
    assert gmacop.FLAG_PAPER_LITERAL == gmacop.FLAG_REPULSIVE | gmacop.FLAG_UNIT_DEPOSIT | gmacop.FLAG_EVAP_UNUSED
    for name in ("FLAG_RANDOM_TAU", "FLAG_REPULSIVE", "FLAG_UNIT_DEPOSIT", "FLAG_EVAP_UNUSED", "FLAG_PAPER_LITERAL",
                 "FLAG_EXACT_H"):
        assert getattr(orc, name) == getattr(gmacop, name), name
