"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and exports every
function that include/panna_gb300.h declares; host-side parameter logic needs no GPU."""
import os
import re

import pytest

from paper_2305_11805_gb300 import build as B
from paper_2305_11805_gb300 import panna as P
from paper_2305_11805_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "panna_gb300.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(panna_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert "panna_energy_forces" in names and "panna_loss_grad" in names
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(P.exported_symbols()) == names


def test_descriptor_size_matches_paper_sizes(lib):
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "descriptor_sizes.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        S, nr, nt, na, D = map(int, r[:5])
        assert P.panna_descriptor_size(W.descriptor_params(S, 5.0, nr, nt, na)) == D


def test_descriptor_size_rejects_invalid(lib):
    d = W.descriptor_params(9, 5.0, 8, 8, 8)   # more than 8 species
    assert P.panna_descriptor_size(d) == -1


def test_version_string(lib):
    assert "sm_103a" in P.panna_version()


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    w = W.make("diamond64")
    with pytest.raises(P.PannaError):
        P.panna_create(w.desc, w.archs)
