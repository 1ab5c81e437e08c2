"""panna_descriptors_static: descriptors without any device allocation.

Some callers of this library cannot allocate device memory: a host program whose own
memory pool already owns the whole GPU, or a callback (a force call made from inside
another code's time step) in which new device allocations are forbidden.  For them the
library offers one entry point whose scratch lives in a static device array.  These
tests call it through the C ABI and check that it gives the same descriptors as the
ordinary (allocating) entry point, on two calls in a row, and that repeated calls leave
the device's free memory unchanged.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2305_11805_gb300 import panna as P
from paper_2305_11805_gb300 import workloads as W
from tests import gpu_common as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_11805_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("name", ["diamond64", "molecules16", "ragged8"])
def test_static_descriptors_match_allocating_entry_point(torch_cuda, name):
    torch = torch_cuda
    wl = W.make(name)
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    G_ref = pot.descriptors(sysd).cpu().numpy().astype(np.float64)
    for _ in range(2):
        G = torch.full((sysd.n_atoms, pot.D), float("nan"), dtype=torch.float32, device="cuda")
        P.panna_descriptors_static(wl.desc, sysd, G)
        torch.cuda.synchronize()
        err = H.descriptor_error(G.cpu().numpy().astype(np.float64), G_ref, wl.desc)
        assert err <= H.TOL_G, err


def test_static_calls_allocate_nothing(torch_cuda):
    torch = torch_cuda
    wl = W.make("water512")
    sysd = P.DeviceSystem(wl.system)
    G = torch.empty((sysd.n_atoms, wl.desc.D), dtype=torch.float32, device="cuda")
    P.panna_descriptors_static(wl.desc, sysd, G)     # first call on this device: address lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        P.panna_descriptors_static(wl.desc, sysd, G)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_rejects_batches_beyond_its_scratch(torch_cuda):
    wl = W.make("diamond64")
    sysd = P.DeviceSystem(wl.system)
    big = P.panna_system(1, 10_000_000, sysd.s.atom_off, sysd.s.pos, sysd.s.species, sysd.s.cell, sysd.s.pbc)
    h = P._DescHolder(wl.desc)
    st = P.load().panna_descriptors_static(ctypes.byref(h.s), ctypes.byref(big), sysd.s.pos, None)
    assert st == P.PANNA_ERR_INVALID_ARG
    assert b"static" in P.load().panna_last_error()
