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


def test_static_reports_neighbour_overflow(torch_cuda):
    """A dense non-periodic cluster (a 7 x 7 x 7 grid, 1 A apart) with rc = 12 A gives every
    atom 342 neighbours, more than the 256 slots per atom of the static scratch.  The
    neighbour kernel writes only the slots below the capacity, so the call is bounded and
    must report the overflow with the atom and its neighbour count."""
    torch = torch_cuda
    g = np.arange(7, dtype=np.float64)
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    n = len(pos)
    system = W.System(np.array([0, n], np.int64), pos, np.zeros(n, np.int32), np.zeros((1, 9)),
                      np.zeros((1, 3), np.uint8), 1)
    desc = W.descriptor_params(1, 12.0, 8, 4, 4)
    sysd = P.DeviceSystem(system)
    G = torch.empty((n, desc.D), dtype=torch.float32, device="cuda")
    with pytest.raises(P.PannaError) as ei:
        P.panna_descriptors_static(desc, sysd, G)
    assert ei.value.status == P.PANNA_ERR_NEIGHBOR_OVERFLOW
    msg = P.load().panna_last_error().decode()
    assert "342 neighbours" in msg and "atom" in msg, msg
    # the scratch is usable again afterwards
    wl = W.make("diamond64")
    sd = P.DeviceSystem(wl.system)
    pot = P.Potential(wl.desc, wl.archs)
    G_ref = pot.descriptors(sd).cpu().numpy().astype(np.float64)
    G2 = torch.empty((sd.n_atoms, pot.D), dtype=torch.float32, device="cuda")
    P.panna_descriptors_static(wl.desc, sd, G2)
    torch.cuda.synchronize()
    assert H.descriptor_error(G2.cpu().numpy().astype(np.float64), G_ref, wl.desc) <= H.TOL_G


def test_static_checks_the_output_buffer(torch_cuda):
    torch = torch_cuda
    wl = W.make("diamond64")
    sysd = P.DeviceSystem(wl.system)
    with pytest.raises(ValueError):
        P.panna_descriptors_static(wl.desc, sysd, torch.empty((sysd.n_atoms, wl.desc.D - 1), device="cuda"))
    with pytest.raises(ValueError):
        P.panna_descriptors_static(wl.desc, sysd, torch.empty((sysd.n_atoms, wl.desc.D), dtype=torch.float64,
                                                              device="cuda"))
