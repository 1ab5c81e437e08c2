"""Thin Python binding of libpanna_gb300 (ctypes).

Argument marshalling only: every step of the path runs in the CUDA kernels of the
library.  Functions keep the C names (``panna_create``, ``panna_energy_forces``, ...);
:class:`Potential` bundles a context with device copies of a workload for convenience.
Device buffers are torch CUDA tensors (torch provides memory and streams only).

Importing this module does not need a GPU; loading the library does, and it fails
loudly when the shared library has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpanna_gb300.so")
MAX_LAYERS = 8

PANNA_OK, PANNA_ERR_INVALID_ARG, PANNA_ERR_UNSUPPORTED, PANNA_ERR_NEIGHBOR_OVERFLOW = 0, 1, 2, 3
PANNA_ERR_TIMEOUT, PANNA_ERR_CUDA, PANNA_ERR_NO_MEMORY, PANNA_ERR_BAD_INPUT = 4, 5, 6, 7
PANNA_MLP_FP32, PANNA_MLP_BF16, PANNA_MLP_BF16_FAST = 0, 1, 2

_dp = C.POINTER(C.c_double)
_vp = C.c_void_p


class panna_desc_params(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("rc", C.c_double),
                ("n_rad", C.c_int32), ("rs_rad", _dp), ("eta_rad", C.c_double),
                ("n_ang_r", C.c_int32), ("rs_ang", _dp),
                ("n_theta", C.c_int32), ("theta_s", _dp),
                ("eta_ang", C.c_double), ("zeta", C.c_double), ("eps_theta", C.c_double),
                ("angular_kind", C.c_int32), ("bp_lambda", _dp), ("bp_zeta", _dp), ("bp_eta", _dp)]


PANNA_ANGULAR_MBP, PANNA_ANGULAR_BP = 0, 1


class panna_mlp_arch(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("widths", C.c_int32 * (MAX_LAYERS + 1)),
                ("act", C.c_int32 * MAX_LAYERS)]


class panna_system(C.Structure):
    _fields_ = [("n_cfg", C.c_int64), ("n_atoms", C.c_int64), ("atom_off", _vp), ("pos", _vp),
                ("species", _vp), ("cell", _vp), ("pbc", _vp), ("ghost", _vp)]


class panna_md_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("temperature", C.c_double), ("friction", C.c_double), ("skin", C.c_double),
                ("mass", C.POINTER(C.c_double)), ("seed", C.c_uint64), ("step0", C.c_int64)]


class panna_loss_options(C.Structure):
    _fields_ = [("energy_loss", C.c_int32), ("force_loss", C.c_int32), ("energy_per_atom", C.c_int32),
                ("l1", C.c_double), ("l2", C.c_double)]


class panna_adam_params(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("decay_rate", C.c_double), ("decay_steps", C.c_double)]


PANNA_LOSS_QUADRATIC, PANNA_LOSS_EXPONENTIAL = 0, 1


class panna_qeq_params(C.Structure):
    _fields_ = [("sigma", _vp), ("chi0", _vp), ("hard0", _vp), ("k_coulomb", C.c_double)]


class panna_store_info(C.Structure):
    _fields_ = [("n_atoms", C.c_int64), ("n_cfg", C.c_int64), ("n_entries", C.c_int64), ("D", C.c_int32),
                ("width", C.c_int32), ("bytes", C.c_int64)]


STORE_SECTIONS = ("G", "row_of_atom", "atom_of_row", "seg_off", "atom_cfg", "ent_off", "ent_idx", "ent_vec", "jac")


class PannaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("panna status %d: %s" % (status, msg))
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libpanna_gb300.so not found at %s: run __graft_entry__.build() "
                           "(there is no CPU fallback)" % path)
    L = C.CDLL(path)
    i32, i64, f32, f64 = C.c_int32, C.c_int64, C.c_float, C.c_double
    sig = {
        "panna_version": (C.c_char_p, []),
        "panna_last_error": (C.c_char_p, []),
        "panna_descriptor_size": (i64, [C.POINTER(panna_desc_params)]),
        "panna_create": (i32, [C.POINTER(panna_desc_params), i32, C.POINTER(panna_mlp_arch), C.POINTER(_vp)]),
        "panna_destroy": (None, [_vp]),
        "panna_param_count": (i64, [_vp]),
        "panna_set_neighbor_capacity": (i32, [_vp, i32]),
        "panna_neighbor_capacity": (i32, [_vp]),
        "panna_set_async": (i32, [_vp, i32]),
        "panna_check": (i32, [_vp, _vp]),
        "panna_set_angular_precision": (i32, [_vp, i32]),
        "panna_set_tuning": (i32, [_vp, C.c_char_p, i32]),
        "panna_tuning_choice": (i32, [_vp, C.c_char_p]),
        "panna_set_loss_normalization": (i32, [_vp, i64, i64]),
        "panna_set_loss_options": (i32, [_vp, C.POINTER(panna_loss_options)]),
        "panna_set_frozen": (i32, [_vp, i32, i32, i32]),
        "panna_adam_step": (i32, [_vp, _vp, _vp, _vp, _vp, i64, C.POINTER(panna_adam_params), _vp]),
        "panna_md_run": (i32, [_vp, C.POINTER(panna_system), _vp, _vp, i32, C.POINTER(panna_md_params), i64, _vp,
                               i32, _vp, _vp, C.POINTER(i64), _vp]),
        "panna_neighbors": (i32, [_vp, C.POINTER(panna_system), i64, _vp, _vp, _vp, C.POINTER(i64), _vp]),
        "panna_descriptors": (i32, [_vp, C.POINTER(panna_system), _vp, _vp]),
        "panna_energy_forces": (i32, [_vp, C.POINTER(panna_system), _vp, i32, _vp, _vp, _vp, _vp, _vp]),
        "panna_param_vjp": (i32, [_vp, C.POINTER(panna_system), _vp, _vp, _vp, _vp, _vp]),
        "panna_loss_grad": (i32, [_vp, C.POINTER(panna_system), _vp, _vp, _vp, f64, _vp, _vp, _vp, _vp, _vp]),
        "panna_last_launch_count": (i32, [_vp]),
        "panna_set_profiling": (i32, [_vp, i32]),
        "panna_stage_ms": (f32, [_vp, C.c_char_p]),
        "panna_descriptors_static": (i32, [C.POINTER(panna_desc_params), C.POINTER(panna_system), _vp, _vp]),
        "panna_measure_alu_peaks": (i32, [C.POINTER(f64), C.POINTER(f64), _vp]),
        "panna_measure_alu_peaks2": (i32, [C.POINTER(f64), C.POINTER(f64), C.POINTER(f64), _vp]),
        "panna_capture": (i32, [_vp, C.POINTER(panna_system), _vp, i32, _vp, _vp, _vp, _vp, _vp]),
        "panna_replay": (i32, [_vp, _vp]),
        "panna_set_qeq": (i32, [_vp, C.POINTER(panna_qeq_params)]),
        "panna_qeq_energy_forces": (i32, [_vp, C.POINTER(panna_system), _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "panna_qeq_loss_grad": (i32, [_vp, C.POINTER(panna_system), _vp, _vp, _vp, _vp, f64, _vp, f64, _vp, _vp, _vp,
                                      _vp, _vp, _vp]),
        "panna_store_plan": (i32, [_vp, C.POINTER(panna_system), C.POINTER(panna_store_info), _vp]),
        "panna_store_sections": (i32, [_vp, C.POINTER(panna_store_info), C.POINTER(i64)]),
        "panna_store_build": (i32, [_vp, C.POINTER(panna_system), C.POINTER(panna_store_info), _vp, _vp]),
        "panna_store_energy_forces": (i32, [_vp, C.POINTER(panna_system), C.POINTER(panna_store_info), _vp, _vp,
                                            i32, _vp, _vp, _vp, _vp, _vp]),
        "panna_store_loss_grad": (i32, [_vp, C.POINTER(panna_system), C.POINTER(panna_store_info), _vp, _vp, _vp,
                                        _vp, f64, _vp, _vp, _vp, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def exported_symbols() -> Sequence[str]:
    return ["panna_version", "panna_last_error", "panna_descriptor_size", "panna_create", "panna_destroy",
            "panna_param_count", "panna_set_neighbor_capacity", "panna_neighbor_capacity", "panna_set_async",
            "panna_check", "panna_set_angular_precision", "panna_set_tuning", "panna_tuning_choice", "panna_set_loss_normalization",
            "panna_md_run", "panna_set_loss_options", "panna_set_frozen", "panna_adam_step",
            "panna_neighbors", "panna_descriptors", "panna_energy_forces", "panna_param_vjp",
            "panna_loss_grad", "panna_last_launch_count", "panna_set_profiling", "panna_stage_ms",
            "panna_descriptors_static", "panna_measure_alu_peaks", "panna_measure_alu_peaks2", "panna_capture", "panna_replay", "panna_store_plan",
            "panna_store_sections", "panna_store_build", "panna_store_energy_forces", "panna_store_loss_grad",
            "panna_set_qeq", "panna_qeq_energy_forces", "panna_qeq_loss_grad"]


def _check(status: int):
    if status != PANNA_OK:
        raise PannaError(status, load().panna_last_error().decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _dev(t, dtype: str, numel: int, name: str):
    """Pointer of a caller-owned device buffer after checking what the C ABI will assume of
    it: a contiguous CUDA tensor of `dtype` (torch dtype name) on the current device holding
    exactly `numel` elements.  The kernels write every element, so a smaller buffer would be
    overwritten past its end."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if str(t.dtype) != "torch." + dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() != numel:
        raise ValueError("%s must hold %d elements, got %d" % (name, numel, t.numel()))
    if t.device.index != torch.cuda.current_device():
        raise ValueError("%s is on cuda:%d, the current device is cuda:%d" % (
            name, t.device.index, torch.cuda.current_device()))
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


# ---------------------------------------------------------------------------- C names

class _DescHolder:
    def __init__(self, d):
        self.rs_rad = np.ascontiguousarray(d.rs_rad, np.float64)
        self.rs_ang = np.ascontiguousarray(d.rs_ang, np.float64)
        self.theta_s = np.ascontiguousarray(d.theta_s, np.float64)
        bp = getattr(d, "angular", "mbp") == "bp"
        self.bp = [np.ascontiguousarray(a, np.float64) for a in (d.bp_lambda, d.bp_zeta, d.bp_eta)] if bp else []
        bp_ptrs = [a.ctypes.data_as(_dp) for a in self.bp] if bp else [None, None, None]
        self.s = panna_desc_params(
            int(d.n_species), float(d.rc), len(self.rs_rad), self.rs_rad.ctypes.data_as(_dp), float(d.eta_rad),
            int(d.n_ang_r), self.rs_ang.ctypes.data_as(_dp), int(d.n_theta),
            self.theta_s.ctypes.data_as(_dp), float(d.eta_ang), float(d.zeta), float(d.eps_theta),
            PANNA_ANGULAR_BP if bp else PANNA_ANGULAR_MBP, *bp_ptrs)


def panna_descriptor_size(desc) -> int:
    h = _DescHolder(desc)
    return int(load().panna_descriptor_size(C.byref(h.s)))


def panna_create(desc, archs) -> int:
    h = _DescHolder(desc)
    arr = (panna_mlp_arch * len(archs))()
    for k, a in enumerate(archs):
        arr[k].n_layers = a.n_layers
        for l, w in enumerate(a.widths):
            arr[k].widths[l] = int(w)
        for l, t in enumerate(a.acts):
            arr[k].act[l] = int(t)
    out = _vp()
    _check(load().panna_create(C.byref(h.s), len(archs), arr, C.byref(out)))
    return out.value


def panna_destroy(ctx: int):
    load().panna_destroy(ctx)


def panna_param_count(ctx: int) -> int:
    return int(load().panna_param_count(ctx))


def panna_set_neighbor_capacity(ctx: int, cap: int):
    _check(load().panna_set_neighbor_capacity(ctx, int(cap)))


def panna_neighbor_capacity(ctx: int) -> int:
    return int(load().panna_neighbor_capacity(ctx))


def panna_set_async(ctx: int, on: bool):
    _check(load().panna_set_async(ctx, 1 if on else 0))


def panna_set_angular_precision(ctx: int, mode: int):
    _check(load().panna_set_angular_precision(ctx, int(mode)))


def panna_set_tuning(ctx: int, knob: str, value: int):
    _check(load().panna_set_tuning(ctx, knob.encode(), int(value)))


def panna_tuning_choice(ctx: int, knob: str) -> int:
    return int(load().panna_tuning_choice(ctx, knob.encode()))


def panna_set_loss_normalization(ctx: int, n_cfg_total: int, n_atoms_total: int):
    _check(load().panna_set_loss_normalization(ctx, int(n_cfg_total), int(n_atoms_total)))


def panna_md_run(ctx: int, sysd: "DeviceSystem", vel, theta, prec: int, dt: float, temperature: float,
                 friction: float, skin: float, mass, seed: int, step0: int, n_steps: int, F, forces_valid: bool,
                 E_cfg, E_traj=None, stream=None) -> int:
    """Langevin dynamics (see the header); moves sysd.pos in place, returns the number of
    neighbour searches."""
    m = (C.c_double * len(mass))(*[float(x) for x in mass])
    prm = panna_md_params(float(dt), float(temperature), float(friction), float(skin),
                          C.cast(m, C.POINTER(C.c_double)), int(seed), int(step0))
    nb = C.c_int64(0)
    _check(load().panna_md_run(ctx, C.byref(sysd.s), _ptr(vel), _ptr(theta), int(prec), C.byref(prm), int(n_steps),
                               _ptr(F), 1 if forces_valid else 0, _ptr(E_cfg), _ptr(E_traj), C.byref(nb),
                               _stream(stream)))
    return int(nb.value)


def panna_set_loss_options(ctx: int, energy_loss=0, force_loss=0, energy_per_atom=False, l1=0.0, l2=0.0):
    o = panna_loss_options(int(energy_loss), int(force_loss), 1 if energy_per_atom else 0, float(l1), float(l2))
    _check(load().panna_set_loss_options(ctx, C.byref(o)))


def panna_set_frozen(ctx: int, species: int, layer: int, frozen: bool):
    _check(load().panna_set_frozen(ctx, int(species), int(layer), 1 if frozen else 0))


def panna_adam_step(ctx: int, theta, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8,
                    decay_rate=1.0, decay_steps=0.0, stream=None):
    a = panna_adam_params(float(lr), float(beta1), float(beta2), float(eps), float(decay_rate), float(decay_steps))
    _check(load().panna_adam_step(ctx, _ptr(theta), _ptr(grad), _ptr(m), _ptr(v), int(t), C.byref(a),
                                  _stream(stream)))


def panna_check(ctx: int, stream=None):
    _check(load().panna_check(ctx, _stream(stream)))


def panna_neighbors(ctx: int, sysd: "DeviceSystem", cap_total: int, nbr_off, nbr_j, nbr_shift, stream=None) -> int:
    n = C.c_int64(0)
    _check(load().panna_neighbors(ctx, C.byref(sysd.s), int(cap_total), _ptr(nbr_off), _ptr(nbr_j),
                                  _ptr(nbr_shift), C.byref(n), _stream(stream)))
    return int(n.value)


def panna_descriptors(ctx: int, sysd: "DeviceSystem", G, stream=None):
    _check(load().panna_descriptors(ctx, C.byref(sysd.s), _ptr(G), _stream(stream)))


def panna_energy_forces(ctx: int, sysd: "DeviceSystem", theta, prec: int, E_cfg, E_atom, F, virial, stream=None):
    _check(load().panna_energy_forces(ctx, C.byref(sysd.s), _ptr(theta), int(prec), _ptr(E_cfg), _ptr(E_atom),
                                      _ptr(F), _ptr(virial), _stream(stream)))


def panna_param_vjp(ctx: int, sysd: "DeviceSystem", theta, dE, dF, dtheta, stream=None):
    _check(load().panna_param_vjp(ctx, C.byref(sysd.s), _ptr(theta), _ptr(dE), _ptr(dF), _ptr(dtheta),
                                  _stream(stream)))


def panna_loss_grad(ctx: int, sysd: "DeviceSystem", theta, E_ref, F_ref, w_force: float, loss, dtheta,
                    E_cfg=None, F=None, stream=None):
    _check(load().panna_loss_grad(ctx, C.byref(sysd.s), _ptr(theta), _ptr(E_ref), _ptr(F_ref), float(w_force),
                                  _ptr(loss), _ptr(dtheta), _ptr(E_cfg), _ptr(F), _stream(stream)))


def panna_last_launch_count(ctx: int) -> int:
    return int(load().panna_last_launch_count(ctx))


def panna_set_profiling(ctx: int, on: bool):
    _check(load().panna_set_profiling(ctx, 1 if on else 0))


def panna_stage_ms(ctx: int, stage: str) -> float:
    return float(load().panna_stage_ms(ctx, stage.encode()))


def panna_descriptors_static(desc, sysd: "DeviceSystem", G, stream=None):
    """Descriptors into G without any device allocation (static scratch; see the header)."""
    h = _DescHolder(desc)
    D = int(load().panna_descriptor_size(C.byref(h.s)))
    if D < 0:
        raise PannaError(PANNA_ERR_INVALID_ARG, "invalid descriptor parameters")
    gp = _dev(G, "float32", sysd.n_atoms * D, "G")
    _check(load().panna_descriptors_static(C.byref(h.s), C.byref(sysd.s), gp, _stream(stream)))


def panna_measure_alu_peaks(stream=None):
    """(FP32 FMA TFLOP/s, ex2 G results/s) measured now on the current device."""
    a, b = C.c_double(0.0), C.c_double(0.0)
    _check(load().panna_measure_alu_peaks(C.byref(a), C.byref(b), _stream(stream)))
    return float(a.value), float(b.value)


def panna_measure_alu_peaks2(stream=None):
    """(FP32 FMA TFLOP/s scalar, packed two-wide, ex2 G results/s) measured now."""
    a, b, c = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
    _check(load().panna_measure_alu_peaks2(C.byref(a), C.byref(b), C.byref(c), _stream(stream)))
    return float(a.value), float(b.value), float(c.value)


def panna_capture(ctx: int, sysd: "DeviceSystem", theta, prec: int, E_cfg, E_atom, F, virial, stream=None):
    _check(load().panna_capture(ctx, C.byref(sysd.s), _ptr(theta), int(prec), _ptr(E_cfg), _ptr(E_atom), _ptr(F),
                                _ptr(virial), _stream(stream)))


def panna_replay(ctx: int, stream=None):
    _check(load().panna_replay(ctx, _stream(stream)))


def panna_set_qeq(ctx: int, sigma, chi0, hard0, k_coulomb: float = 0.0):
    arrs = [np.ascontiguousarray(a, np.float64) for a in (sigma, chi0, hard0)]
    p = panna_qeq_params(arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data, float(k_coulomb))
    _check(load().panna_set_qeq(ctx, C.byref(p)))


def panna_qeq_energy_forces(ctx: int, sysd: "DeviceSystem", theta, total_charge, E_cfg, E_atom, charges, F,
                            stream=None):
    _check(load().panna_qeq_energy_forces(ctx, C.byref(sysd.s), _ptr(theta), _ptr(total_charge), _ptr(E_cfg),
                                          _ptr(E_atom), _ptr(charges), _ptr(F), _stream(stream)))


def panna_qeq_loss_grad(ctx: int, sysd: "DeviceSystem", theta, total_charge, E_ref, F_ref, w_force: float, q_ref,
                        w_charge: float, loss, dtheta, E_cfg=None, charges=None, F=None, stream=None):
    _check(load().panna_qeq_loss_grad(ctx, C.byref(sysd.s), _ptr(theta), _ptr(total_charge), _ptr(E_ref), _ptr(F_ref),
                                      float(w_force), _ptr(q_ref), float(w_charge), _ptr(loss), _ptr(dtheta),
                                      _ptr(E_cfg), _ptr(charges), _ptr(F), _stream(stream)))


def panna_store_plan(ctx: int, sysd: "DeviceSystem", stream=None) -> panna_store_info:
    info = panna_store_info()
    _check(load().panna_store_plan(ctx, C.byref(sysd.s), C.byref(info), _stream(stream)))
    return info


def panna_store_sections(ctx: int, info: panna_store_info):
    off = (C.c_int64 * 9)()
    _check(load().panna_store_sections(ctx, C.byref(info), off))
    return [int(x) for x in off]


def panna_store_build(ctx: int, sysd: "DeviceSystem", info: panna_store_info, store, stream=None):
    _check(load().panna_store_build(ctx, C.byref(sysd.s), C.byref(info), _ptr(store), _stream(stream)))


def panna_store_energy_forces(ctx: int, sysd: "DeviceSystem", info: panna_store_info, store, theta, prec: int,
                              E_cfg, E_atom, F, virial, stream=None):
    _check(load().panna_store_energy_forces(ctx, C.byref(sysd.s), C.byref(info), _ptr(store), _ptr(theta),
                                            int(prec), _ptr(E_cfg), _ptr(E_atom), _ptr(F), _ptr(virial),
                                            _stream(stream)))


def panna_store_loss_grad(ctx: int, sysd: "DeviceSystem", info: panna_store_info, store, theta, E_ref, F_ref,
                          w_force: float, loss, dtheta, E_cfg=None, F=None, stream=None):
    _check(load().panna_store_loss_grad(ctx, C.byref(sysd.s), C.byref(info), _ptr(store), _ptr(theta),
                                        _ptr(E_ref), _ptr(F_ref), float(w_force), _ptr(loss), _ptr(dtheta),
                                        _ptr(E_cfg), _ptr(F), _stream(stream)))


def panna_version() -> str:
    return load().panna_version().decode()


# ---------------------------------------------------------------------------- helpers

class DeviceSystem:
    """Device copies (torch CUDA tensors) of a workloads.System plus the C struct."""

    def __init__(self, system, device="cuda", ghost=None):
        import torch
        self.atom_off = torch.as_tensor(np.ascontiguousarray(system.atom_off, np.int64), device=device)
        self.pos = torch.as_tensor(np.ascontiguousarray(system.pos, np.float64), device=device)
        self.species = torch.as_tensor(np.ascontiguousarray(system.species, np.int32), device=device)
        self.cell = torch.as_tensor(np.ascontiguousarray(system.cell, np.float64), device=device)
        self.pbc = torch.as_tensor(np.ascontiguousarray(system.pbc, np.uint8), device=device)
        self.ghost = None if ghost is None else torch.as_tensor(np.ascontiguousarray(ghost, np.uint8), device=device)
        self.n_cfg = int(system.n_cfg)
        self.n_atoms = int(system.n_atoms)
        self.s = panna_system(self.n_cfg, self.n_atoms, self.atom_off.data_ptr(), self.pos.data_ptr(),
                              self.species.data_ptr(), self.cell.data_ptr(), self.pbc.data_ptr(), _ptr(self.ghost))

    @classmethod
    def from_tensors(cls, atom_off, pos, species, cell, pbc, ghost=None):
        obj = cls.__new__(cls)
        obj.atom_off, obj.pos, obj.species, obj.cell, obj.pbc = atom_off, pos, species, cell, pbc
        obj.ghost = ghost
        obj.n_cfg = int(atom_off.shape[0] - 1)
        obj.n_atoms = int(pos.shape[0])
        obj.s = panna_system(obj.n_cfg, obj.n_atoms, atom_off.data_ptr(), pos.data_ptr(), species.data_ptr(),
                             cell.data_ptr(), pbc.data_ptr(), _ptr(ghost))
        return obj


class Potential:
    """A context plus convenience calls returning torch tensors."""

    def __init__(self, desc, archs, neighbor_capacity: Optional[int] = None):
        self.desc = desc
        self.archs = list(archs)
        self.ctx = panna_create(desc, archs)
        self.D = panna_descriptor_size(desc)
        self.P = panna_param_count(self.ctx)
        if neighbor_capacity:
            panna_set_neighbor_capacity(self.ctx, neighbor_capacity)

    def close(self):
        if self.ctx:
            panna_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def descriptors(self, sysd: DeviceSystem):
        import torch
        G = torch.empty((sysd.n_atoms, self.D), dtype=torch.float32, device="cuda")
        panna_descriptors(self.ctx, sysd, G)
        return G

    def neighbors(self, sysd: DeviceSystem):
        import torch
        cap = max(1, sysd.n_atoms * panna_neighbor_capacity(self.ctx))
        while True:
            off = torch.empty(sysd.n_atoms + 1, dtype=torch.int64, device="cuda")
            j = torch.empty(cap, dtype=torch.int64, device="cuda")
            sh = torch.empty((cap, 3), dtype=torch.int32, device="cuda")
            try:
                n = panna_neighbors(self.ctx, sysd, cap, off, j, sh)
                return off, j[:n], sh[:n]
            except PannaError as e:
                if e.status != PANNA_ERR_INVALID_ARG:
                    raise
                cap *= 2

    def energy_forces(self, sysd: DeviceSystem, theta, prec: int = PANNA_MLP_FP32, virial: bool = True,
                      atom_energies: bool = True):
        import torch
        E = torch.empty(sysd.n_cfg, dtype=torch.float64, device="cuda")
        Ea = torch.empty(sysd.n_atoms, dtype=torch.float32, device="cuda") if atom_energies else None
        F = torch.empty((sysd.n_atoms, 3), dtype=torch.float32, device="cuda")
        V = torch.empty((sysd.n_cfg, 3, 3), dtype=torch.float64, device="cuda") if virial else None
        _dev(theta, "float32", self.P, "theta")
        panna_energy_forces(self.ctx, sysd, theta, prec, E, Ea, F, V)
        return E, Ea, F, V

    def qeq_energy_forces(self, sysd: DeviceSystem, theta, total_charge=None):
        """(E_cfg, E_atom, charges, F) with charge equilibration (panna_set_qeq first)."""
        import torch
        E = torch.empty(sysd.n_cfg, dtype=torch.float64, device="cuda")
        Ea = torch.empty(sysd.n_atoms, dtype=torch.float32, device="cuda")
        q = torch.empty(sysd.n_atoms, dtype=torch.float64, device="cuda")
        F = torch.empty((sysd.n_atoms, 3), dtype=torch.float32, device="cuda")
        panna_qeq_energy_forces(self.ctx, sysd, theta, total_charge, E, Ea, q, F)
        return E, Ea, q, F

    def param_vjp(self, sysd: DeviceSystem, theta, dE=None, dF=None):
        import torch
        out = torch.empty(self.P, dtype=torch.float32, device="cuda")
        _dev(theta, "float32", self.P, "theta")
        if dE is not None:
            _dev(dE, "float64", sysd.n_cfg, "dE")
        if dF is not None:
            _dev(dF, "float32", 3 * sysd.n_atoms, "dF")
        panna_param_vjp(self.ctx, sysd, theta, dE, dF, out)
        return out

    def loss_grad(self, sysd: DeviceSystem, theta, E_ref, F_ref, w_force: float):
        import torch
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
        g = torch.empty(self.P, dtype=torch.float32, device="cuda")
        E = torch.empty(sysd.n_cfg, dtype=torch.float64, device="cuda")
        F = torch.empty((sysd.n_atoms, 3), dtype=torch.float32, device="cuda")
        _dev(theta, "float32", self.P, "theta")
        _dev(E_ref, "float64", sysd.n_cfg, "E_ref")
        _dev(F_ref, "float32", 3 * sysd.n_atoms, "F_ref")
        panna_loss_grad(self.ctx, sysd, theta, E_ref, F_ref, w_force, loss, g, E, F)
        return loss, g, E, F


class Store:
    """Precomputed descriptors and Jacobians of one batch in a torch-owned device buffer
    (the nine sections of the store format, at the offsets the library reports)."""

    def __init__(self, pot: "Potential", sysd: DeviceSystem):
        import torch
        self.pot = pot
        self.info = panna_store_plan(pot.ctx, sysd)
        # torch's caching allocator returns blocks aligned to at least 512 bytes
        self.buf = torch.empty(max(int(self.info.bytes), 1), dtype=torch.uint8, device="cuda")
        if self.buf.data_ptr() % 256:
            raise RuntimeError("store buffer is not 256-byte aligned")
        panna_store_build(pot.ctx, sysd, self.info, self.buf)

    @property
    def nbytes(self) -> int:
        return int(self.info.bytes)

    def sections(self):
        """Views of the nine sections as torch tensors (shapes of the store format)."""
        import torch
        off = panna_store_sections(self.pot.ctx, self.info)
        N, P, D, W = int(self.info.n_atoms), int(self.info.n_entries), int(self.info.D), int(self.info.width)
        S = len(self.pot.archs)
        spec = [(torch.float32, (N, D)), (torch.int32, (N,)), (torch.int32, (N,)), (torch.int32, (S + 1,)),
                (torch.int32, (N,)), (torch.int64, (N + 1,)), (torch.int32, (P, 2)), (torch.float32, (P, 4)),
                (torch.float32, (P, 3, W))]
        out = {}
        for name, o, (dt, shape) in zip(STORE_SECTIONS, off, spec):
            n = int(np.prod(shape)) * torch.empty(0, dtype=dt).element_size()
            out[name] = self.buf[o:o + n].view(dt).view(shape)
        return out

    def energy_forces(self, sysd: DeviceSystem, theta, prec: int = PANNA_MLP_FP32, virial: bool = True):
        import torch
        E = torch.empty(sysd.n_cfg, dtype=torch.float64, device="cuda")
        Ea = torch.empty(sysd.n_atoms, dtype=torch.float32, device="cuda")
        F = torch.empty((sysd.n_atoms, 3), dtype=torch.float32, device="cuda")
        V = torch.empty((sysd.n_cfg, 3, 3), dtype=torch.float64, device="cuda") if virial else None
        panna_store_energy_forces(self.pot.ctx, sysd, self.info, self.buf, theta, prec, E, Ea, F, V)
        return E, Ea, F, V

    def loss_grad(self, sysd: DeviceSystem, theta, E_ref, F_ref, w_force: float):
        import torch
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
        g = torch.empty(self.pot.P, dtype=torch.float32, device="cuda")
        E = torch.empty(sysd.n_cfg, dtype=torch.float64, device="cuda")
        F = torch.empty((sysd.n_atoms, 3), dtype=torch.float32, device="cuda")
        panna_store_loss_grad(self.pot.ctx, sysd, self.info, self.buf, theta, E_ref, F_ref, w_force, loss, g, E, F)
        return loss, g, E, F
