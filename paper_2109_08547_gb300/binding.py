"""Thin ctypes binding of the C ABI in include/ephb.h.

Argument marshalling only: every numerical step runs in the CUDA library.  Loading
fails loudly when the shared library cannot be built or opened; there is no CPU path.
Function names follow the C entry points (set_wannier_model, build_meshes_ibz,
compute_transition_rates, solve_coupled_bte, transport_coefficients).
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np

from . import build as _build

_lib = None

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ENOCONV, ETIMEOUT, EINTERNAL = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ESTATE", "ENOCONV", "ETIMEOUT", "EINTERNAL"]
FP64, SPLIT_TF32, SPLIT_BF16, FP64_SLICED = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp64-sliced": FP64_SLICED, "split-bf16": SPLIT_BF16}
SOLVE_PRECISIONS = {"fp64": 0, "mixed": 1}
RTA, PARTIAL, DRAGLESS, DRAGGED = 0, 1, 2, 3
LEVELS = {"rta": RTA, "partial": PARTIAL, "dragless": DRAGLESS, "dragged": DRAGGED}

ARR = dict(eps=0, vel=1, omega=2, vph=3, ibz_rep=4, ibz_op=5, ibzw_list=6, row_ptr=7, entry_kpns=8, entry_x=9,
           pair_q=10, w_e=11, w_ph=12, I=13, J=14, F=15, G=16, pair_ptr=17, active=18, state_eps=19,
           state_vel=20, state_weight=21)
NOALLOC_MAX_ITEMS = 4194304
_DT = {0: np.float64, 1: np.complex128, 2: np.int32, 3: np.int64, 4: np.uint32}

EXPORTED = ["ephb_create", "ephb_destroy", "ephb_last_error", "ephb_set_wannier_model", "ephb_build_meshes_ibz",
            "ephb_compute_transition_rates", "ephb_solve_coupled_bte", "ephb_transport_coefficients",
            "ephb_get_device_array", "ephb_copy_array_to_host", "ephb_kernel_launches",
            "ephb_transport_coefficients_noalloc", "ephb_select_instance", "ephb_num_instances",
            "ephb_instance_solve_info", "ephb_num_states", "ephb_state_features", "ephb_state_targets",
            "ephb_set_warm_start", "ephb_mlp_create", "ephb_mlp_destroy", "ephb_mlp_last_error",
            "ephb_mlp_num_params", "ephb_mlp_set_bf16", "ephb_mlp_get_params", "ephb_mlp_set_params",
            "ephb_mlp_forward", "ephb_mlp_loss_grad", "ephb_mlp_train_step", "ephb_set_tuning",
            "ephb_selftest_exp_ff", "ephb_set_impurities", "ephb_set_isotopes"]
MAX_DOPANTS = 4   # EPHB_MAX_DOPANTS
NFEAT = 6
MAX_ACCEL_DEPTH = 8   # EPHB_MAX_ACCEL_DEPTH

_pd = C.POINTER(C.c_double)
_pi = C.POINTER(C.c_int32)


class ModelC(C.Structure):
    _fields_ = [("lattice", C.c_double * 9), ("nat", C.c_int), ("mass_amu", _pd), ("tau_cart", _pd),
                ("nb", C.c_int), ("nRe", C.c_int), ("Re", _pi), ("H_R", _pd), ("nRd", C.c_int), ("Rd", _pi),
                ("D_R", _pd), ("nRge", C.c_int), ("nRgp", C.c_int), ("Rge", _pi), ("Rgp", _pi), ("g_R", _pd),
                ("omega_ref_eV", C.c_double), ("nsym", C.c_int), ("sym_rot", _pi), ("sym_cart", _pd),
                ("spin_deg", C.c_double), ("bg_rate_coeff", C.c_double), ("bg_omega_ref_eV", C.c_double),
                ("bg_T_ref", C.c_double)]


class MeshOptsC(C.Structure):
    _fields_ = [("kmesh", C.c_int * 3), ("qmesh", C.c_int * 3), ("window_lo_eV", C.c_double),
                ("window_hi_eV", C.c_double), ("degen_tol_eV", C.c_double), ("omega_min_eV", C.c_double)]


class MeshInfoC(C.Structure):
    _fields_ = [("nk", C.c_int64), ("nq", C.c_int64), ("n_active_states", C.c_int64), ("n_ibz", C.c_int64),
                ("n_ibz_window", C.c_int64), ("n_pairs", C.c_int64), ("ms", C.c_double)]


class ThermoC(C.Structure):
    _fields_ = [("T_K", C.c_double), ("mu_eV", C.c_double), ("window_lo_eV", C.c_double),
                ("window_hi_eV", C.c_double)]


class DeltaC(C.Structure):
    _fields_ = [("sigma_eV", C.c_double), ("cutoff_sigmas", C.c_double), ("kind", C.c_int)]


DELTA_GAUSS, DELTA_TETRA = 0, 1   # EPHB_DELTA_*
DELTAS = {"gauss": DELTA_GAUSS, "tetra": DELTA_TETRA}


class RatesInfoC(C.Structure):
    _fields_ = [("n_tuples", C.c_int64), ("n_entries", C.c_int64), ("n_ph_entries", C.c_int64),
                ("n_pairs", C.c_int64), ("ms", C.c_double), ("ms_stage_a", C.c_double), ("ms_stage_b", C.c_double),
                ("stage_a_flops", C.c_double), ("stage_b_flops", C.c_double), ("ms_epilogue", C.c_double),
                ("tensor_flops", C.c_double), ("rot_flops", C.c_double), ("ms_gemm", C.c_double),
                ("tc_cols", C.c_int), ("autotuned", C.c_int), ("tc_kblock", C.c_int), ("tc_stages", C.c_int),
                ("tensor_flops_a", C.c_double)]


class SolveOptsC(C.Structure):
    _fields_ = [("level", C.c_int), ("tol", C.c_double), ("inner_tol", C.c_double), ("max_outer", C.c_int),
                ("max_inner", C.c_int), ("ko_correction", C.c_int), ("warm_start", C.c_int),
                ("precision", C.c_int), ("accel_depth", C.c_int), ("device_loop", C.c_int)]


class SolveInfoC(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("inner_iters_total", C.c_int), ("converged", C.c_int),
                ("n_zero_rate_states", C.c_int), ("residual", C.c_double), ("lambda_", C.c_double),
                ("n_sweeps", C.c_int64), ("ms", C.c_double), ("ms_e_sweep", C.c_double),
                ("ms_ph_sweep", C.c_double), ("e_sweep_bytes", C.c_double), ("ms_drag", C.c_double),
                ("n_runs", C.c_int64), ("ms_self_kernel", C.c_double), ("e_sweep_flops", C.c_double),
                ("n_sweeps32", C.c_int64), ("ms_corr", C.c_double), ("outer_iters32", C.c_int),
                ("graph_launches", C.c_int), ("graph_reused", C.c_int)]


class CoeffsC(C.Structure):
    _fields_ = [(n, C.c_double * 9) for n in
                ("sigma", "sigmaS", "S", "alpha_el", "kappa0_el", "kappa_el", "alpha_ph", "kappa_ph")]


class ImpuritiesC(C.Structure):
    _fields_ = [("n_species", C.c_int), ("n_cm3", C.c_double * 4), ("Z", C.c_double * 4), ("eps_r", C.c_double)]


class CoeffInputsC(C.Structure):
    _fields_ = [("n_states", C.c_int64), ("eps", C.c_void_p), ("vel", C.c_void_p), ("weight", C.c_void_p),
                ("I", C.c_void_p), ("J", C.c_void_p), ("n_modes", C.c_int64), ("omega", C.c_void_p),
                ("vph", C.c_void_p), ("F", C.c_void_p), ("G", C.c_void_p), ("T_K", C.c_double),
                ("mu_eV", C.c_double), ("spin_deg", C.c_double), ("volume_A3", C.c_double), ("nk", C.c_int64),
                ("nq", C.c_int64), ("omega_min_eV", C.c_double), ("nsym", C.c_int),
                ("sym_cart", C.c_double * (48 * 9))]


class EphbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def load(path: str = None):
    """Open (building first if sources changed) the CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.build()
    lib = C.CDLL(path)
    lib.ephb_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]
    lib.ephb_destroy.argtypes = [C.c_void_p]
    lib.ephb_destroy.restype = None
    lib.ephb_last_error.argtypes = [C.c_void_p]
    lib.ephb_last_error.restype = C.c_char_p
    lib.ephb_set_wannier_model.argtypes = [C.c_void_p, C.POINTER(ModelC)]
    lib.ephb_build_meshes_ibz.argtypes = [C.c_void_p, C.POINTER(MeshOptsC), C.POINTER(MeshInfoC)]
    lib.ephb_compute_transition_rates.argtypes = [C.c_void_p, C.POINTER(ThermoC), C.c_int, C.POINTER(DeltaC),
                                                  C.c_int, C.POINTER(RatesInfoC)]
    lib.ephb_solve_coupled_bte.argtypes = [C.c_void_p, C.POINTER(SolveOptsC), C.POINTER(SolveInfoC)]
    lib.ephb_transport_coefficients.argtypes = [C.c_void_p, C.c_int, C.POINTER(CoeffsC)]
    lib.ephb_set_impurities.argtypes = [C.c_void_p, C.POINTER(ImpuritiesC)]
    lib.ephb_set_isotopes.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.c_int]
    lib.ephb_get_device_array.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                          C.POINTER(C.c_int)]
    lib.ephb_copy_array_to_host.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]
    lib.ephb_transport_coefficients_noalloc.argtypes = [C.POINTER(CoeffInputsC), C.c_void_p, C.c_void_p]
    lib.ephb_kernel_launches.argtypes = []
    lib.ephb_select_instance.argtypes = [C.c_void_p, C.c_int]
    lib.ephb_num_instances.argtypes = [C.c_void_p]
    lib.ephb_instance_solve_info.argtypes = [C.c_void_p, C.c_int, C.POINTER(SolveInfoC)]
    lib.ephb_set_tuning.argtypes = [C.c_void_p, C.c_int, C.c_int]
    lib.ephb_num_states.argtypes = [C.c_void_p]
    lib.ephb_state_features.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]
    lib.ephb_state_targets.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]
    lib.ephb_set_warm_start.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]
    lib.ephb_mlp_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_uint64]
    lib.ephb_mlp_destroy.argtypes = [C.c_void_p]
    lib.ephb_mlp_last_error.argtypes = [C.c_void_p]
    lib.ephb_mlp_num_params.argtypes = [C.c_void_p]
    lib.ephb_mlp_set_bf16.argtypes = [C.c_void_p, C.c_int]
    lib.ephb_mlp_get_params.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    lib.ephb_mlp_set_params.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    lib.ephb_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
    lib.ephb_mlp_loss_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_float),
                                       C.c_void_p]
    lib.ephb_mlp_train_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float,
                                        C.POINTER(C.c_float)]
    for name in EXPORTED:
        if name not in ("ephb_destroy", "ephb_last_error", "ephb_kernel_launches", "ephb_num_states",
                        "ephb_mlp_destroy", "ephb_mlp_last_error", "ephb_mlp_num_params"):
            getattr(lib, name).restype = C.c_int
    lib.ephb_kernel_launches.restype = C.c_int64
    lib.ephb_num_states.restype = C.c_int64
    lib.ephb_mlp_destroy.restype = None
    lib.ephb_mlp_last_error.restype = C.c_char_p
    lib.ephb_mlp_num_params.restype = C.c_int64
    _lib = lib
    return lib


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(load().ephb_kernel_launches())


def _check(ctx, status, allow=()):
    if status != OK and status not in allow:
        msg = _lib.ephb_last_error(ctx.handle).decode() if ctx is not None and ctx.handle else ""
        raise EphbError(status, msg)
    return status


class Context:
    """Owns one ephb_ctx (device memory of one model / mesh / rate set)."""

    def __init__(self, device: int = 0, stream: int = None):
        lib = load()
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except ImportError:
                stream = None
        h = C.c_void_p()
        st = lib.ephb_create(C.byref(h), int(device), C.c_void_p(stream) if stream else None)
        if st != OK:
            raise EphbError(st, "ephb_create failed (is a CUDA device visible?)")
        self.handle = h
        self._keep = []

    def close(self):
        if getattr(self, "handle", None):
            _lib.ephb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _arr(x, dtype):
    a = np.ascontiguousarray(x, dtype=dtype)
    return a


def set_wannier_model(ctx: Context, m) -> None:
    """ephb_set_wannier_model from a WannierModel (numpy arrays)."""
    keep = {
        "mass": _arr(m.mass_amu, np.float64), "tau": _arr(m.tau_cart, np.float64), "Re": _arr(m.Re, np.int32),
        "H": _arr(m.H_R, np.complex128), "Rd": _arr(m.Rd, np.int32), "D": _arr(m.D_R, np.complex128),
        "Rge": _arr(m.Rge, np.int32), "Rgp": _arr(m.Rgp, np.int32), "g": _arr(m.g_R, np.complex128),
        "rot": _arr(m.sym_rot, np.int32), "cart": _arr(m.sym_cart, np.float64),
    }
    mc = ModelC()
    mc.lattice[:] = list(np.asarray(m.lattice, dtype=np.float64).ravel())
    mc.nat = int(m.mass_amu.shape[0])
    mc.mass_amu = keep["mass"].ctypes.data_as(_pd)
    mc.tau_cart = keep["tau"].ctypes.data_as(_pd)
    mc.nb = int(m.nb)
    mc.nRe = int(keep["Re"].shape[0])
    mc.Re = keep["Re"].ctypes.data_as(_pi)
    mc.H_R = keep["H"].ctypes.data_as(_pd)
    mc.nRd = int(keep["Rd"].shape[0])
    mc.Rd = keep["Rd"].ctypes.data_as(_pi)
    mc.D_R = keep["D"].ctypes.data_as(_pd)
    mc.nRge = int(keep["Rge"].shape[0])
    mc.nRgp = int(keep["Rgp"].shape[0])
    mc.Rge = keep["Rge"].ctypes.data_as(_pi)
    mc.Rgp = keep["Rgp"].ctypes.data_as(_pi)
    mc.g_R = keep["g"].ctypes.data_as(_pd)
    mc.omega_ref_eV = float(m.omega_ref_eV)
    mc.nsym = int(keep["rot"].shape[0])
    mc.sym_rot = keep["rot"].ctypes.data_as(_pi)
    mc.sym_cart = keep["cart"].ctypes.data_as(_pd)
    mc.spin_deg = float(m.spin_deg)
    mc.bg_rate_coeff = float(m.bg_rate_coeff)
    mc.bg_omega_ref_eV = float(m.bg_omega_ref_eV)
    mc.bg_T_ref = float(m.bg_T_ref)
    _check(ctx, _lib.ephb_set_wannier_model(ctx.handle, C.byref(mc)))


def build_meshes_ibz(ctx: Context, kmesh, qmesh, window, degen_tol_eV=1e-6, omega_min_eV=1e-4) -> dict:
    o = MeshOptsC()
    o.kmesh[:] = [int(x) for x in kmesh]
    o.qmesh[:] = [int(x) for x in qmesh]
    o.window_lo_eV, o.window_hi_eV = float(window[0]), float(window[1])
    o.degen_tol_eV = float(degen_tol_eV)
    o.omega_min_eV = float(omega_min_eV)
    info = MeshInfoC()
    _check(ctx, _lib.ephb_build_meshes_ibz(ctx.handle, C.byref(o), C.byref(info)))
    return {f: getattr(info, f) for f, _ in MeshInfoC._fields_}


def compute_transition_rates(ctx: Context, T_K, mu_eV, sigma_eV=0.01, cutoff_sigmas=8.0, precision=FP64,
                             instances=None, delta="gauss") -> dict:
    """One (T_K, mu_eV) instance on the mesh window, or ``instances``: a list of
    (T_K, mu_eV) or (T_K, mu_eV, window_lo_eV, window_hi_eV) tuples (T_K, mu_eV ignored)."""
    if instances is None:
        instances = [(T_K, mu_eV)]
    arr = (ThermoC * len(instances))()
    for i, t in enumerate(instances):
        lo, hi = (t[2], t[3]) if len(t) > 2 else (0.0, 0.0)
        arr[i] = ThermoC(float(t[0]), float(t[1]), float(lo), float(hi))
    de = DeltaC(float(sigma_eV), float(cutoff_sigmas), DELTAS[delta] if isinstance(delta, str) else int(delta))
    info = RatesInfoC()
    _check(ctx, _lib.ephb_compute_transition_rates(ctx.handle, arr, len(instances), C.byref(de), int(precision),
                                                   C.byref(info)))
    return {f: getattr(info, f) for f, _ in RatesInfoC._fields_}


TUNE_TC_COLS = 0
TUNE_WITHHOLD_MMA = 1
TUNE_DEFER_INSTANCES = 2
TUNE_STAGE_A_TMEM_A = 3


def set_tuning(ctx: Context, key: int, value: int) -> None:
    _check(ctx, _lib.ephb_set_tuning(ctx.handle, int(key), int(value)))


def select_instance(ctx: Context, inst: int) -> None:
    _check(ctx, _lib.ephb_select_instance(ctx.handle, int(inst)))


def num_instances(ctx: Context) -> int:
    return int(_lib.ephb_num_instances(ctx.handle))


def instance_solve_info(ctx: Context, inst: int) -> dict:
    info = SolveInfoC()
    _check(ctx, _lib.ephb_instance_solve_info(ctx.handle, int(inst), C.byref(info)))
    d = {f: getattr(info, f) for f, _ in SolveInfoC._fields_}
    d["lambda"] = d.pop("lambda_")
    return d


def solve_coupled_bte(ctx: Context, level="dragged", tol=1e-10, inner_tol=0.0, max_outer=500, max_inner=5000,
                      ko_correction=True, allow_noconv=False, warm_start=False, solve_precision="fp64",
                      accel=0, device_loop=False) -> dict:
    """accel: Anderson history depth of the outer iteration (0: the plain iteration).
    device_loop: the whole solve of every instance as one CUDA graph launch (device-driven loops)."""
    o = SolveOptsC(LEVELS[level] if isinstance(level, str) else int(level), float(tol), float(inner_tol),
                   int(max_outer), int(max_inner), 1 if ko_correction else 0, 1 if warm_start else 0,
                   SOLVE_PRECISIONS[solve_precision], int(accel), 1 if device_loop else 0)
    info = SolveInfoC()
    st = _check(ctx, _lib.ephb_solve_coupled_bte(ctx.handle, C.byref(o), C.byref(info)),
                allow=(ENOCONV,) if allow_noconv else ())
    d = {f: getattr(info, f) for f, _ in SolveInfoC._fields_}
    d["lambda"] = d.pop("lambda_")
    d["status"] = st
    return d


def set_impurities(ctx: Context, imp=None) -> None:
    """Charged impurities of the e-chimp channel (an object with n_cm3, Z, eps_r, e.g.
    synthetic.Impurities), or None to clear them."""
    if imp is None or len(imp.n_cm3) == 0:
        _check(ctx, _lib.ephb_set_impurities(ctx.handle, None))
        return
    c = ImpuritiesC()
    c.n_species = len(imp.n_cm3)      # the library rejects more than MAX_DOPANTS
    for i, (n, z) in enumerate(list(zip(imp.n_cm3, imp.Z))[:MAX_DOPANTS]):
        c.n_cm3[i] = float(n)
        c.Z[i] = float(z)
    c.eps_r = float(imp.eps_r)
    _check(ctx, _lib.ephb_set_impurities(ctx.handle, C.byref(c)))


def set_isotopes(ctx: Context, g=None) -> None:
    """Mass-variance parameter of each atom for the ph-isotope channel, or None to clear it."""
    if g is None or len(g) == 0:
        _check(ctx, _lib.ephb_set_isotopes(ctx.handle, None, 0))
        return
    arr = (C.c_double * len(g))(*[float(x) for x in g])
    _check(ctx, _lib.ephb_set_isotopes(ctx.handle, arr, len(g)))


def transport_coefficients(ctx: Context, inst: int = 0) -> dict:
    c = CoeffsC()
    _check(ctx, _lib.ephb_transport_coefficients(ctx.handle, int(inst), C.byref(c)))
    return {f: np.array(getattr(c, f)[:]).reshape(3, 3) for f, _ in CoeffsC._fields_}


def get_array(ctx: Context, which: str) -> np.ndarray:
    """Copy one of the context's device arrays into a new numpy array."""
    p = C.c_void_p()
    shape = (C.c_int64 * 4)()
    dt = C.c_int()
    _check(ctx, _lib.ephb_get_device_array(ctx.handle, ARR[which], C.byref(p), shape, C.byref(dt)))
    shp = [int(s) for s in shape]
    out = np.empty(shp, dtype=_DT[dt.value])
    _check(ctx, _lib.ephb_copy_array_to_host(ctx.handle, ARR[which], out.ctypes.data_as(C.c_void_p), out.nbytes))
    while out.ndim > 1 and out.shape[-1] == 1:
        out = out.reshape(out.shape[:-1])
    return out


def device_array(ctx: Context, which: str):
    """Borrowed device pointer, shape and numpy dtype of a context array."""
    p = C.c_void_p()
    shape = (C.c_int64 * 4)()
    dt = C.c_int()
    _check(ctx, _lib.ephb_get_device_array(ctx.handle, ARR[which], C.byref(p), shape, C.byref(dt)))
    return p.value, tuple(int(s) for s in shape), _DT[dt.value]


def transport_coefficients_noalloc(ptrs: dict, n_states: int, n_modes: int, T_K: float, mu_eV: float,
                                   spin_deg: float, volume_A3: float, nk: int, nq: int, omega_min_eV: float,
                                   sym_cart, out_dev: int, stream: int = 0) -> int:
    """ephb_transport_coefficients_noalloc: `ptrs` maps eps, vel, weight, I, J, omega, vph, F, G
    to device addresses; `out_dev` is the device address of 72 doubles.  Returns the status."""
    lib = load()
    c = CoeffInputsC()
    c.n_states, c.n_modes = int(n_states), int(n_modes)
    for name in ("eps", "vel", "weight", "I", "J", "omega", "vph", "F", "G"):
        setattr(c, name, C.c_void_p(ptrs[name]) if ptrs.get(name) else None)
    c.T_K, c.mu_eV, c.spin_deg, c.volume_A3 = float(T_K), float(mu_eV), float(spin_deg), float(volume_A3)
    c.nk, c.nq, c.omega_min_eV = int(nk), int(nq), float(omega_min_eV)
    ops = np.ascontiguousarray(sym_cart, dtype=np.float64).reshape(-1, 9)
    c.nsym = int(ops.shape[0])
    flat = np.zeros(48 * 9)
    flat[:ops.size] = ops.ravel()
    c.sym_cart[:] = list(flat)
    return int(lib.ephb_transport_coefficients_noalloc(C.byref(c), C.c_void_p(out_dev),
                                                        C.c_void_p(stream) if stream else None))


def selftest_exp_ff(y_dev: int, out_dev: int, n: int, stream: int = 0) -> int:
    """ephb_selftest_exp_ff: e^y of n device doubles through the library's float-float
    exponential.  Returns the status."""
    return int(load().ephb_selftest_exp_ff(C.c_void_p(y_dev), C.c_void_p(out_dev), C.c_int64(n),
                                           C.c_void_p(stream) if stream else None))


@dataclasses.dataclass
class PathResult:
    mesh: dict
    rates: dict
    solve: dict
    coeffs: dict


def run_path(ctx: Context, wl, level="dragged", ko_correction=True, tol=None, max_outer=500, max_inner=5000,
             precision=FP64, allow_noconv=False, solve_precision="fp64", accel=0,
             device_loop=False) -> PathResult:
    """The whole hot path for one workload on an existing context whose model is set."""
    set_impurities(ctx, getattr(wl, "chimp", None))
    set_isotopes(ctx, getattr(wl, "isotopes", None))
    mesh = build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
    rates = compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas, precision,
                                     delta=getattr(wl, "delta", "gauss"))
    solve = solve_coupled_bte(ctx, level, wl.tol if tol is None else tol, 0.0, max_outer, max_inner, ko_correction,
                              allow_noconv, solve_precision=solve_precision, accel=accel, device_loop=device_loop)
    return PathResult(mesh, rates, solve, transport_coefficients(ctx))


# ----------------------------------------------------------------------------------------
# learned warm start
# ----------------------------------------------------------------------------------------

def num_states(ctx: Context) -> int:
    return int(_lib.ephb_num_states(ctx.handle))


def state_features(ctx: Context, inst: int, out_ptr: int) -> None:
    """Network inputs of instance inst into device memory out_ptr ([num_states][NFEAT] FP32)."""
    _check(ctx, _lib.ephb_state_features(ctx.handle, int(inst), C.c_void_p(out_ptr), num_states(ctx)))


def state_targets(ctx: Context, inst: int, out_ptr: int) -> None:
    """Training targets of a solved instance into device memory out_ptr ([num_states][2] FP32)."""
    _check(ctx, _lib.ephb_state_targets(ctx.handle, int(inst), C.c_void_p(out_ptr), num_states(ctx)))


def set_warm_start(ctx: Context, inst: int, scale_ptr) -> None:
    """Scale factors [num_states][2] (device FP32) for the next solve of instance inst; None clears."""
    _check(ctx, _lib.ephb_set_warm_start(ctx.handle, int(inst), C.c_void_p(scale_ptr) if scale_ptr else None,
                                         num_states(ctx)))


class MLP:
    """The warm-start network (device parameters; see include/ephb.h)."""

    def __init__(self, n_in=NFEAT, width=128, depth=3, n_out=2, seed=0, device=0, stream=None):
        load()
        h = C.c_void_p()
        st = _lib.ephb_mlp_create(C.byref(h), int(device), C.c_void_p(stream) if stream else None, int(n_in),
                                  int(width), int(depth), int(n_out), C.c_uint64(seed))
        if st != OK:
            raise EphbError(st, "ephb_mlp_create failed")
        self.handle = h
        self.n_in, self.width, self.depth, self.n_out = n_in, width, depth, n_out

    def _check(self, st):
        if st != OK:
            raise EphbError(st, _lib.ephb_mlp_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            _lib.ephb_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self) -> int:
        return int(_lib.ephb_mlp_num_params(self.handle))

    def set_bf16(self, on: bool) -> None:
        self._check(_lib.ephb_mlp_set_bf16(self.handle, 1 if on else 0))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        self._check(_lib.ephb_mlp_get_params(self.handle, out.ctypes.data_as(C.c_void_p), out.size))
        return out

    def set_params(self, v) -> None:
        v = np.ascontiguousarray(v, dtype=np.float32)
        self._check(_lib.ephb_mlp_set_params(self.handle, v.ctypes.data_as(C.c_void_p), v.size))

    def forward(self, x_ptr: int, n: int, y_ptr: int) -> None:
        self._check(_lib.ephb_mlp_forward(self.handle, C.c_void_p(x_ptr), int(n), C.c_void_p(y_ptr)))

    def loss_grad(self, x_ptr: int, t_ptr: int, n: int, grad_ptr: int = 0) -> float:
        lo = C.c_float()
        self._check(_lib.ephb_mlp_loss_grad(self.handle, C.c_void_p(x_ptr), C.c_void_p(t_ptr), int(n), C.byref(lo),
                                            C.c_void_p(grad_ptr) if grad_ptr else None))
        return float(lo.value)

    def train_step(self, x_ptr: int, t_ptr: int, n: int, lr: float) -> float:
        lo = C.c_float()
        self._check(_lib.ephb_mlp_train_step(self.handle, C.c_void_p(x_ptr), C.c_void_p(t_ptr), int(n), float(lr),
                                             C.byref(lo)))
        return float(lo.value)
