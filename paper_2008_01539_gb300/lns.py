"""Python binding of liblns (the C ABI in include/lns.h): argument marshalling only.

Every entry point keeps its C name (``lns_timestep``, ``lns_active_set`` ...).  Device
memory comes from PyTorch's caching allocator and work runs on the current PyTorch CUDA
stream; every computation runs in the library's CUDA kernels.  There is no CPU fallback:
loading fails loudly when the library is not built or no GPU is present.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import build as _build

PSI = 6894.757293168

LNS_OK, LNS_EINVAL, LNS_ENOMEM, LNS_ECUDA, LNS_ENOCONV, LNS_EKRYLOV, LNS_ETIMEOUT, LNS_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
LNS_MODE_FULL, LNS_MODE_LOCAL, LNS_MODE_DD, LNS_MODE_RESIDUAL = 0, 1, 2, 3
LNS_PRECOND_BJAC, LNS_PRECOND_BJAC_CELL = 0, 1
_STATUS = {0: "LNS_OK", -1: "LNS_EINVAL", -2: "LNS_ENOMEM", -3: "LNS_ECUDA", -4: "LNS_ENOCONV",
           -5: "LNS_EKRYLOV", -6: "LNS_ETIMEOUT", -7: "LNS_ESTATE"}


class LnsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class lns_fluid(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("p_ref", "c_r", "b_o_ref", "c_o", "b_w_ref", "c_w", "rho_o_ref",
                                           "rho_w_ref", "mu_o", "mu_w", "swc", "sor")] + \
               [("n_w", C.c_int32), ("n_o", C.c_int32), ("gravity", C.c_double)]


class lns_model_desc(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("n_adj", C.c_int32), ("row_ptr", C.c_void_p), ("nbr", C.c_void_p),
                ("trans", C.c_void_p), ("pv_ref", C.c_void_p), ("depth", C.c_void_p), ("line_id", C.c_void_p),
                ("always_active", C.c_void_p), ("n_wells", C.c_int32), ("well_cell", C.c_void_p),
                ("well_wi", C.c_void_p), ("well_bhp", C.c_void_p), ("fluid", lns_fluid), ("p0", C.c_void_p),
                ("sw0", C.c_void_p)]


class lns_options(C.Structure):
    _fields_ = [("mode", C.c_int32), ("eps_p", C.c_double), ("eps_sw", C.c_double), ("m_layers", C.c_int32),
                ("tol_dp", C.c_double), ("tol_cnv", C.c_double), ("max_newton", C.c_int32),
                ("max_dd_outer", C.c_int32), ("sat_chop", C.c_double), ("krylov_fp32", C.c_int32),
                ("precond", C.c_int32), ("krylov_rtol", C.c_double), ("krylov_maxit", C.c_int32),
                ("krylov_fail_rtol", C.c_double), ("p_scale", C.c_double), ("profile", C.c_int32),
                ("fp64_fallback", C.c_int32), ("krylov_cluster", C.c_int32), ("autotune", C.c_int32),
                ("dd_local_newton", C.c_int32), ("dd_local_shrink", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class lns_allocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class lns_iter_stats(C.Structure):
    _fields_ = [("n_active", C.c_int32), ("is_expand", C.c_int32), ("converged", C.c_int32),
                ("step_done", C.c_int32), ("krylov_iters", C.c_int32), ("krylov_status", C.c_int32),
                ("fp64_retry", C.c_int32), ("max_dp", C.c_double), ("max_dsw", C.c_double), ("cnv", C.c_double),
                ("krylov_relres", C.c_double), ("krylov_solver", C.c_int32)]


class lns_step_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("krylov_iters", C.c_int32),
                ("n_subdomains", C.c_int32), ("dd_outer", C.c_int32), ("fp64_retries", C.c_int32),
                ("cell_updates", C.c_int64),
                ("last_max_dp", C.c_double), ("last_cnv", C.c_double)]


class lns_dt_control(C.Structure):
    _fields_ = [("dt_init", C.c_double), ("dt_min", C.c_double), ("dt_max", C.c_double), ("grow", C.c_double),
                ("cut", C.c_double), ("easy_iters", C.c_int32)]


class lns_advance_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("steps", C.c_int32), ("cuts", C.c_int32), ("iterations", C.c_int32),
                ("krylov_iters", C.c_int64), ("cell_updates", C.c_int64), ("t_done", C.c_double),
                ("dt_next", C.c_double)]


class lns_batch_stats(C.Structure):
    _fields_ = [("rounds", C.c_int32), ("cluster_solves", C.c_int64), ("grid_solves", C.c_int64)]


class lns_bo_fluid(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("p_ref", "c_r", "b_w_ref", "c_w", "rho_w_sc", "mu_w", "b_o_ref", "c_o",
                                           "kappa", "rho_o_sc", "mu_o", "b_g_per_pa", "rho_g_sc", "mu_g", "rs_max",
                                           "p_bubble", "swc", "sor", "gravity")] + \
               [("n_w", C.c_int32), ("n_o", C.c_int32), ("n_g", C.c_int32)]


def bo_fluid(fl) -> lns_bo_fluid:
    """lns_bo_fluid from an object with the same field names (casegen.BlackOilFluid)."""
    return lns_bo_fluid(*[getattr(fl, k) for k, _ in lns_bo_fluid._fields_])


class lns_tuning(C.Structure):
    _fields_ = [("cluster_max_rows", C.c_int32), ("asm_block", C.c_int32), ("asm_blocks_per_sm", C.c_int32),
                ("set_blocks_per_sm", C.c_int32), ("measured", C.c_int32)]


class lns_server_options(C.Structure):
    _fields_ = [("workers", C.c_int32), ("hbm_budget_bytes", C.c_int64), ("dt_min_fraction", C.c_double)]


class lns_completion(C.Structure):
    _fields_ = [("request_id", C.c_int64), ("model", C.c_int32), ("status", C.c_int32), ("dt", C.c_double),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("stats", lns_step_stats)]


class lns_server_stats(C.Structure):
    _fields_ = [("models", C.c_int32), ("resident_models", C.c_int32), ("queued", C.c_int32),
                ("in_flight", C.c_int32), ("submitted", C.c_int64), ("completed", C.c_int64),
                ("failed", C.c_int64), ("cancelled", C.c_int64), ("admissions", C.c_int64), ("evictions", C.c_int64),
                ("resident_bytes", C.c_int64), ("cell_updates", C.c_int64)]


class lns_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int64), ("total_ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


def _as_dict(s: C.Structure) -> Dict:
    return {k: (getattr(s, k).decode() if isinstance(getattr(s, k), bytes) else getattr(s, k)) for k, _ in s._fields_}


_lib = None
EXPORTS = ["lns_options_default", "lns_model_create", "lns_model_destroy", "lns_set_options", "lns_timestep",
           "lns_newton_iter", "lns_active_set", "lns_dd_expand", "lns_solve_local", "lns_assemble",
           "lns_get_state", "lns_set_state", "lns_get_state_device", "lns_set_state_device", "lns_set_support",
           "lns_set_stream", "lns_reset", "lns_get_support", "lns_kernel_times", "lns_reset_kernel_times",
           "lns_launch_count", "lns_last_error", "lns_active_set_noalloc",
           "lns_server_create", "lns_server_destroy", "lns_server_add_model", "lns_server_submit",
           "lns_server_poll", "lns_server_drain", "lns_server_get_state", "lns_server_get_stats", "lns_server_now",
           "lns_server_cancel", "lns_debug_fault", "lns_advance", "lns_compact", "lns_batch_advance",
           "lns_autotune", "lns_get_tuning", "lns_set_tuning", "lns_tune_pick", "lns_tune_cache_lookup",
           "lns_tune_cache_store", "lns_tune_cache_clear", "lns_bo_assemble", "lns_bo_update"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Load liblns.so (building it first when asked).  Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"liblns.so is not built ({path}); run __graft_entry__.build() first")
    L = C.CDLL(path)
    vp, i32, f64 = C.c_void_p, C.c_int32, C.c_double
    P = C.POINTER
    sig = {
        "lns_options_default": [P(lns_options)],
        "lns_model_create": [P(lns_model_desc), P(lns_options), P(lns_allocator), vp, P(vp)],
        "lns_model_destroy": [vp],
        "lns_set_options": [vp, P(lns_options)],
        "lns_timestep": [vp, f64, P(lns_step_stats)],
        "lns_newton_iter": [vp, f64, P(lns_iter_stats)],
        "lns_active_set": [vp, vp, vp, i32, i32, vp, vp, P(i32)],
        "lns_dd_expand": [vp, vp, vp, i32, vp, vp, vp, vp, vp, P(i32)],
        "lns_solve_local": [vp, f64, vp, vp, vp, P(lns_iter_stats)],
        "lns_assemble": [vp, f64, vp, vp, vp, vp],
        "lns_compact": [vp, vp, vp, vp, P(i32)],
        "lns_batch_advance": [vp, i32, f64, P(lns_dt_control), vp, P(lns_batch_stats)],
        "lns_autotune": [vp, P(lns_tuning)],
        "lns_get_tuning": [vp, P(lns_tuning)],
        "lns_set_tuning": [vp, P(lns_tuning)],
        "lns_get_state": [vp, vp, vp],
        "lns_set_state": [vp, vp, vp, vp, vp],
        "lns_get_state_device": [vp, vp, vp],
        "lns_set_state_device": [vp, vp, vp],
        "lns_set_support": [vp, vp],
        "lns_set_stream": [vp, vp],
        "lns_server_create": [P(lns_server_options), P(vp)],
        "lns_server_destroy": [vp],
        "lns_server_add_model": [vp, P(lns_model_desc), P(lns_options), P(i32)],
        "lns_server_submit": [vp, i32, f64, C.c_int64],
        "lns_server_cancel": [vp, C.c_int64],
        "lns_debug_fault": [vp, i32],
        "lns_advance": [vp, C.c_double, P(lns_dt_control), P(lns_advance_stats)],
        "lns_server_poll": [vp, P(lns_completion), i32, f64, P(i32)],
        "lns_server_drain": [vp, f64],
        "lns_server_get_state": [vp, i32, vp, vp],
        "lns_server_get_stats": [vp, P(lns_server_stats)],
        "lns_reset": [vp],
        "lns_get_support": [vp, vp],
        "lns_kernel_times": [vp, P(lns_kernel_time), i32, P(i32)],
        "lns_reset_kernel_times": [vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.lns_last_error.argtypes = []
    L.lns_last_error.restype = C.c_char_p
    L.lns_launch_count.argtypes = []
    L.lns_launch_count.restype = C.c_int64
    L.lns_server_now.argtypes = [vp]
    L.lns_server_now.restype = C.c_double
    L.lns_tune_pick.argtypes = [i32, vp, vp, vp]
    L.lns_tune_pick.restype = C.c_int32
    L.lns_tune_cache_lookup.argtypes = [i32, i32, i32, i32, P(lns_tuning)]
    L.lns_tune_cache_lookup.restype = C.c_int32
    L.lns_tune_cache_store.argtypes = [i32, i32, i32, i32, P(lns_tuning)]
    L.lns_tune_cache_store.restype = None
    L.lns_tune_cache_clear.argtypes = []
    L.lns_tune_cache_clear.restype = None
    L.lns_active_set_noalloc.argtypes = [i32, vp, vp, vp, vp, vp, f64, f64, i32, i32, vp, vp, P(i32), vp]
    L.lns_active_set_noalloc.restype = C.c_int
    L.lns_bo_assemble.argtypes = [P(lns_bo_fluid), i32] + [vp] * 5 + [i32] + [vp] * 13 + [f64] + [vp] * 5
    L.lns_bo_assemble.restype = C.c_int
    L.lns_bo_update.argtypes = [P(lns_bo_fluid), i32, f64] + [vp] * 9
    L.lns_bo_update.restype = C.c_int
    _lib = L
    return L


def lns_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().lns_launch_count())


def lns_active_set_noalloc(n_cells: int, row_ptr: int, nbr: int, always_bits: int, dp: int, dsw: int,
                           eps_p: float, eps_sw: float, m_layers: int, converged: bool, va_bits: int, vb_bits: int,
                           stream: int = 0) -> int:
    """Allocation-free active-set update on caller-owned DEVICE arrays (integer device
    addresses, 0 for an optional NULL), for callers that cannot allocate device memory.
    Returns is_expand; va_bits is updated in place and vb_bits written."""
    ie = C.c_int32(0)
    _check(load().lns_active_set_noalloc(int(n_cells), row_ptr or None, nbr or None, always_bits or None, dp or None,
                                         dsw or None, float(eps_p), float(eps_sw), int(m_layers), int(bool(converged)),
                                         va_bits or None, vb_bits or None, C.byref(ie), stream or None))
    return int(ie.value)


def lns_bo_assemble(fluid: lns_bo_fluid, n_cells: int, graph: Dict[str, int], state: Dict[str, int],
                    old: Dict[str, int], dt: float, F: int = 0, Jd: int = 0, Jo: int = 0, cnv: int = 0,
                    stream: int = 0) -> None:
    """Black-oil residual, Jacobian and CNV of every cell (lns_bo_assemble) on caller-owned DEVICE
    arrays given by integer addresses: graph keys row_ptr, nbr, trans, pv_ref, depth, n_wells,
    well_cell, well_wi, well_bhp; state and old keys p, sw, sg, rs, sat; outputs 0 for NULL."""
    g = graph
    _check(load().lns_bo_assemble(C.byref(fluid), int(n_cells), g["row_ptr"], g["nbr"], g["trans"], g["pv_ref"],
                                  g["depth"], int(g["n_wells"]), g["well_cell"] or None, g["well_wi"] or None,
                                  g["well_bhp"] or None, state["p"], state["sw"], state["sg"], state["rs"],
                                  state["sat"], old["p"], old["sw"], old["sg"], old["rs"], old["sat"], float(dt),
                                  F or None, Jd or None, Jo or None, cnv or None, stream or None))


def lns_bo_update(fluid: lns_bo_fluid, n_cells: int, sat_chop: float, du: int, state: Dict[str, int],
                  va_bits: int = 0, switched: int = 0, stream: int = 0) -> None:
    """Black-oil update with the primary-variable switch (lns_bo_update) on DEVICE arrays (integer
    addresses; state keys p, sw, sg, rs, sat, updated in place)."""
    _check(load().lns_bo_update(C.byref(fluid), int(n_cells), float(sat_chop), du, va_bits or None, state["p"],
                                state["sw"], state["sg"], state["rs"], state["sat"], switched or None,
                                stream or None))


def lns_batch_advance(models, t_span: float, dt_init: Optional[float] = None, dt_min: Optional[float] = None,
                      dt_max: Optional[float] = None, grow: float = 2.0, cut: float = 0.5, easy_iters: int = 4,
                      allow_noconv: bool = False) -> Tuple[List[Dict], Dict]:
    """Advance every Model in `models` by t_span seconds together (lns_batch_advance), each with its
    own time-step controller; returns the members' statistics and the batch's."""
    ctl = lns_dt_control(float(dt_init if dt_init is not None else t_span),
                         float(dt_min if dt_min is not None else t_span / 1024.0),
                         float(dt_max if dt_max is not None else t_span), float(grow), float(cut), int(easy_iters))
    hs = (C.c_void_p * max(len(models), 1))(*[m.h for m in models])
    outs = (lns_advance_stats * max(len(models), 1))()
    bst = lns_batch_stats()
    rc = load().lns_batch_advance(hs, len(models), float(t_span), C.byref(ctl), outs, C.byref(bst))
    _check(rc, allow=(LNS_ENOCONV,) if allow_noconv else ())
    return [_as_dict(outs[i]) for i in range(len(models))], _as_dict(bst)


def lns_tune_pick(sizes, t_cluster, t_grid) -> int:
    """The autotuner's solver rule (host only): largest size up to which the cluster solver won."""
    a = np.ascontiguousarray(sizes, np.int32)
    b = np.ascontiguousarray(t_cluster, np.float64)
    c = np.ascontiguousarray(t_grid, np.float64)
    return int(load().lns_tune_pick(int(a.shape[0]), a.ctypes.data, b.ctypes.data, c.ctypes.data))


def lns_tune_cache(device: int, krylov_fp32: int, precond: int, n_cells: int) -> Optional[Dict]:
    t = lns_tuning()
    if load().lns_tune_cache_lookup(int(device), int(krylov_fp32), int(precond), int(n_cells), C.byref(t)):
        return _as_dict(t)
    return None


def lns_tune_cache_store(device: int, krylov_fp32: int, precond: int, n_cells: int, **kw) -> None:
    t = lns_tuning(**{k: int(v) for k, v in kw.items()})
    load().lns_tune_cache_store(int(device), int(krylov_fp32), int(precond), int(n_cells), C.byref(t))


def lns_tune_cache_clear() -> None:
    load().lns_tune_cache_clear()


def _check(rc: int, allow=()) -> int:
    if rc != LNS_OK and rc not in allow:
        msg = load().lns_last_error().decode(errors="replace")
        raise LnsError(rc, msg)
    return rc


@dataclasses.dataclass
class Options:
    """Mirror of lns_options (SI units).  Defaults: Algorithm 1, eps = tol_dp = 0.3 psi, m = 2."""
    mode: int = LNS_MODE_LOCAL
    eps_p: float = 0.3 * PSI
    eps_sw: float = 0.0
    m_layers: int = 2
    tol_dp: float = 0.3 * PSI
    tol_cnv: float = 1e-6
    max_newton: int = 25
    max_dd_outer: int = 25
    sat_chop: float = 0.2
    krylov_fp32: int = 0
    precond: int = LNS_PRECOND_BJAC
    krylov_rtol: float = 1e-6
    krylov_maxit: int = 2000
    krylov_fail_rtol: float = 1e-3
    p_scale: float = 0.0
    profile: int = 0
    fp64_fallback: int = 1
    krylov_cluster: int = -1
    autotune: int = 1
    dd_local_newton: int = 1
    dd_local_shrink: int = 0

    def c(self) -> lns_options:
        return lns_options(*[getattr(self, f.name) for f in dataclasses.fields(self)])


def nwords(n: int) -> int:
    return (n + 31) // 32


def mask_to_bits(mask: np.ndarray) -> np.ndarray:
    """Byte mask (n,) -> little-endian uint32 bitset words."""
    mask = np.asarray(mask).astype(bool)
    n = mask.shape[0]
    pad = np.zeros(nwords(n) * 32, dtype=bool)
    pad[:n] = mask
    return np.packbits(pad.reshape(-1, 8), axis=1, bitorder="little").reshape(-1, 4).copy().view(np.uint32).ravel()


def bits_to_mask(bits: np.ndarray, n: int) -> np.ndarray:
    b = np.ascontiguousarray(bits, dtype=np.uint32).view(np.uint8)
    return np.unpackbits(b, bitorder="little")[:n].astype(np.uint8)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def case_desc(case) -> Tuple[lns_model_desc, Dict]:
    """lns_model_desc of a casegen.Case, and the arrays it points into (keep them alive)."""
    keep = dict(
        row_ptr=np.ascontiguousarray(case.row_ptr, np.int32), nbr=np.ascontiguousarray(case.nbr, np.int32),
        trans=np.ascontiguousarray(case.trans, np.float64), pv_ref=np.ascontiguousarray(case.pv_ref, np.float64),
        depth=np.ascontiguousarray(case.depth, np.float64), line_id=np.ascontiguousarray(case.line_id, np.int32),
        always=np.ascontiguousarray(case.always_active, np.uint8),
        well_cell=np.ascontiguousarray(case.well_cell, np.int32),
        well_wi=np.ascontiguousarray(case.well_wi, np.float64),
        well_bhp=np.ascontiguousarray(case.well_bhp, np.float64),
        p0=np.ascontiguousarray(case.p0, np.float64), sw0=np.ascontiguousarray(case.sw0, np.float64))
    fl = case.fluid
    desc = lns_model_desc(
        int(case.n), int(case.nbr.shape[0]), _ptr(keep["row_ptr"]), _ptr(keep["nbr"]), _ptr(keep["trans"]),
        _ptr(keep["pv_ref"]), _ptr(keep["depth"]), _ptr(keep["line_id"]), _ptr(keep["always"]),
        int(case.well_cell.shape[0]), _ptr(keep["well_cell"]), _ptr(keep["well_wi"]), _ptr(keep["well_bhp"]),
        lns_fluid(fl.p_ref, fl.c_r, fl.b_o_ref, fl.c_o, fl.b_w_ref, fl.c_w, fl.rho_o_ref, fl.rho_w_ref,
                  fl.mu_o, fl.mu_w, fl.swc, fl.sor, int(fl.n_w), int(fl.n_o), fl.gravity),
        _ptr(keep["p0"]), _ptr(keep["sw0"]))
    return desc, keep


class Model:
    """A model resident on the GPU (lns_model).  Methods call the C entry points."""

    def __init__(self, case, opts: Optional[Options] = None, use_torch_allocator: bool = True, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("liblns needs a CUDA GPU")
        L = load()
        self.n = int(case.n)
        self.n_adj = int(case.nbr.shape[0])
        self.opts = opts or Options()
        desc, self._keep = case_desc(case)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        self._alloc = None
        if use_torch_allocator:
            dev = torch.cuda.current_device()
            tstream = self._stream

            def _a(ctx, nbytes, s):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, tstream)
                except Exception:  # out of memory is reported to the library as NULL
                    return None

            def _f(ctx, ptr, s):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (ALLOC_FN(_a), FREE_FN(_f))
            self._alloc = lns_allocator(None, self._cb[0], self._cb[1])
        h = C.c_void_p()
        oc = self.opts.c()
        _check(L.lns_model_create(C.byref(desc), C.byref(oc), C.byref(self._alloc) if self._alloc else None,
                                  C.c_void_p(self._stream.cuda_stream), C.byref(h)))
        self.h = h

    # ---- lifecycle ----
    def close(self) -> None:
        if getattr(self, "h", None):
            load().lns_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, opts: Options) -> None:
        self.opts = opts
        oc = opts.c()
        _check(load().lns_set_options(self.h, C.byref(oc)))

    # ---- Newton ----
    def lns_timestep(self, dt: float, allow_noconv: bool = False) -> Dict:
        st = lns_step_stats()
        rc = load().lns_timestep(self.h, float(dt), C.byref(st))
        _check(rc, allow=(LNS_ENOCONV,) if allow_noconv else ())
        d = _as_dict(st)
        d["rc"] = rc
        return d

    def lns_advance(self, t_span: float, dt_init: Optional[float] = None, dt_min: Optional[float] = None,
                    dt_max: Optional[float] = None, grow: float = 2.0, cut: float = 0.5, easy_iters: int = 4,
                    allow_noconv: bool = False) -> Dict:
        """Advance by t_span seconds with the cut/grow time-step controller (lns_advance)."""
        ctl = lns_dt_control(float(dt_init if dt_init is not None else t_span),
                             float(dt_min if dt_min is not None else t_span / 1024.0),
                             float(dt_max if dt_max is not None else t_span), float(grow), float(cut), int(easy_iters))
        st = lns_advance_stats()
        rc = load().lns_advance(self.h, float(t_span), C.byref(ctl), C.byref(st))
        _check(rc, allow=(LNS_ENOCONV,) if allow_noconv else ())
        return _as_dict(st)

    def lns_newton_iter(self, dt: float) -> Dict:
        st = lns_iter_stats()
        _check(load().lns_newton_iter(self.h, float(dt), C.byref(st)))
        return _as_dict(st)

    def run(self, dts) -> List[Dict]:
        return [self.lns_timestep(float(dt)) for dt in dts]

    # ---- set logic ----
    def lns_active_set(self, va_mask, dp, dsw=None, converged: bool = False) -> Tuple[np.ndarray, np.ndarray, int]:
        va = mask_to_bits(va_mask)
        vb = np.zeros_like(va)
        dp = np.ascontiguousarray(dp, np.float64)
        dsw = None if dsw is None else np.ascontiguousarray(dsw, np.float64)
        ie = C.c_int32(0)
        _check(load().lns_active_set(self.h, _ptr(dp), None if dsw is None else _ptr(dsw), 0, int(bool(converged)),
                                     _ptr(va), _ptr(vb), C.byref(ie)))
        return bits_to_mask(va, self.n), bits_to_mask(vb, self.n), int(ie.value)

    def lns_dd_expand(self, vb_k_mask, dp, vt_mask, dsw=None):
        vb = mask_to_bits(vb_k_mask)
        vt = mask_to_bits(vt_mask)
        va_n = np.zeros_like(vt)
        vb_n = np.zeros_like(vt)
        vd_n = np.zeros_like(vt)
        dp = np.ascontiguousarray(dp, np.float64)
        dsw = None if dsw is None else np.ascontiguousarray(dsw, np.float64)
        ie = C.c_int32(0)
        _check(load().lns_dd_expand(self.h, _ptr(dp), None if dsw is None else _ptr(dsw), 0, _ptr(vb), _ptr(vt),
                                    _ptr(va_n), _ptr(vb_n), _ptr(vd_n), C.byref(ie)))
        n = self.n
        return (bits_to_mask(vt, n), bits_to_mask(va_n, n), bits_to_mask(vb_n, n), bits_to_mask(vd_n, n),
                int(ie.value))

    # ---- local solve / assembly ----
    def lns_solve_local(self, dt: float, va_mask) -> Tuple[np.ndarray, np.ndarray, Dict]:
        va = mask_to_bits(va_mask)
        dp = np.zeros(self.n)
        dsw = np.zeros(self.n)
        st = lns_iter_stats()
        _check(load().lns_solve_local(self.h, float(dt), _ptr(va), _ptr(dp), _ptr(dsw), C.byref(st)))
        return dp, dsw, _as_dict(st)

    def lns_compact(self, va_mask) -> Tuple[np.ndarray, np.ndarray]:
        """Compaction of V_A: (act, inv) -- the ascending active cells and the inverse map
        (-1 outside V_A)."""
        va = mask_to_bits(va_mask)
        act = np.zeros(max(self.n, 1), np.int32)
        inv = np.zeros(max(self.n, 1), np.int32)
        na = C.c_int32(0)
        _check(load().lns_compact(self.h, _ptr(va), _ptr(act), _ptr(inv), C.byref(na)))
        return act[: na.value].copy(), inv[: self.n].copy()

    def lns_assemble(self, dt: float, va_mask):
        va = mask_to_bits(va_mask)
        F = np.zeros((self.n, 2))
        Jd = np.zeros((self.n, 2, 2))
        Jo = np.zeros((max(self.n_adj, 1), 2, 2))
        _check(load().lns_assemble(self.h, float(dt), _ptr(va), _ptr(F), _ptr(Jd), _ptr(Jo)))
        return F, Jd, Jo[: self.n_adj]

    # ---- state ----
    def lns_get_state(self) -> Tuple[np.ndarray, np.ndarray]:
        p = np.zeros(self.n)
        sw = np.zeros(self.n)
        _check(load().lns_get_state(self.h, _ptr(p), _ptr(sw)))
        return p, sw

    def lns_set_state(self, p, sw, pn=None, swn=None) -> None:
        arrs = [None if a is None else np.ascontiguousarray(a, np.float64) for a in (p, sw, pn, swn)]
        _check(load().lns_set_state(self.h, *[None if a is None else _ptr(a) for a in arrs]))

    def lns_set_state_ptrs(self, p_ptr: int, sw_ptr: int) -> None:
        """Host pointers (e.g. pinned torch tensors) of n doubles each."""
        _check(load().lns_set_state(self.h, C.c_void_p(p_ptr), C.c_void_p(sw_ptr), None, None))

    def lns_get_state_ptrs(self, p_ptr: int, sw_ptr: int) -> None:
        _check(load().lns_get_state(self.h, C.c_void_p(p_ptr), C.c_void_p(sw_ptr)))

    def lns_get_state_device(self, p_ptr: int, sw_ptr: int) -> None:
        _check(load().lns_get_state_device(self.h, C.c_void_p(p_ptr), C.c_void_p(sw_ptr)))

    def lns_reset(self) -> None:
        _check(load().lns_reset(self.h))

    def lns_get_support(self) -> np.ndarray:
        bits = np.zeros(nwords(self.n), np.uint32)
        _check(load().lns_get_support(self.h, _ptr(bits)))
        return bits_to_mask(bits, self.n)

    def lns_set_support(self, bits: Optional[np.ndarray]) -> None:
        """Restore the previous timestep's support (bitset words, e.g. mask_to_bits of
        lns_get_support); None forgets it."""
        if bits is None:
            _check(load().lns_set_support(self.h, None))
            return
        b = np.ascontiguousarray(bits, np.uint32)
        _check(load().lns_set_support(self.h, _ptr(b)))

    def lns_set_state_device(self, p_ptr: int, sw_ptr: int) -> None:
        _check(load().lns_set_state_device(self.h, C.c_void_p(p_ptr), C.c_void_p(sw_ptr)))

    def lns_kernel_times(self) -> List[Dict]:
        arr = (lns_kernel_time * 16)()
        cnt = C.c_int32(0)
        _check(load().lns_kernel_times(self.h, arr, 16, C.byref(cnt)))
        return [_as_dict(arr[k]) for k in range(cnt.value)]

    def lns_reset_kernel_times(self) -> None:
        _check(load().lns_reset_kernel_times(self.h))

    # ---- autotuning ----
    def lns_autotune(self) -> Dict:
        """Measure launch shapes and the cluster/grid solver threshold on this model (lns_autotune)."""
        t = lns_tuning()
        _check(load().lns_autotune(self.h, C.byref(t)))
        return _as_dict(t)

    def lns_get_tuning(self) -> Dict:
        t = lns_tuning()
        _check(load().lns_get_tuning(self.h, C.byref(t)))
        return _as_dict(t)

    def lns_set_tuning(self, tuning: Optional[Dict] = None, **kw) -> None:
        """Set the tuning (keys of lns_tuning; missing keys keep their current value); None: back to
        the cached or default tuning."""
        if tuning is None and not kw:
            _check(load().lns_set_tuning(self.h, None))
            return
        cur = self.lns_get_tuning()
        cur.update(tuning or {})
        cur.update(kw)
        t = lns_tuning(**{k: int(v) for k, v in cur.items()})
        _check(load().lns_set_tuning(self.h, C.byref(t)))

    def lns_debug_fault(self, code: int) -> None:
        """Inject a solver fault for failure tests (1: a barrier wait runs out, 2: breakdown; 0: none)."""
        _check(load().lns_debug_fault(self.h, int(code)))


class Server:
    """A request loop over many resident models (lns_server_*): submit 'advance model k by dt'
    requests from any thread; poll for completions with their timestamps (seconds on the
    server clock) and step statistics."""

    def __init__(self, workers: int = 4, hbm_budget_bytes: int = 0, dt_min_fraction: float = 0.0):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("liblns needs a CUDA GPU")
        h = C.c_void_p()
        o = lns_server_options(int(workers), int(hbm_budget_bytes), float(dt_min_fraction))
        _check(load().lns_server_create(C.byref(o), C.byref(h)))
        self.h = h
        self.n = []

    def add_model(self, case, opts: Optional[Options] = None) -> int:
        desc, keep = case_desc(case)  # copied by the server during the call
        oc = (opts or Options()).c()
        mid = C.c_int32()
        _check(load().lns_server_add_model(self.h, C.byref(desc), C.byref(oc), C.byref(mid)))
        del keep
        self.n.append(int(case.n))
        return int(mid.value)

    def submit(self, model: int, dt: float, request_id: int) -> None:
        _check(load().lns_server_submit(self.h, int(model), float(dt), int(request_id)))

    def cancel(self, request_id: int) -> bool:
        """Cancel a queued request; False if it is not queued (running, finished or unknown)."""
        return load().lns_server_cancel(self.h, int(request_id)) == LNS_OK

    def poll(self, cap: int = 256, timeout_s: float = 0.0) -> List[Dict]:
        buf = (lns_completion * cap)()
        cnt = C.c_int32()
        _check(load().lns_server_poll(self.h, buf, int(cap), float(timeout_s), C.byref(cnt)))
        out = []
        for c in buf[: cnt.value]:
            d = {k: getattr(c, k) for k, _ in c._fields_ if k != "stats"}
            d["stats"] = _as_dict(c.stats)
            out.append(d)
        return out

    def drain(self, timeout_s: float = 600.0) -> None:
        _check(load().lns_server_drain(self.h, float(timeout_s)))

    def get_state(self, model: int) -> Tuple[np.ndarray, np.ndarray]:
        n = self.n[model]
        p = np.empty(n, np.float64)
        sw = np.empty(n, np.float64)
        _check(load().lns_server_get_state(self.h, int(model), _ptr(p), _ptr(sw)))
        return p, sw

    def stats(self) -> Dict:
        st = lns_server_stats()
        _check(load().lns_server_get_stats(self.h, C.byref(st)))
        return _as_dict(st)

    def now(self) -> float:
        return float(load().lns_server_now(self.h))

    def close(self) -> None:
        if getattr(self, "h", None):
            load().lns_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
