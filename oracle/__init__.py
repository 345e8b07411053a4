"""CPU FP64 oracle for the localized fully implicit Newton solver (arXiv 2008.01539).

TEST INFRASTRUCTURE ONLY.  The oracle checks the CUDA path; it is called by the tests,
the smoke check and the benchmark's CPU-baseline leg, never by the library.  It shares
no code with the CUDA path: its arithmetic lives in ``lns_oracle.c`` (plain serial C,
double precision), compiled here with gcc and called through ctypes.

What it computes (paper passages in ``lns_oracle.h``): the oil-water backward-Euler
TPFA residual and Jacobian (Appendix A), standard Newton (Section 4.1), localized
Newton (Section 4.3, Algorithm 1), adaptive nonlinear domain decomposition
(Section 4.4, Algorithm 2), with a hand-written block sparse LU as the linear step.
``blackoil.py`` holds the three-phase black-oil model with primary-variable switching (the
black-oil form of Section 3.1's variable substitution), in numpy.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lns_oracle.c")
_HDR = os.path.join(_HERE, "lns_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblns_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no floating-point contraction, so results do not
    depend on whether the host has fused multiply-add)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Fluid(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("p_ref", "c_r", "b_o_ref", "c_o", "b_w_ref", "c_w", "rho_o_ref",
                                           "rho_w_ref", "mu_o", "mu_w", "swc", "sor")] + \
               [("n_w", C.c_int32), ("n_o", C.c_int32), ("gravity", C.c_double)]


class _Model(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_adj", C.c_int32),
                ("row_ptr", C.c_void_p), ("nbr", C.c_void_p), ("trans", C.c_void_p),
                ("pv_ref", C.c_void_p), ("depth", C.c_void_p), ("always", C.c_void_p),
                ("n_wells", C.c_int32), ("well_cell", C.c_void_p), ("well_wi", C.c_void_p),
                ("well_bhp", C.c_void_p), ("fl", _Fluid)]


class _Opts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("eps_p", C.c_double), ("eps_sw", C.c_double),
                ("m_layers", C.c_int32), ("tol_dp", C.c_double), ("tol_cnv", C.c_double),
                ("max_newton", C.c_int32), ("sat_chop", C.c_double), ("max_dd_outer", C.c_int32),
                ("dd_local_newton", C.c_int32), ("dd_local_shrink", C.c_int32),
                ("linear", C.c_int32), ("lin_rtol", C.c_double), ("lin_maxit", C.c_int32)]


class StepStats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("cell_updates", C.c_int64),
                ("n_subdomains", C.c_int32), ("dd_outer", C.c_int32),
                ("last_max_dp", C.c_double), ("last_cnv", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _configure(L):
    vp = C.c_void_p
    L.orc_assemble.argtypes = [C.POINTER(_Model), vp, vp, vp, vp, C.c_double, vp, vp, vp]
    L.orc_cnv.argtypes = [C.POINTER(_Model), vp, vp, C.c_double, vp]
    L.orc_lu_solve.argtypes = [C.c_int32, vp, vp, vp, vp, vp, vp, C.POINTER(C.c_int64)]
    L.orc_lu_solve.restype = C.c_int
    L.orc_ilu0_bicgstab.argtypes = [C.c_int32, vp, vp, vp, vp, vp, vp, C.c_double, C.c_int32,
                                    C.POINTER(C.c_int32)]
    L.orc_ilu0_bicgstab.restype = C.c_int
    L.orc_dilate.argtypes = [C.POINTER(_Model), vp, C.c_int32, vp]
    L.orc_boundary.argtypes = [C.POINTER(_Model), vp, vp]
    L.orc_outer_halo.argtypes = [C.POINTER(_Model), vp, vp]
    L.orc_active_set_update.argtypes = [C.POINTER(_Model), C.POINTER(_Opts), vp, vp, vp, C.c_int32,
                                        vp, C.POINTER(C.c_int32)]
    L.orc_dd_expand.argtypes = [C.POINTER(_Model), C.POINTER(_Opts), vp, vp, vp, vp, vp, vp, vp,
                                C.POINTER(C.c_int32)]
    L.orc_local_solve.argtypes = [C.POINTER(_Model), C.POINTER(_Opts), vp, vp, vp, vp, C.c_double, vp,
                                  vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.orc_local_solve.restype = C.c_int
    L.orc_timestep.argtypes = [C.POINTER(_Model), C.POINTER(_Opts), vp, vp, vp, C.POINTER(C.c_int32),
                               C.c_double, C.POINTER(StepStats), vp, C.c_int32, vp]
    L.orc_timestep.restype = C.c_int
    L.orc_initial_set.argtypes = [C.POINTER(_Model), C.POINTER(_Opts), vp, C.c_int32, vp]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(C.CDLL(build()))
    return _lib


def build_variant(src_text: str, out_dir: str, name: str) -> str:
    """Compile a modified copy of the oracle source (used by the tests that plant a mistake in
    the oracle to show that a pin catches it); returns the library path."""
    src = os.path.join(out_dir, name + ".c")
    with open(src, "w") as fh:
        fh.write(src_text)
    import shutil
    shutil.copy(_HDR, os.path.join(out_dir, "lns_oracle.h"))
    so = os.path.join(out_dir, "lib" + name + ".so")
    subprocess.run(["gcc", "-O1", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
                    "-o", so, src, "-lm"], check=True)
    return so


class use_library:
    """Context manager: route every oracle call through the library at `path` (a variant
    built by build_variant), restoring the regular build afterwards."""

    def __init__(self, path: str) -> None:
        self.path = path

    def __enter__(self):
        global _lib
        lib()
        with _lock:
            self._saved = _lib
            _lib = _configure(C.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self._saved
        return False


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


@dataclasses.dataclass
class Options:
    """Solver options.  mode: 0 standard Newton, 1 Algorithm 1, 2 Algorithm 2, 3 residual-based
    active sets (unconverged cells inflated by m_layers; the Lu-Beckner estimate the paper cites).
    Cutoffs and tolerances in SI (Pa); eps_p = 0.3 psi as in the paper's runs.  Algorithm 2
    variants: dd_local_newton steps per subdomain visit (to local convergence), dd_local_shrink
    (later steps of a visit solve only the previous step's support within the subdomain)."""
    mode: int = 1
    eps_p: float = 0.3 * 6894.757293168
    eps_sw: float = 0.0
    m_layers: int = 2
    tol_dp: float = 0.3 * 6894.757293168
    tol_cnv: float = 1e-6
    max_newton: int = 25
    sat_chop: float = 0.2
    max_dd_outer: int = 25
    dd_local_newton: int = 1
    dd_local_shrink: int = 0
    linear: int = 0          # 0 block sparse LU, 1 block ILU(0)-preconditioned BiCGStab
    lin_rtol: float = 1e-10
    lin_maxit: int = 5000

    def _c(self) -> _Opts:
        return _Opts(self.mode, self.eps_p, self.eps_sw, self.m_layers, self.tol_dp, self.tol_cnv,
                     self.max_newton, self.sat_chop, self.max_dd_outer, self.dd_local_newton,
                     self.dd_local_shrink, self.linear, self.lin_rtol, self.lin_maxit)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Model:
    """The oracle's view of a model: holds contiguous copies of the case arrays."""

    def __init__(self, case) -> None:
        self.case = case
        self.n = int(case.n)
        self._keep = dict(
            row_ptr=np.ascontiguousarray(case.row_ptr, np.int32),
            nbr=np.ascontiguousarray(case.nbr, np.int32),
            trans=np.ascontiguousarray(case.trans, np.float64),
            pv_ref=np.ascontiguousarray(case.pv_ref, np.float64),
            depth=np.ascontiguousarray(case.depth, np.float64),
            always=np.ascontiguousarray(case.always_active, np.uint8),
            well_cell=np.ascontiguousarray(case.well_cell, np.int32),
            well_wi=np.ascontiguousarray(case.well_wi, np.float64),
            well_bhp=np.ascontiguousarray(case.well_bhp, np.float64),
        )
        fl = case.fluid
        k = self._keep
        self.c = _Model(self.n, int(case.nbr.shape[0]), _ptr(k["row_ptr"]), _ptr(k["nbr"]), _ptr(k["trans"]),
                        _ptr(k["pv_ref"]), _ptr(k["depth"]), _ptr(k["always"]), int(case.well_cell.shape[0]),
                        _ptr(k["well_cell"]), _ptr(k["well_wi"]), _ptr(k["well_bhp"]),
                        _Fluid(fl.p_ref, fl.c_r, fl.b_o_ref, fl.c_o, fl.b_w_ref, fl.c_w, fl.rho_o_ref,
                               fl.rho_w_ref, fl.mu_o, fl.mu_w, fl.swc, fl.sor, int(fl.n_w), int(fl.n_o),
                               fl.gravity))

    @property
    def n_adj(self) -> int:
        return int(self._keep["nbr"].shape[0])


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def assemble(m: Model, p, sw, pn, swn, dt: float) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Full-domain residual F (n, 2) and Jacobian blocks: diagonal (n, 2, 2) and
    off-diagonal per adjacency entry (n_adj, 2, 2)."""
    p, sw, pn, swn = _f64(p), _f64(sw), _f64(pn), _f64(swn)
    F = np.zeros((m.n, 2))
    Jd = np.zeros((m.n, 2, 2))
    Jo = np.zeros((m.n_adj, 2, 2))
    lib().orc_assemble(C.byref(m.c), _ptr(p), _ptr(sw), _ptr(pn), _ptr(swn), float(dt), _ptr(F), _ptr(Jd), _ptr(Jo))
    return F, Jd, Jo


def residual(m: Model, p, sw, pn, swn, dt: float) -> np.ndarray:
    p, sw, pn, swn = _f64(p), _f64(sw), _f64(pn), _f64(swn)
    F = np.zeros((m.n, 2))
    lib().orc_assemble(C.byref(m.c), _ptr(p), _ptr(sw), _ptr(pn), _ptr(swn), float(dt), _ptr(F), None, None)
    return F


def cnv(m: Model, p, F, dt: float) -> np.ndarray:
    p, F = _f64(p), _f64(F)
    out = np.zeros(m.n)
    lib().orc_cnv(C.byref(m.c), _ptr(p), _ptr(F), float(dt), _ptr(out))
    return out


def lu_solve(row_ptr, col, diag, off, rhs) -> Tuple[np.ndarray, int]:
    """Hand-written block sparse LU solve.  diag (nb, 2, 2), off (nnz, 2, 2), rhs (nb, 2)."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    diag, off, rhs = _f64(diag), _f64(off), _f64(rhs)
    nb = row_ptr.shape[0] - 1
    x = np.zeros((nb, 2))
    fill = C.c_int64(0)
    rc = lib().orc_lu_solve(nb, _ptr(row_ptr), _ptr(col), _ptr(diag), _ptr(off), _ptr(rhs), _ptr(x), C.byref(fill))
    if rc != 0:
        raise ArithmeticError("singular block pivot in the oracle's sparse LU")
    return x, int(fill.value)


def ilu0_bicgstab(row_ptr, col, diag, off, rhs, rtol: float = 1e-10, maxit: int = 5000):
    """BiCGStab with a block ILU(0) preconditioner on the block system (as lu_solve).
    Returns (x, status, iterations): status 0 converged, 1 maxit, 2 breakdown."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    diag, off, rhs = _f64(diag), _f64(off), _f64(rhs)
    nb = row_ptr.shape[0] - 1
    x = np.zeros((nb, 2))
    its = C.c_int32(0)
    st = lib().orc_ilu0_bicgstab(nb, _ptr(row_ptr), _ptr(col), _ptr(diag), _ptr(off), _ptr(rhs), _ptr(x),
                                 float(rtol), int(maxit), C.byref(its))
    return x, int(st), int(its.value)


def dilate(m: Model, seed, layers: int) -> np.ndarray:
    seed = _u8(seed)
    out = np.zeros(m.n, np.uint8)
    lib().orc_dilate(C.byref(m.c), _ptr(seed), int(layers), _ptr(out))
    return out


def boundary(m: Model, va) -> np.ndarray:
    va = _u8(va)
    out = np.zeros(m.n, np.uint8)
    lib().orc_boundary(C.byref(m.c), _ptr(va), _ptr(out))
    return out


def outer_halo(m: Model, va) -> np.ndarray:
    va = _u8(va)
    out = np.zeros(m.n, np.uint8)
    lib().orc_outer_halo(C.byref(m.c), _ptr(va), _ptr(out))
    return out


def active_set_update(m: Model, o: Options, va, dp, dsw, converged: bool):
    """Algorithm 1, steps 3-4, on a given update.  Returns (new V_A, new V_B, is_expand)."""
    va = _u8(va).copy()
    dp, dsw = _f64(dp), _f64(dsw)
    vb = np.zeros(m.n, np.uint8)
    ie = C.c_int32(0)
    oc = o._c()
    lib().orc_active_set_update(C.byref(m.c), C.byref(oc), _ptr(va), _ptr(dp), _ptr(dsw), int(bool(converged)),
                                _ptr(vb), C.byref(ie))
    return va, vb, int(ie.value)


def dd_expand(m: Model, o: Options, vb_k, dp, dsw, vt):
    """Algorithm 2, one expansion step.  Returns (V_T, V_A^{k+1}, V_B^{k+1}, V_dB^{k+1}, is_expand)."""
    vb_k = _u8(vb_k)
    vt = _u8(vt).copy()
    dp, dsw = _f64(dp), _f64(dsw)
    va_n = np.zeros(m.n, np.uint8)
    vb_n = np.zeros(m.n, np.uint8)
    vd_n = np.zeros(m.n, np.uint8)
    ie = C.c_int32(0)
    oc = o._c()
    lib().orc_dd_expand(C.byref(m.c), C.byref(oc), _ptr(vb_k), _ptr(dp), _ptr(dsw), _ptr(vt), _ptr(va_n),
                        _ptr(vb_n), _ptr(vd_n), C.byref(ie))
    return vt, va_n, vb_n, vd_n, int(ie.value)


def local_solve(m: Model, o: Options, p, sw, pn, swn, dt: float, va):
    """One localized Newton step (no state change).  Returns (dp, dsw, max CNV over V_A, max |dp|)."""
    p, sw, pn, swn = _f64(p), _f64(sw), _f64(pn), _f64(swn)
    va = _u8(va)
    dp = np.zeros(m.n)
    dsw = np.zeros(m.n)
    cm = C.c_double(0)
    dm = C.c_double(0)
    oc = o._c()
    rc = lib().orc_local_solve(C.byref(m.c), C.byref(oc), _ptr(p), _ptr(sw), _ptr(pn), _ptr(swn), float(dt),
                               _ptr(va), _ptr(dp), _ptr(dsw), C.byref(cm), C.byref(dm))
    if rc != 0:
        raise ArithmeticError("singular block pivot in the oracle's sparse LU")
    return dp, dsw, float(cm.value), float(dm.value)


def initial_set(m: Model, o: Options, prev_supp, has_prev: bool) -> np.ndarray:
    prev_supp = _u8(prev_supp)
    out = np.zeros(m.n, np.uint8)
    oc = o._c()
    lib().orc_initial_set(C.byref(m.c), C.byref(oc), _ptr(prev_supp), int(bool(has_prev)), _ptr(out))
    return out


class Sim:
    """Stateful oracle simulation: u = (p, Sw) and the previous step's support set."""

    def __init__(self, case, opts: Optional[Options] = None) -> None:
        self.m = Model(case)
        self.o = opts or Options()
        self.p = _f64(case.p0).copy()
        self.sw = _f64(case.sw0).copy()
        self.prev_supp = np.zeros(case.n, np.uint8)
        self.has_prev = C.c_int32(0)

    def timestep(self, dt: float, trace_cap: int = 256):
        """One timestep; returns the step statistics, the per-iteration active-set sizes
        ('trace') and the union of the sets solved during the step ('union')."""
        st = StepStats()
        trace = np.zeros(trace_cap, np.int32)
        union = np.zeros(self.m.n, np.uint8)
        oc = self.o._c()
        lib().orc_timestep(C.byref(self.m.c), C.byref(oc), _ptr(self.p), _ptr(self.sw), _ptr(self.prev_supp),
                           C.byref(self.has_prev), float(dt), C.byref(st), _ptr(trace), trace_cap, _ptr(union))
        d = st.as_dict()
        d["trace"] = trace[: min(st.iterations, trace_cap)].tolist()
        d["union"] = union
        return d

    def run(self, dts) -> list:
        return [self.timestep(float(dt)) for dt in dts]

    def advance(self, t_span: float, dt_init: float, dt_min: float, dt_max: float, grow: float = 2.0,
                cut: float = 0.5, easy_iters: int = 4) -> dict:
        """Advance by t_span with the usual cut/grow controller: a step that fails (Newton
        iteration limit or a singular local solve) is undone and retried with dt * cut; a step of
        at most easy_iters iterations lets the next grow to min(dt * grow, dt_max); the last step
        ends exactly at t_span.  Returns counts, the time advanced and the next dt."""
        out = dict(status=0, steps=0, cuts=0, iterations=0, krylov_iters=0, cell_updates=0, t_done=0.0,
                   dt_next=0.0, dts=[])
        t, dt = 0.0, min(dt_init, dt_max)
        while t < t_span:
            h = min(dt, t_span - t)
            saved = (self.p.copy(), self.sw.copy(), self.prev_supp.copy(), self.has_prev.value)
            st = self.timestep(h)
            out["iterations"] += st["iterations"]
            out["cell_updates"] += st["cell_updates"]
            if st["status"] == 0:
                t = t_span if h == t_span - t else t + h
                out["steps"] += 1
                out["dts"].append(h)
                if st["iterations"] <= easy_iters:
                    dt = min(dt * grow, dt_max)
                continue
            self.p, self.sw, self.prev_supp = saved[0], saved[1], saved[2]
            self.has_prev.value = saved[3]
            out["cuts"] += 1
            dt = h * cut
            if dt < dt_min:
                out["status"] = -4
                break
        out["t_done"], out["dt_next"] = t, dt
        return out
