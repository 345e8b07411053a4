"""The black-oil physics of the CUDA path (csrc/bo_physics.cuh: cell properties, face fluxes,
producer terms, CNV and the update with Section 3.1's variable switch), built for the host, against
the black-oil oracle (oracle/blackoil.py); and its 3x3 block arithmetic (csrc/blk3.cuh: block
inverse, the fracture-line block's block Thomas factorization and solve) against numpy's dense
inverse and solve.

The header's derivatives are written out by hand; the oracle's come from forward-mode dual
numbers, so the Jacobians agree only if every hand-written chain rule is right.  Residuals and
Jacobians agree to rounding (1e-11 of each component's scale); the update and switch bit for bit.
States: mixed (cells with and without free gas), cells at the Corey clamps, and the state the
oracle reaches on the small 3D model after gas has appeared.
"""
import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from oracle import blackoil as B
from paper_2008_01539_gb300 import casegen as cg

PSI = cg.PSI
HERE = os.path.dirname(os.path.abspath(__file__))
_FIELDS = ("p_ref", "c_r", "b_w_ref", "c_w", "rho_w_sc", "mu_w", "b_o_ref", "c_o", "kappa", "rho_o_sc", "mu_o",
           "b_g_per_pa", "rho_g_sc", "mu_g", "rs_max", "p_bubble", "swc", "sor", "gravity")


class _Fluid(C.Structure):
    _fields_ = [(k, C.c_double) for k in _FIELDS] + [("n_w", C.c_int), ("n_o", C.c_int), ("n_g", C.c_int)]


def _fluid(fl):
    return _Fluid(*[getattr(fl, k) for k in _FIELDS], fl.n_w, fl.n_o, fl.n_g)


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    O.build()
    out = tmp_path_factory.mktemp("bo_host") / "bo_host.so"
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-o", str(out),
                    os.path.join(HERE, "harness", "bo_host.cpp")], check=True)
    L = C.CDLL(str(out))
    L.bo_host_assemble.restype = None
    L.bo_host_update.restype = C.c_int
    return L


def _p(a):
    return C.c_void_p(a.ctypes.data)


def _assemble_host(L, bo, st, old, dt):
    c, n = bo.case, bo.n
    arrs = dict(rp=np.ascontiguousarray(c.row_ptr, np.int32), nbr=np.ascontiguousarray(c.nbr, np.int32),
                T=np.ascontiguousarray(c.trans, np.float64), pv=np.ascontiguousarray(c.pv_ref, np.float64),
                z=np.ascontiguousarray(c.depth, np.float64), wc=np.ascontiguousarray(c.well_cell, np.int32),
                wi=np.ascontiguousarray(c.well_wi, np.float64), bhp=np.ascontiguousarray(c.well_bhp, np.float64))
    u = [np.ascontiguousarray(a, np.float64) for a in (st.p, st.sw, st.x, old.p, old.sw, old.x)]
    sat, sat_o = np.ascontiguousarray(st.sat, np.uint8), np.ascontiguousarray(old.sat, np.uint8)
    F = np.zeros((n, 3))
    Jd = np.zeros((n, 3, 3))
    Jo = np.zeros((c.nbr.shape[0], 3, 3))
    cv = np.zeros(n)
    f = _fluid(bo.fluid)
    L.bo_host_assemble(C.byref(f), n, _p(arrs["rp"]), _p(arrs["nbr"]), _p(arrs["T"]), _p(arrs["pv"]), _p(arrs["z"]),
                       int(c.well_cell.shape[0]), _p(arrs["wc"]), _p(arrs["wi"]), _p(arrs["bhp"]), _p(u[0]), _p(u[1]),
                       _p(u[2]), _p(sat), _p(u[3]), _p(u[4]), _p(u[5]), _p(sat_o), C.c_double(dt), _p(F), _p(Jd),
                       _p(Jo), _p(cv))
    return F, Jd, Jo, cv


def _model():
    return cg.blackoil(cg.small_dfn3d(12, 10, 4, seed=9), p_init=3800.0 * PSI, bhp=2000.0 * PSI)


def _mixed(bo, seed, clamps=False):
    rng = np.random.default_rng(seed)
    n, fl = bo.n, bo.fluid
    z = bo.case.depth - bo.case.depth.min()
    p = 3000.0 * PSI + 700.0 * cg.GRAVITY * z + rng.normal(0.0, 5e3, n)
    sw = rng.uniform(0.25, 0.5, n)
    sat = (rng.random(n) < 0.5).astype(np.uint8)
    sg = np.where(sat == 1, rng.uniform(0.02, 0.2, n), 0.0)
    rs_s = fl.rs_max * p / fl.p_bubble
    rs = np.where(sat == 1, rs_s, rng.uniform(0.5, 0.9, n) * rs_s)
    if clamps:
        k = rng.choice(n, n // 4, replace=False)
        sw[k[: len(k) // 2]] = rng.uniform(0.1, 0.2, len(k) // 2)       # water below connate
        kk = k[len(k) // 2:]
        sat[kk] = 1
        sg[kk] = 0.85 - sw[kk]  # So = 0.15 < sor
        rs[kk] = rs_s[kk]
        assert np.sum(sw < fl.swc) > 0 and np.sum(1.0 - sw - sg < fl.sor) > 0
    return B.State(p, sw, sg, rs, sat)


def _compare(F, Jd, Jo, cv, Fr, Jdr, Jor, cvr):
    for r in range(3):
        s = np.max(np.abs(Fr[:, r]))
        assert np.max(np.abs(F[:, r] - Fr[:, r])) <= 1e-11 * s, ("F", r)
        for k in range(3):
            for J, Jr, name in ((Jd, Jdr, "Jd"), (Jo, Jor, "Jo")):
                s = np.max(np.abs(Jr[:, r, k]))
                assert np.max(np.abs(J[:, r, k] - Jr[:, r, k])) <= 1e-11 * s + 1e-300, (name, r, k)
    assert np.max(np.abs(cv - cvr)) <= 1e-11 * np.max(cvr)


@pytest.mark.parametrize("clamps", [False, True])
def test_assembly_matches_oracle_mixed_states(host, clamps):
    bo = _model()
    st, old = _mixed(bo, 1, clamps), _mixed(bo, 2, clamps)
    dt = 2.0 * cg.DAY
    F, Jd, Jo, cv = _assemble_host(host, bo, st, old, dt)
    Fr, Jdr, Jor = B.assemble(bo, st, old, dt)
    _compare(F, Jd, Jo, cv, Fr, Jdr, Jor, B.cnv(bo, st, Fr, dt))


def test_assembly_matches_oracle_after_gas_appears(host):
    bo = cg.small_blackoil3d()
    sim = B.Sim(bo, B.Options(mode=0))
    old = sim.st.copy()
    dt = float(bo.case.dt_schedule[0])
    st = old.copy()
    for _ in range(2):  # two Newton iterations in: the fracture cells near the producer hold free gas
        du, _, _ = B.local_solve(bo, st, old, dt, np.ones(bo.n, np.uint8))
        st, _ = B.apply_update(bo.fluid, st, du, np.ones(bo.n, np.uint8))
    assert 0 < st.sat.sum() < bo.n
    F, Jd, Jo, cv = _assemble_host(host, bo, st, old, dt)
    Fr, Jdr, Jor = B.assemble(bo, st, old, dt)
    _compare(F, Jd, Jo, cv, Fr, Jdr, Jor, B.cnv(bo, st, Fr, dt))


@pytest.mark.parametrize("chop", [0.0, 0.2])
def test_update_and_switch_match_oracle_bit_for_bit(host, chop):
    bo = _model()
    fl = bo.fluid
    rng = np.random.default_rng(3)
    st = _mixed(bo, 4)
    n = bo.n
    # updates that cross the bubble point both ways, and chop-sized saturation steps
    du = np.stack([rng.normal(0.0, 300.0 * PSI, n), rng.normal(0.0, 0.15, n),
                   np.where(st.sat == 1, rng.normal(0.0, 0.15, n), rng.normal(0.0, 0.5, n) * fl.rs_max)], axis=1)
    ref_du = du.copy()
    if chop > 0.0:  # the oracle chops in its Newton step: |dSw|, and |dSg| where free gas is present
        ref_du[:, 1] = np.clip(ref_du[:, 1], -chop, chop)
        s = st.sat == 1
        ref_du[s, 2] = np.clip(ref_du[s, 2], -chop, chop)
    ref, ref_sw = B.apply_update(fl, st, ref_du, np.ones(n, np.uint8))
    h = st.copy()
    sw_mask = np.zeros(n, np.uint8)
    f = _fluid(fl)
    du_c = np.ascontiguousarray(du)
    k = host.bo_host_update(C.byref(f), C.c_double(chop), n, _p(du_c), _p(h.p), _p(h.sw), _p(h.sg), _p(h.rs),
                            _p(h.sat), _p(sw_mask))
    assert k == int(ref_sw.sum()) and 0 < k
    assert np.any((st.sat == 1) & (ref.sat == 0)) and np.any((st.sat == 0) & (ref.sat == 1))
    assert np.array_equal(sw_mask.astype(bool), ref_sw)
    assert np.array_equal(h.sat, ref.sat)
    for a, b in ((h.p, ref.p), (h.sw, ref.sw), (h.sg, ref.sg), (h.rs, ref.rs)):
        assert np.array_equal(a, b)


# ---------------------------------------------------------------------------------------
# 3x3 block arithmetic of the black-oil preconditioner (csrc/blk3.cuh)
# ---------------------------------------------------------------------------------------
def test_block_inverse_matches_numpy(host):
    rng = np.random.default_rng(11)
    host.b3_host_inv.restype = C.c_int
    for _ in range(50):
        a = rng.normal(size=(3, 3)) + 3.0 * np.eye(3)
        r = np.zeros((3, 3))
        assert host.b3_host_inv(_p(np.ascontiguousarray(a)), _p(r)) == 1
        assert np.max(np.abs(r - np.linalg.inv(a))) <= 1e-13 * np.max(np.abs(np.linalg.inv(a)))
    s = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [0.0, 1.0, 1.0]])  # rank 2
    assert host.b3_host_inv(_p(s), _p(np.zeros((3, 3)))) == 0


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("length", [1, 2, 7, 40])
def test_line_block_thomas_matches_dense_solve(host, fp32, length):
    """The fracture-line block of the row-scaled system (identity diagonal blocks, couplings L_t to
    the previous row and U_t to the next) solved by the block Thomas factorization, against a dense
    solve of the assembled block-tridiagonal matrix."""
    rng = np.random.default_rng(100 + length)
    host.b3_host_line.restype = C.c_int
    L = 0.3 * rng.normal(size=(length, 3, 3)) / 3.0
    U = 0.3 * rng.normal(size=(length, 3, 3)) / 3.0
    r = rng.normal(size=(length, 3))
    M = np.eye(3 * length)
    for t in range(length):
        if t > 0:
            M[3 * t:3 * t + 3, 3 * (t - 1):3 * t] = L[t]
        if t + 1 < length:
            M[3 * t:3 * t + 3, 3 * (t + 1):3 * t + 6] = U[t]
    want = np.linalg.solve(M, r.ravel()).reshape(length, 3)
    z = np.zeros((length, 3))
    ok = host.b3_host_line(length, _p(np.ascontiguousarray(L)), _p(np.ascontiguousarray(U)),
                           _p(np.ascontiguousarray(r)), _p(z), fp32)
    assert ok == 1
    tol = 2e-5 if fp32 else 1e-12
    assert np.max(np.abs(z - want)) <= tol * np.max(np.abs(want))
