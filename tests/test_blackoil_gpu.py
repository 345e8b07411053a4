"""The black-oil kernels through the C ABI (lns_bo_assemble, lns_bo_update) against the black-oil
oracle (oracle/blackoil.py): residual, 3x3 Jacobian blocks and CNV of every cell within 1e-11 of
each component's scale (the device contracts multiply-adds the host does not), the update with
the primary-variable switch (Section 3.1, black-oil form) bit for bit.  Models of 283 and 3,059
cells (2 and 24 blocks of 128 threads, ragged tails); mixed states, cells at the Corey clamps, and
the state the oracle reaches after gas appears."""
import numpy as np
import pytest

import oracle as O
from oracle import blackoil as B
from paper_2008_01539_gb300 import casegen as cg
from paper_2008_01539_gb300 import lns

pytestmark = pytest.mark.gpu
PSI = cg.PSI


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    lns.load(build_if_missing=True)
    O.build()


def _dev(a, dtype=None):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype)), device="cuda")


def _graph(bo):
    c = bo.case
    t = dict(row_ptr=_dev(c.row_ptr, np.int32), nbr=_dev(c.nbr, np.int32), trans=_dev(c.trans, np.float64),
             pv_ref=_dev(c.pv_ref, np.float64), depth=_dev(c.depth, np.float64),
             well_cell=_dev(c.well_cell, np.int32), well_wi=_dev(c.well_wi, np.float64),
             well_bhp=_dev(c.well_bhp, np.float64))
    g = {k: v.data_ptr() if v.numel() else 0 for k, v in t.items()}
    g["n_wells"] = int(c.well_cell.shape[0])
    return g, t


def _state(st):
    t = dict(p=_dev(st.p, np.float64), sw=_dev(st.sw, np.float64), sg=_dev(st.sg, np.float64),
             rs=_dev(st.rs, np.float64), sat=_dev(st.sat, np.uint8))
    return {k: v.data_ptr() for k, v in t.items()}, t


def _assemble_gpu(bo, st, old, dt):
    import torch

    n, na = bo.n, bo.case.nbr.shape[0]
    g, keep_g = _graph(bo)
    s, keep_s = _state(st)
    o, keep_o = _state(old)
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    Jd = torch.zeros((n, 3, 3), dtype=torch.float64, device="cuda")
    Jo = torch.zeros((na, 3, 3), dtype=torch.float64, device="cuda")
    cv = torch.zeros(n, dtype=torch.float64, device="cuda")
    lns.lns_bo_assemble(lns.bo_fluid(bo.fluid), n, g, s, o, dt, F.data_ptr(), Jd.data_ptr(), Jo.data_ptr(),
                        cv.data_ptr())
    return F.cpu().numpy(), Jd.cpu().numpy(), Jo.cpu().numpy(), cv.cpu().numpy()


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
        sw[k[: len(k) // 2]] = rng.uniform(0.1, 0.2, len(k) // 2)  # water below connate
        kk = k[len(k) // 2:]
        sat[kk] = 1
        sg[kk] = 0.85 - sw[kk]  # So = 0.15 < sor
        rs[kk] = rs_s[kk]
    return B.State(p, sw, sg, rs, sat)


def _compare(got, bo, st, old, dt):
    F, Jd, Jo, cv = got
    Fr, Jdr, Jor = B.assemble(bo, st, old, dt)
    cvr = B.cnv(bo, st, Fr, dt)
    for r in range(3):
        assert np.max(np.abs(F[:, r] - Fr[:, r])) <= 1e-11 * np.max(np.abs(Fr[:, r])), ("F", r)
        for k in range(3):
            for J, Jr, name in ((Jd, Jdr, "Jd"), (Jo, Jor, "Jo")):
                s = np.max(np.abs(Jr[:, r, k]))
                assert np.max(np.abs(J[:, r, k] - Jr[:, r, k])) <= 1e-11 * s + 1e-300, (name, r, k)
    assert np.max(np.abs(cv - cvr)) <= 1e-11 * np.max(cvr)


MODELS = {"283 cells": lambda: cg.small_blackoil3d(),
          "3059 cells": lambda: cg.blackoil(cg.small_dfn3d(24, 20, 6), p_init=3800.0 * PSI, bhp=2000.0 * PSI)}


@pytest.mark.parametrize("model", list(MODELS))
@pytest.mark.parametrize("clamps", [False, True])
def test_bo_assemble_matches_oracle(model, clamps):
    bo = MODELS[model]()
    st, old = _mixed(bo, 1, clamps), _mixed(bo, 2, clamps)
    dt = 2.0 * cg.DAY
    _compare(_assemble_gpu(bo, st, old, dt), bo, st, old, dt)


def test_bo_assemble_matches_oracle_after_gas_appears():
    bo = cg.small_blackoil3d()
    old = B.initial_state(bo)
    dt = float(bo.case.dt_schedule[0])
    st = old.copy()
    for _ in range(2):
        du, _, _ = B.local_solve(bo, st, old, dt, np.ones(bo.n, np.uint8))
        st, _ = B.apply_update(bo.fluid, st, du, np.ones(bo.n, np.uint8))
    assert 0 < st.sat.sum() < bo.n
    _compare(_assemble_gpu(bo, st, old, dt), bo, st, old, dt)


@pytest.mark.parametrize("chop", [0.0, 0.2])
@pytest.mark.parametrize("masked", [False, True])
def test_bo_update_matches_oracle_bit_for_bit(chop, masked):
    import torch

    bo = MODELS["3059 cells"]()
    fl, n = bo.fluid, bo.n
    rng = np.random.default_rng(3)
    st = _mixed(bo, 4)
    du = np.stack([rng.normal(0.0, 300.0 * PSI, n), rng.normal(0.0, 0.15, n),
                   np.where(st.sat == 1, rng.normal(0.0, 0.15, n), rng.normal(0.0, 0.5, n) * fl.rs_max)], axis=1)
    va = (rng.random(n) < 0.6).astype(np.uint8) if masked else np.ones(n, np.uint8)
    ref_du = du.copy()
    if chop > 0.0:  # the oracle chops in its Newton step: |dSw|, and |dSg| where free gas is present
        ref_du[:, 1] = np.clip(ref_du[:, 1], -chop, chop)
        s = st.sat == 1
        ref_du[s, 2] = np.clip(ref_du[s, 2], -chop, chop)
    ref, ref_sw = B.apply_update(fl, st, ref_du, va)
    s_d, keep = _state(st)
    du_d = _dev(du, np.float64)
    bits = _dev(lns.mask_to_bits(va).view(np.int32)) if masked else None  # the bitset's words, as int32
    sw_d = torch.zeros(n, dtype=torch.uint8, device="cuda")
    lns.lns_bo_update(lns.bo_fluid(fl), n, chop, du_d.data_ptr(), s_d, bits.data_ptr() if masked else 0,
                      sw_d.data_ptr())
    assert ref_sw.sum() > 0
    assert np.array_equal(sw_d.cpu().numpy().astype(bool), ref_sw)
    for k, a in (("p", ref.p), ("sw", ref.sw), ("sg", ref.sg), ("rs", ref.rs), ("sat", ref.sat)):
        assert np.array_equal(keep[k].cpu().numpy(), a), k


def test_bo_assemble_full_size_3d_sampled():
    """The 3D workload's geometry with its black-oil physics (1,064,029 cells, 6.2M CSR entries; 8,313
    blocks): the whole model assembled on the device, 20,000 random rows plus the producers' rows
    recomputed by the oracle one by one (its full assembly takes minutes) and compared as above."""
    import torch

    bo = cg.config2_blackoil()
    st, old = _mixed(bo, 5), _mixed(bo, 6)
    dt = 5.0 * cg.DAY
    F, Jd, Jo, cv = _assemble_gpu(bo, st, old, dt)
    rng = np.random.default_rng(7)
    cells = np.unique(np.concatenate([rng.choice(bo.n, 20000, replace=False),
                                      bo.case.well_cell.astype(np.int64)]))
    Fr, Jdr, Jor, e = B.assemble_cells(bo, st, old, dt, cells)
    cvr = B.cnv(bo, st, Fr, dt, cells)
    F, Jd, Jo, cv = F[cells], Jd[cells], Jo[e], cv[cells]
    for r in range(3):
        assert np.max(np.abs(F[:, r] - Fr[:, r])) <= 1e-11 * np.max(np.abs(Fr[:, r])), ("F", r)
        for k in range(3):
            for J, Jr, name in ((Jd, Jdr, "Jd"), (Jo, Jor, "Jo")):
                sc = np.max(np.abs(Jr[:, r, k]))
                assert np.max(np.abs(J[:, r, k] - Jr[:, r, k])) <= 1e-11 * sc + 1e-300, (name, r, k)
    assert np.max(np.abs(cv - cvr)) <= 1e-11 * np.max(cvr)
    torch.cuda.synchronize()

