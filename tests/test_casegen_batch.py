"""Structure of the batched-ensemble generator (host only)."""
import numpy as np

from paper_2008_01539_gb300 import casegen as cg


def test_union_is_disjoint_and_preserves_members():
    members = [cg.small_dfn(24, 20, 6, seed=7, n_steps=3), cg.small_dfn(19, 23, 4, seed=5, n_steps=3)]
    u = cg.batch(members)
    offs = u.meta["offsets"]
    assert u.n == sum(c.n for c in members) and offs == [0, members[0].n, u.n]
    for k, c in enumerate(members):
        lo, hi = offs[k], offs[k + 1]
        rows = u.row_ptr[lo:hi + 1]
        assert np.array_equal(np.diff(rows), np.diff(c.row_ptr))
        nb = u.nbr[rows[0]:rows[-1]]
        assert nb.min() >= lo and nb.max() < hi  # no connection leaves the member
        assert np.array_equal(nb - lo, c.nbr)
        assert np.array_equal(u.trans[rows[0]:rows[-1]], c.trans)
        assert np.array_equal(u.p0[lo:hi], c.p0) and np.array_equal(u.always_active[lo:hi], c.always_active)
    # fracture ids of different members never coincide
    ids = [set(u.line_id[offs[k]:offs[k + 1]][u.line_id[offs[k]:offs[k + 1]] >= 0].tolist()) for k in range(2)]
    assert not (ids[0] & ids[1])
    assert np.array_equal(u.well_cell, np.concatenate([members[0].well_cell, members[1].well_cell + offs[1]]))


def test_realizations_are_seeded_and_uneven():
    a, b = cg.realization(3), cg.realization(3)
    assert a.n == b.n and np.array_equal(a.trans, b.trans)
    sizes = [cg.realization(i).meta["nx"] for i in range(6)]
    assert all(150 <= s <= 500 for s in sizes) and len(set(sizes)) > 1


def test_batch_rejects_mismatched_schedules():
    import pytest

    with pytest.raises(ValueError):
        cg.batch([cg.small_dfn(n_steps=3), cg.small_dfn(n_steps=4)])


def test_3d_generator_structure():
    c = cg.small_dfn3d()
    nx, ny, nz = c.meta["nx"], c.meta["ny"], c.meta["nz"]
    assert c.n_matrix == nx * ny * nz
    rows = np.repeat(np.arange(c.n), np.diff(c.row_ptr))
    # symmetric, no self loops, neighbours ascending within a row
    pairs = set(zip(rows.tolist(), c.nbr.tolist()))
    assert all((j, i) in pairs for i, j in pairs) and all(i != j for i, j in pairs)
    assert all(np.all(np.diff(c.nbr[c.row_ptr[i]:c.row_ptr[i + 1]]) > 0) for i in range(c.n))
    # layers: depth grows with the layer index; the initial pressure follows the oil gradient
    d = c.depth[: c.n_matrix].reshape(nz, ny, nx)
    assert np.all(np.diff(d[:, 0, 0]) > 0)
    assert np.allclose(np.diff(c.p0[: c.n_matrix].reshape(nz, ny, nx)[:, 0, 0]),
                       c.fluid.rho_o_ref * cg.GRAVITY * c.meta["dz"])
    # every fracture cell is always active and belongs to a line; the producer sits in the HF
    assert np.all(c.always_active[c.line_id >= 0] == 1)
    assert c.line_id[c.well_cell[0]] >= 0
