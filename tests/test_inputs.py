"""Invariants of the seeded input generator shared by the oracle and the GPU path.

The generator holds none of the method's arithmetic; these checks make sure the meshes, orderings,
boundary masks and parameter draws are what the workloads state (orientation, volume, ordering
contract of the subdomain blocks, face bits, Kuhn connectivity, documented sizes and ranges).
"""
import numpy as np
import pytest

import ect_inputs as E


@pytest.mark.parametrize("jitter", [0.0, 0.15])
def test_box_mesh_orientation_and_volume(jitter):
    shape, lengths = (6, 5, 9), (20e-3, 16e-3, 40e-3)
    m = E.box_mesh(shape, lengths, (2, 2, 4), jitter=jitter, seed=3)
    vol = E.tet_volumes(m.xyz, m.tets)
    assert np.all(vol > 0.0)                                   # positively oriented
    assert vol.sum() == pytest.approx(np.prod(lengths), rel=1e-12)
    nx, ny, nz = shape
    assert m.n_nodes == nx * ny * nz and m.n_tets == 6 * (nx - 1) * (ny - 1) * (nz - 1)


def test_subdomain_blocks_are_contiguous_ranges_of_at_most_16_nodes():
    m = E.box_mesh((7, 5, 9), (1.0, 1.0, 1.0), (2, 2, 4))
    b = m.block_of_node
    d = np.diff(b)
    assert b[0] == 0 and np.all((d == 0) | (d == 1))
    sizes = np.bincount(b)
    assert sizes.max() == 16 and sizes.min() >= 1
    # every node id is used by some tet, and each block's nodes span at most a 2 x 2 x 4 box
    assert np.unique(m.tets).size == m.n_nodes
    h = np.array([1.0 / 6, 1.0 / 4, 1.0 / 8])
    for blk in range(sizes.size):
        ext = np.ptp(m.xyz[b == blk], axis=0) / h
        assert np.all(ext <= np.array([1, 1, 3]) + 1e-9), blk


def test_boundary_mask_bits_on_the_faces():
    shape, lengths = (5, 6, 7), (1.0, 2.0, 3.0)
    m = E.box_mesh(shape, lengths, (2, 2, 4))
    x, y, z = m.xyz.T
    onx = np.isclose(np.abs(x), lengths[0] / 2)
    ony = np.isclose(np.abs(y), lengths[1] / 2)
    onz = np.isclose(np.abs(z), lengths[2] / 2)
    want = onx * E.BC_AX + ony * E.BC_AY + onz * E.BC_AZ
    assert np.array_equal(m.bc_mask.astype(int), want.astype(int))


def test_kuhn_connectivity_interior_nodes_have_14_neighbours():
    m = E.box_mesh((5, 5, 5), (1.0, 1.0, 1.0), (1, 1, 1))
    nb = [set() for _ in range(m.n_nodes)]
    for t in m.tets:
        for a in t:
            nb[a].update(int(v) for v in t if v != a)
    x, y, z = m.xyz.T
    interior = (np.abs(x) < 0.49) & (np.abs(y) < 0.49) & (np.abs(z) < 0.49)
    assert interior.sum() == 27
    assert all(len(nb[i]) == 14 for i in np.nonzero(interior)[0])


def test_documented_config_sizes():
    shape, lengths, jitter = E.CONFIGS["c1"]
    assert shape == (16, 16, 32) and jitter == 0.0
    assert np.prod(shape) == 8192 and 6 * 15 * 15 * 31 == 41850
    for name, nodes in (("c2", 1_000_004), ("c3", 500_094), ("c4", 4_000_752), ("c5", 250_000)):
        assert np.prod(E.CONFIGS[name][0]) == nodes


def test_deposit_parameters_within_stated_ranges_and_seeded():
    P = np.array([E.deposit_params(s) for s in range(200)])
    lo = np.array([0.0, 2e-3, 1e4, 1.0, 0.0, -10e-3])
    hi = np.array([0.5e-3, 20e-3, 1e6, 5.0, 2 * np.pi, 10e-3])
    assert np.all(P >= lo) and np.all(P <= hi)
    assert np.array_equal(E.deposit_params(7), E.deposit_params(7))
    assert not np.array_equal(E.deposit_params(7), E.deposit_params(8))
