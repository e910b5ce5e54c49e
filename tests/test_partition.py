"""Host logic of the partitioner (ect_partition: recursive coordinate
bisection into contiguous subdomains), called through the C ABI on the CPU;
it does no GPU work.  Also the TetGen reader/writer of the input module."""
import numpy as np
import pytest

import ect_inputs as E


@pytest.fixture(scope="module")
def ect():
    from paper_1602_03207_gb300 import build, ect as ect_mod
    build.build()
    ect_mod.load_library()
    return ect_mod


@pytest.mark.parametrize("s", [1, 5, 8, 16])
def test_partition_is_a_valid_contiguous_blocking(ect, s):
    m = E.unstructured_box_mesh((9, 8, 13), (20e-3, 20e-3, 40e-3), seed=2)
    new_id, blk = ect.partition(m.xyz, s)
    n = m.n_nodes
    assert np.array_equal(np.sort(new_id), np.arange(n))                 # a permutation
    assert blk[0] == 0 and np.all(np.diff(blk) >= 0) and np.all(np.diff(blk) <= 1)
    sizes = np.bincount(blk)
    assert sizes.max() <= s and sizes.min() >= 1
    assert sizes.size == -(-n // s) or s == 1 or sizes.size <= 2 * (-(-n // s))
    # blocks are compact: each block's extent is at most a few mesh steps per axis
    xyz = np.empty_like(m.xyz)
    xyz[new_id] = m.xyz
    h = np.array(m.lengths) / (np.array(m.shape) - 1)
    for b in range(0, sizes.size, 7):
        pts = xyz[blk == b]
        ext = (pts.max(axis=0) - pts.min(axis=0)) / h
        assert ext.max() <= 2.0 * s + 2.0
    # deterministic
    new2, blk2 = ect.partition(m.xyz, s)
    assert np.array_equal(new_id, new2) and np.array_equal(blk, blk2)


def test_partition_of_exact_multiple_gives_equal_blocks(ect):
    m = E.box_mesh((8, 8, 8), (1.0, 1.0, 1.0), (1, 1, 1))
    new_id, blk = ect.partition(m.xyz, 16)
    sizes = np.bincount(blk)
    assert sizes.size == 32 and np.all(sizes == 16)
    # on a regular grid the bisection of a cube of 512 nodes yields 2x2x4 or 4x2x2 boxes
    xyz = np.empty_like(m.xyz)
    xyz[new_id] = m.xyz
    for b in range(32):
        pts = xyz[blk == b]
        ext = np.round((pts.max(axis=0) - pts.min(axis=0)) * 7).astype(int) + 1
        assert sorted(ext.tolist()) == [2, 2, 4]


def test_partition_rejects_bad_arguments(ect):
    xyz = np.zeros((10, 3))
    with pytest.raises(ect.EctError):
        ect.partition(xyz, 17)
    with pytest.raises(ect.EctError):
        ect.partition(xyz, 0)
    bad = xyz.copy()
    bad[3, 1] = np.nan
    with pytest.raises(ect.EctError):
        ect.partition(bad, 8)


def test_permuted_mesh_is_the_same_mesh():
    m = E.unstructured_box_mesh((6, 7, 8), (1.0, 1.0, 1.0), seed=1)
    rng = np.random.default_rng(0)
    new_id = rng.permutation(m.n_nodes)
    pm = E.permute_mesh(m, new_id, np.zeros(m.n_nodes, dtype=np.int32))
    np.testing.assert_array_equal(pm.xyz[pm.tets], m.xyz[m.tets])
    np.testing.assert_array_equal(pm.bc_mask[new_id], m.bc_mask)
    np.testing.assert_allclose(E.tet_volumes(pm.xyz, pm.tets), E.tet_volumes(m.xyz, m.tets))


def test_unstructured_mesh_fills_the_box_and_is_not_kuhn():
    m = E.unstructured_box_mesh((7, 6, 9), (2.0, 1.0, 3.0), seed=5)
    vol = E.tet_volumes(m.xyz, m.tets)
    assert vol.min() > 0 and abs(vol.sum() - 6.0) < 1e-12
    # box faces stay planar (A.n = 0 needs them) and the face masks match the coordinates
    for a, bit in enumerate((E.BC_AX, E.BC_AY, E.BC_AZ)):
        on = (m.bc_mask & bit) != 0
        assert np.allclose(np.abs(m.xyz[on, a]), 0.5 * m.lengths[a], rtol=0, atol=1e-15)
        assert np.all(np.abs(np.abs(m.xyz[~on, a]) - 0.5 * m.lengths[a]) > 1e-9)
    # every cell's 12 tets share its centre node; node valences vary (a Kuhn mesh has
    # 15-node stencils everywhere inside)
    G = np.zeros(m.n_nodes, dtype=int)
    pairs = {(min(a, b), max(a, b)) for t in m.tets for a in t for b in t if a != b}
    for a, b in pairs:
        G[a] += 1
        G[b] += 1
    assert len(set(G.tolist())) > 5
    # conforming: every interior triangle is shared by exactly two tets
    from collections import Counter
    faces = Counter(tuple(sorted((int(t[a]), int(t[b]), int(t[c])))) for t in m.tets
                    for a, b, c in ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)))
    assert max(faces.values()) == 2
    on_box = lambda f: any(np.all(np.isclose(np.abs(m.xyz[list(f), a]), 0.5 * m.lengths[a])) for a in range(3))  # noqa
    assert all(on_box(f) for f, n in faces.items() if n == 1)


def test_tetgen_round_trip_and_one_based_files(tmp_path):
    m = E.unstructured_box_mesh((5, 5, 6), (1.0, 1.0, 1.0), seed=3)
    region = np.arange(m.n_tets) % 3
    E.write_tetgen(str(tmp_path / "m"), m, region)
    xyz, tets, bc, reg = E.read_tetgen(str(tmp_path / "m"))
    assert np.array_equal(xyz, m.xyz) and np.array_equal(tets, m.tets)
    assert np.array_equal(bc, m.bc_mask) and np.array_equal(reg, region)
    # a hand-written 1-based file with comments and no boundary markers
    (tmp_path / "u.node").write_text("# unit tet\n4 3 0 0\n1 0 0 0\n2 1 0 0\n3 0 1 0\n4 0 0 1\n")
    (tmp_path / "u.ele").write_text("1 4 0\n1 1 2 3 4  # one tet\n")
    xyz, tets, bc, reg = E.read_tetgen(str(tmp_path / "u"))
    assert tets.tolist() == [[0, 1, 2, 3]] and bc is None and reg is None
    assert abs(E.tet_volumes(xyz, tets)[0] - 1.0 / 6.0) < 1e-15
