"""Pins of the oracle's neighbour graph (paper section II.A) against things other than itself:
an explicit image-enumeration brute force, scipy's periodic k-d tree, and the graph's
stated invariants (directed, same batch index only, minimum image, cell check)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2405_01491_b300 import synth
from conftest import structure


def _edge_set(ei, ej, es):
    return set(zip(ei.tolist(), ej.tolist(), map(tuple, es.tolist())))


def _brute_images(s, R):
    """Every ordered pair and every periodic image in -2..2 per axis, kept when closer than R."""
    out = set()
    pos = s.pos.astype(np.float64)
    for m in range(s.n_mol):
        a0, a1 = int(s.mol_offsets[m]), int(s.mol_offsets[m + 1])
        L = np.diag(s.cell[m].reshape(3, 3)).astype(np.float64)
        imgs = np.array(list(itertools.product(range(-2, 3), repeat=3)) if s.pbc[m] else [(0, 0, 0)])
        x = pos[a0:a1]
        for i in range(a1 - a0):
            d = x[None, :, :] - x[i][None, None, :] + (imgs * L)[:, None, :]   # [img, j, 3]
            d2 = np.einsum("ijk,ijk->ij", d, d)
            for n_idx, j in zip(*np.nonzero(d2 < R * R)):
                if j != i:
                    out.add((a0 + i, a0 + int(j), tuple(int(v) for v in imgs[n_idx])))
    return out


@pytest.mark.parametrize("name,R", [("gas24", 5.1), ("gas24", 3.5), ("box300", 5.1), ("box300", 6.1)])
def test_matches_image_enumeration(name, R):
    s = structure(name)
    got = _edge_set(*oracle.neighbors(s, R))
    assert got == _brute_images(s, R)


@pytest.mark.parametrize("name,R", [("box1500", 5.1), ("water216", 6.1), ("batch64", 5.1)])
def test_matches_scipy_kdtree(name, R):
    from scipy.spatial import cKDTree
    s = structure(name)
    ei, ej, es = oracle.neighbors(s, R)
    got = set(zip(ei.tolist(), ej.tolist()))
    want = set()
    for m in range(s.n_mol):
        a0 = int(s.mol_offsets[m])
        x = s.pos[a0:s.mol_offsets[m + 1]].astype(np.float64)
        if s.pbc[m]:
            L = float(s.cell[m, 0])
            tree = cKDTree(np.mod(x, L), boxsize=L)
        else:
            tree = cKDTree(x)
        for a, b in tree.query_pairs(R):
            want.add((a0 + a, a0 + b))
            want.add((a0 + b, a0 + a))
    assert got == want


def test_directed_and_batch_local():
    s = structure("batch64")
    ei, ej, es = oracle.neighbors(s, 5.1)
    E = _edge_set(ei, ej, es)
    for i, j, n in E:
        assert (j, i, tuple(-x for x in n)) in E
    mol = np.repeat(np.arange(s.n_mol), np.diff(s.mol_offsets))
    assert np.all(mol[ei] == mol[ej])
    assert np.all(ei != ej)
    # sorted by (i, j)
    key = ei.astype(np.int64) * s.n_atoms + ej
    assert np.all(np.diff(key) > 0)


def test_minimum_image_shift_is_nearest_image():
    s = structure("box300")
    L = float(s.cell[0, 0])
    # move some atoms by whole lattice vectors: the graph keeps the same pairs, shifts absorb the move
    s2 = synth.Structures(s.Z, s.pos.copy(), s.mol_offsets, s.cell, s.pbc)
    s2.pos[::7, 0] += np.float32(L)
    s2.pos[::5, 2] -= np.float32(2 * L)
    ei, ej, es = oracle.neighbors(s, 5.1)
    ei2, ej2, es2 = oracle.neighbors(s2, 5.1)
    assert np.array_equal(ei, ei2) and np.array_equal(ej, ej2)
    moved = np.zeros((s.n_atoms, 3), np.int64)
    moved[::7, 0] += 1
    moved[::5, 2] -= 2
    assert np.array_equal(es2.astype(np.int64), es.astype(np.int64) + moved[ei2] - moved[ej2])


def test_cell_too_small_is_rejected():
    s = structure("box300")
    L = float(s.cell[0, 0])
    with pytest.raises(oracle.OracleError):
        oracle.neighbors(s, L / 2)          # L <= 2R
    s2 = synth.Structures(s.Z, s.pos, s.mol_offsets, s.cell.copy(), s.pbc)
    s2.cell[0, 1] = 0.5                      # not orthorhombic
    with pytest.raises(oracle.OracleError):
        oracle.neighbors(s2, 5.1)


def test_empty_and_single_atom():
    s = synth.Structures(np.zeros(0, np.int32), np.zeros((0, 3), np.float32), np.array([0], np.int32),
                         np.zeros((0, 9), np.float32), np.zeros(0, np.uint8))
    ei, ej, es = oracle.neighbors(s, 5.1)
    assert ei.size == 0
    s1 = synth.Structures(np.array([6], np.int32), np.zeros((1, 3), np.float32), np.array([0, 1], np.int32),
                          np.zeros((1, 9), np.float32), np.zeros(1, np.uint8))
    assert oracle.neighbors(s1, 5.1)[0].size == 0
