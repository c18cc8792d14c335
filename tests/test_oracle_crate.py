"""Pins of the oracle's CRATE angular resource (Appendix A, angular resources; first interaction layer)."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_01491_b300 import synth
from conftest import structure

P0 = oracle.Params()
SHIFTS = P0.shf_a0 + np.arange(8) * (P0.rc_ang - P0.shf_a0) / 8
E_OF_Z = oracle.ELEMENT_OF_Z


def _struct(Z, pos, cell=None):
    n = len(Z)
    c = np.zeros((1, 9)) if cell is None else np.asarray(cell, np.float64).reshape(1, 9)
    return synth.Structures(np.asarray(Z, np.int32), np.asarray(pos, np.float64), np.array([0, n], np.int32), c,
                            np.array([0 if cell is None else 1], np.uint8))


@pytest.mark.parametrize("sw", ["cosine", "polynomial", "exponential"])
def test_torch_switch_matches_the_c_switch(sw):
    import torch
    P = oracle.Params(switch=sw)
    r = np.linspace(0.0, 4.0, 81)
    got = oracle._switch_torch(torch.tensor(r), 3.5, P).numpy()
    want = np.array([oracle.switch(x, 3.5, P)[0] for x in r])
    assert np.abs(got - want).max() < 1e-14


def test_single_triplet_closed_form():
    """One centre (C) with an H on a radial-basis centre and an O at 60 degrees on another: only V[H, 2, :]
    and V[O, 5, :] are non-zero, so D_H = f(r_H) V[H, 2], D_O = f(r_O) V[O, 5] and g_C[n] = cos(60 n) D_H D_O."""
    rH, rO = SHIFTS[2], SHIFTS[5]
    pos = [[0, 0, 0], [rH, 0, 0], [rO * 0.5, rO * math.sqrt(3) / 2, 0]]
    s = _struct([6, 1, 8], pos)
    V = np.zeros((7, 8, 32))
    ch = np.arange(32)
    V[E_OF_Z[1], 2] = 1.0 + ch
    V[E_OF_Z[8], 5] = 2.0 - 0.01 * ch
    g = oracle.crate_angular(s, V)
    fH, fO = oracle.switch(rH, P0.rc_ang, P0)[0], oracle.switch(rO, P0.rc_ang, P0)[0]
    want = np.outer([1.0, 0.5, -0.5, -1.0], fH * (1 + ch) * fO * (2 - 0.01 * ch))
    np.testing.assert_allclose(g[0], want, rtol=1e-12, atol=1e-14)


def _min_image_vectors(s):
    x = np.asarray(s.pos, np.float64)
    d = x[None, :, :] - x[:, None, :]
    if s.pbc[0]:
        L = np.asarray(s.cell[0], np.float64)[[0, 4, 8]]
        d -= L * np.round(d / L)
    return d


@pytest.mark.parametrize("name", ["gas24", "water216"])
def test_unordered_pair_sum_identity(name):
    """With V = 1 every channel of D_ij is f(r) sum_a B_a(r), and Theta_0 = 1: g_i[0, c] is the sum over
    unordered neighbour pairs, ((sum D)^2 - sum D^2) / 2, with the neighbours found by brute force."""
    s = structure(name)
    g = oracle.crate_angular(s, np.ones((7, 8, 32)))
    d = _min_image_vectors(s)
    r = np.linalg.norm(d, axis=-1)
    np.fill_diagonal(r, np.inf)
    D = np.where(r < P0.rc_ang, np.array([[oracle.switch(x, P0.rc_ang, P0)[0] if x < P0.rc_ang else 0.0 for x in row]
                                           for row in r]) * np.exp(-P0.eta_a * (r[..., None] - SHIFTS) ** 2).sum(-1),
                 0.0)
    want = (D.sum(1) ** 2 - (D ** 2).sum(1)) / 2
    for c in (0, 17, 31):
        np.testing.assert_allclose(g[:, 0, c], want, rtol=1e-11, atol=1e-12)


def test_brute_force_triplets_with_angles_from_atan2():
    s = structure("gas24")
    V = np.random.default_rng(3).standard_normal((7, 8, 32))
    g = oracle.crate_angular(s, V)
    x = np.asarray(s.pos, np.float64)
    el = oracle.elements(s.Z)
    want = np.zeros_like(g)
    for i in range(s.n_atoms):
        nb = [j for j in range(s.n_atoms) if j != i and np.linalg.norm(x[j] - x[i]) < P0.rc_ang]
        D = {}
        for j in nb:
            r = float(np.linalg.norm(x[j] - x[i]))
            f = 0.5 * math.cos(math.pi * r / P0.rc_ang) + 0.5
            D[j] = f * sum(math.exp(-P0.eta_a * (r - SHIFTS[a]) ** 2) * V[el[j], a] for a in range(8))
        for a in range(len(nb)):
            for b in range(a + 1, len(nb)):
                u, v = x[nb[a]] - x[i], x[nb[b]] - x[i]
                th = math.atan2(np.linalg.norm(np.cross(u, v)), float(u @ v))
                for n in range(4):
                    want[i, n] += math.cos(n * th) * D[nb[a]] * D[nb[b]]
    np.testing.assert_allclose(g, want, rtol=1e-10, atol=1e-12)


def test_rotation_translation_permutation_invariance():
    s = structure("gas24")
    V = np.random.default_rng(4).standard_normal((7, 8, 32))
    g = oracle.crate_angular(s, V)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]]) @ \
        np.array([[1, 0, 0], [0, math.cos(1.1), -math.sin(1.1)], [0, math.sin(1.1), math.cos(1.1)]])
    perm = np.random.default_rng(5).permutation(s.n_atoms)
    x = (np.asarray(s.pos, np.float64) @ R.T + np.array([3.0, -2.0, 7.5]))[perm]
    g2 = oracle.crate_angular(_struct(s.Z[perm], x), V)
    np.testing.assert_allclose(g2, g[perm], rtol=1e-10, atol=1e-12)


def test_vjp_matches_finite_differences():
    s = structure("gas24")
    rng = np.random.default_rng(6)
    V = rng.standard_normal((7, 8, 32))
    G = rng.standard_normal((s.n_atoms, 4, 32))
    _, gx, gV = oracle.crate_angular(s, V, G=G)
    x0 = np.asarray(s.pos, np.float64)
    L = lambda x, W: float((oracle.crate_angular(_struct(s.Z, x), W) * G).sum())
    h = 1e-5
    for i, a in [(0, 0), (5, 1), (11, 2), (20, 0)]:
        xp, xm = x0.copy(), x0.copy()
        xp[i, a] += h
        xm[i, a] -= h
        fd = (L(xp, V) - L(xm, V)) / (2 * h)
        assert abs(fd - gx[i, a]) <= 1e-6 * max(1.0, abs(gx[i, a]))
    assert np.abs(gx.sum(0)).max() <= 1e-9 * np.abs(gx).max()          # no net force
    for e, a, c in [(0, 3, 7), (1, 6, 30), (3, 0, 1)]:
        Vp, Vm = V.copy(), V.copy()
        Vp[e, a, c] += h
        Vm[e, a, c] -= h
        fd = (L(x0, Vp) - L(x0, Vm)) / (2 * h)
        assert abs(fd - gV[e, a, c]) <= 1e-6 * max(1.0, abs(gV[e, a, c]))


def test_continuity_at_the_triplet_cutoff():
    V = np.random.default_rng(8).standard_normal((7, 8, 32))
    base = [[0, 0, 0], [1.1, 0, 0], [0, 1.3, 0.2]]
    g_in = oracle.crate_angular(_struct([6, 1, 8, 1], base + [[P0.rc_ang - 1e-7, 0.0, 0.0]]), V)[0]
    g_out = oracle.crate_angular(_struct([6, 1, 8, 1], base + [[P0.rc_ang + 1e-7, 0.0, 0.0]]), V)[0]
    assert np.abs(g_in - g_out).max() < 1e-9 * max(1.0, np.abs(g_in).max())
