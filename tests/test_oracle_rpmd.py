"""Pins of the oracle's ring-polymer molecular dynamics (section V.D, NQE methods)."""
import numpy as np
import pytest

import oracle
from paper_2405_01491_b300 import synth
from conftest import structure, weights


@pytest.mark.parametrize("P", [1, 2, 5, 8, 32])
def test_normal_modes_diagonalise_the_ring_springs(P):
    """C is orthogonal and turns the ring's spring matrix (2 on the diagonal, -1 to each cyclic neighbour)
    into the diagonal of its eigenvalues, which a library eigensolver confirms are (2 sin(k pi / P))^2."""
    C, wk = oracle.rpmd_normal_modes(P)
    assert np.abs(C.T @ C - np.eye(P)).max() < 1e-13
    K = 2 * np.eye(P) - np.roll(np.eye(P), 1, 0) - np.roll(np.eye(P), -1, 0) if P > 2 else \
        (np.zeros((1, 1)) if P == 1 else np.array([[2.0, -2.0], [-2.0, 2.0]]))
    D = C.T @ K @ C
    assert np.abs(D - np.diag(np.diag(D))).max() < 1e-12
    np.testing.assert_allclose(np.sort(np.diag(D)), np.sort(np.linalg.eigvalsh(K)), atol=1e-12)
    np.testing.assert_allclose(np.diag(D), wk ** 2, atol=1e-12)


def test_one_bead_is_velocity_verlet():
    s = structure("gas24")
    w = weights(1)
    v0 = synth.maxwell_boltzmann(s.Z, 300.0, seed=3)
    E, H, x, v, F = oracle.rpmd(s, w, 1, s.pos[None], v0[None], 10, 0.5, 300.0)
    Er, xr, vr, Fr = oracle.velocity_verlet(s, w, v0, 10, 0.5)
    assert np.abs(E[:, 0] - Er[:, 0]).max() < 1e-10 and np.abs(x[0] - xr).max() < 1e-12


def _free_atoms(n):
    Z = np.array([1, 8] * (n // 2), np.int32)
    pos = (np.arange(n)[:, None] * np.array([20.0, 0.0, 0.0])).astype(np.float32)
    return synth.Structures(Z, pos, np.array([0, n], np.int32), np.zeros((1, 9), np.float32), np.zeros(1, np.uint8))


def test_free_ring_polymer_conserves_its_hamiltonian_exactly():
    """Atoms too far apart to interact: the beads feel only their springs, which the normal-mode step integrates
    exactly, so the ring-polymer Hamiltonian is constant for any dt and the centroid moves at constant velocity."""
    s = _free_atoms(6)
    P = 16
    rng = np.random.default_rng(2)
    x0 = np.asarray(s.pos, np.float64)[None] + 0.05 * rng.standard_normal((P, s.n_atoms, 3))
    v0 = 0.01 * rng.standard_normal((P, s.n_atoms, 3))
    E, H, x, v, F = oracle.rpmd(s, weights(1), P, x0, v0, 40, 2.0, 300.0)
    assert np.abs(F).max() == 0.0
    assert np.abs(H - H[0]).max() < 1e-10 * abs(H[0])
    cen0, cen = x0.mean(0), x.mean(0)
    np.testing.assert_allclose(cen, cen0 + 39 * 2.0 * v0.mean(0), atol=1e-10)


def test_hamiltonian_error_scales_as_dt_squared():
    s = structure("gas24")
    P = 4
    rng = np.random.default_rng(3)
    x0 = np.asarray(s.pos, np.float64)[None] + 0.02 * rng.standard_normal((P, s.n_atoms, 3))
    v0 = np.repeat(synth.maxwell_boltzmann(s.Z, 300.0, seed=4)[None], P, 0)
    errs = []
    for dt in (0.2, 0.1):
        n = int(round(4.0 / dt))
        E, H, *_ = oracle.rpmd(s, weights(1), P, x0, v0, n + 1, dt, 300.0)
        errs.append(np.abs(H - H[0]).max())
    assert 2.5 < errs[0] / errs[1] < 6.0


def test_cyclic_relabelling_of_beads():
    s = structure("gas24")
    P = 4
    rng = np.random.default_rng(5)
    x0 = np.asarray(s.pos, np.float64)[None] + 0.02 * rng.standard_normal((P, s.n_atoms, 3))
    v0 = 0.005 * rng.standard_normal((P, s.n_atoms, 3))
    E, H, x, v, F = oracle.rpmd(s, weights(1), P, x0, v0, 6, 0.5, 300.0)
    E2, H2, x2, v2, F2 = oracle.rpmd(s, weights(1), P, np.roll(x0, 1, 0), np.roll(v0, 1, 0), 6, 0.5, 300.0)
    np.testing.assert_allclose(x2, np.roll(x, 1, 0), atol=1e-10)
    np.testing.assert_allclose(H2, H, rtol=1e-12)
