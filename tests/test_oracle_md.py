"""Pins of the oracle's Langevin integrator (BAOAB, section V.D) and of its noise generator.

Philox-4x32-10 against the generator's published known-answer vectors; the Box-Muller normals against
the standard normal distribution; BAOAB without friction against the (separately pinned) velocity
Verlet oracle; and the thermostat's stationary kinetic temperature against the bath temperature
(equipartition) for atoms that feel no force."""
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2405_01491_b300 import synth
from conftest import structure, weights

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) if l.strip()
            and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        got = oracle.philox4x32_10(np.array([v[:4]], np.uint64), v[4:6])[0]
        assert [int(g) for g in got] == v[6:10]


def test_langevin_noise_is_standard_normal_and_independent():
    g = oracle.langevin_noise(200_000, 12345, seed=0x1234_5678_9abc)
    for c in range(3):
        assert abs(g[:, c].mean()) < 0.01 and abs(g[:, c].var() - 1.0) < 0.01
        assert stats.kstest(g[:, c], "norm").pvalue > 1e-4
    cc = np.corrcoef(g.T)
    assert np.abs(cc - np.eye(3)).max() < 0.01
    # another step, another key: uncorrelated streams
    h = oracle.langevin_noise(200_000, 12346, seed=0x1234_5678_9abc)
    k = oracle.langevin_noise(200_000, 12345, seed=0x1234_5678_9abd)
    assert abs(np.corrcoef(g[:, 0], h[:, 0])[0, 1]) < 0.01 and abs(np.corrcoef(g[:, 0], k[:, 0])[0, 1]) < 0.01


def test_baoab_without_friction_is_velocity_verlet():
    s = structure("gas24")
    w = weights(1)
    v0 = synth.maxwell_boltzmann(s.Z, 300.0, seed=3)
    E, K, x, v, F = oracle.langevin_baoab(s, w, v0, 12, 0.5, 300.0, 0.0, seed=9)
    Er, xr, vr, Fr = oracle.velocity_verlet(s, w, v0, 12, 0.5)
    assert np.abs(E - Er).max() < 1e-10 and np.abs(x - xr).max() < 1e-12 and np.abs(v - vr).max() < 1e-12
    # the kinetic history is that of v_k: at the last step, of the returned velocities
    assert np.allclose(K[-1], oracle.kinetic_energies(s, vr), rtol=1e-12)


def _isolated_atoms(n, seed=8):
    """n atoms far apart (each its own gas-phase structure): no neighbours, so no forces."""
    rng = np.random.default_rng(seed)
    Z = rng.choice([1, 6, 8, 16], size=n).astype(np.int32)
    pos = (np.arange(n)[:, None] * np.array([20.0, 0.0, 0.0])).astype(np.float32)
    return synth.Structures(Z, pos, np.arange(n + 1, dtype=np.int32), np.zeros((n, 9), np.float32),
                            np.zeros(n, np.uint8))


def test_baoab_thermostat_reaches_the_bath_temperature():
    s = _isolated_atoms(3000)
    w = weights(1)
    T, n, dt = 300.0, 60, 1.0
    E, K, x, v, F = oracle.langevin_baoab(s, w, np.zeros((s.n_atoms, 3)), n, dt, T, 0.5, seed=77)
    assert np.abs(F).max() == 0.0
    # equipartition: K = 3/2 N kB T on average once the velocities have decorrelated (c1^k ~ e^(-k/2))
    Kt = K[30:].sum(axis=1)
    T_est = 2 * Kt.mean() / (3 * s.n_atoms * oracle.KB_KCAL)
    assert abs(T_est - T) / T < 0.02, T_est
    # every mass equilibrates to the same temperature
    el = oracle.elements(s.Z)
    for e in np.unique(el):
        idx = np.where(el == e)[0]
        T_e = 2 * K[30:, idx].sum(axis=1).mean() / (3 * len(idx) * oracle.KB_KCAL)
        assert abs(T_e - T) / T < 0.06, (e, T_e)
