"""Pins of the oracle's AEV and its derivatives (paper sections II.A, II.B, II.E, Appendix A).

Special-value pins choose the symmetry-function constants so that the expected
numbers are exact constants (a Gaussian at its centre is 1, the cosine switch
at half the cutoff is 1/2, a Gaussian one step away is 1/2 by the choice of
eta); counting pins switch the Gaussians and angular powers off so each slot
counts neighbours or neighbour pairs, checked by brute-force enumeration;
derivative pins use central finite differences; the rest are invariances.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2405_01491_b300 import synth
from conftest import structure, weights

ELEM = {1: 0, 6: 1, 7: 2, 8: 3, 9: 4, 16: 5, 17: 6}


def gas(Z, pos):
    Z = np.asarray(Z, np.int32)
    return synth.Structures(Z, np.asarray(pos, np.float64), np.array([0, len(Z)], np.int32),
                            np.zeros((1, 9)), np.zeros(1, np.uint8))


def rot(seed):
    q = np.random.default_rng(seed).normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def angular_slot(a, b, m, s):
    a, b = min(a, b), max(a, b)
    # upper-triangle pair index written out as an explicit enumeration (independent of the oracle's formula)
    pairs = [(x, y) for x in range(7) for y in range(x, 7)]
    return 112 + pairs.index((a, b)) * 32 + m * 4 + s


def test_radial_special_values():
    # shifts R_k = 0.3 k, cutoff 4.8: at r = 2.4 = R_8 the Gaussian is 1 and the switch is 1/2;
    # eta = ln2 / 0.09 makes the Gaussians one shift away exactly 1/2, two away 1/16.
    P = Params(rc_rad=4.8, shf_r0=0.0, eta_r=math.log(2) / 0.09)
    u = rot(1) @ np.array([1.0, 0, 0])
    s = gas([1, 6], [[0.3, -0.2, 0.1], np.array([0.3, -0.2, 0.1]) + 2.4 * u])
    A = oracle.aev(s, P)
    want_H = np.zeros(1008)   # H sees one C: element block 1
    for k, v in {8: 0.125, 7: 0.0625, 9: 0.0625, 6: 0.125 / 16, 10: 0.125 / 16}.items():
        want_H[16 + k] = v
    got = A[0].copy()
    for k in range(16):
        if k not in (6, 7, 8, 9, 10):
            want_H[16 + k] = got[16 + k]  # far shifts: tiny, checked for sign/size below
    np.testing.assert_allclose(got[:112], want_H[:112], rtol=1e-12, atol=1e-15)
    assert np.all(got[16:32] > 0) and np.all(got[:16] == 0) and np.all(got[32:112] == 0)
    assert np.all(got[112:] == 0)           # two atoms: no angle
    np.testing.assert_allclose(A[1][[8, 7, 9]], [0.125, 0.0625, 0.0625], rtol=1e-12)
    assert np.all(A[1][16:] == 0)


def test_angular_special_values():
    # angular shifts a_m = 0.4 m, cutoff 3.2; both neighbours at r = 1.6 = a_4 = rc/2 (switch 1/2 each);
    # 0.95 cos(theta) = cos(pi/8) puts theta' on the first section centre, so that section's power is 1.
    zeta = 14.1
    P = Params(rc_ang=3.2, shf_a0=0.0, eta_a=math.log(2) / 0.16, zeta=zeta)
    c = math.cos(math.pi / 8) / 0.95
    R = rot(7)
    o = np.array([1.0, 2.0, -0.5])
    pos = [o, o + R @ np.array([1.6, 0, 0]), o + R @ np.array([1.6 * c, 1.6 * math.sqrt(1 - c * c), 0])]
    s = gas([8, 1, 7], pos)
    A = oracle.aev(s, P)[0]
    sq = math.sqrt(2) / 2
    sec = [1.0, ((1 + sq) / 2) ** zeta, 0.5 ** zeta, ((1 - sq) / 2) ** zeta]
    gau = {4: 1.0, 3: 0.5, 5: 0.5, 2: 1 / 16, 6: 1 / 16}
    for m, gm in gau.items():
        for sidx in range(4):
            want = 2 * sec[sidx] * gm * 0.25
            assert A[angular_slot(0, 2, m, sidx)] == pytest.approx(want, rel=1e-12, abs=1e-300)
    others = np.ones(1008, bool)
    others[:112] = False
    others[angular_slot(0, 2, 0, 0):angular_slot(0, 2, 0, 0) + 32] = False
    assert np.all(A[others] == 0)


@pytest.mark.parametrize("seed", [0, 1])
def test_counting_pins_bruteforce(seed):
    # Huge cutoffs make the switch 1 to 1e-11; eta = 0 and zeta = 0 make every Gaussian and power 1.
    # Then radial slot (e, k) = 1/4 * #neighbours of element e and angular slot (p, m, s) =
    # 2 * #unordered neighbour pairs of element pair p: brute-force counts.
    P = Params(rc_rad=1e6, rc_ang=1e6, eta_r=0.0, eta_a=0.0, zeta=0.0)
    rng = np.random.default_rng(seed)
    Z = rng.choice(list(ELEM), size=17)
    s = gas(Z, rng.uniform(0, 8, size=(17, 3)))
    A = oracle.aev(s, P)
    el = [ELEM[int(z)] for z in Z]
    for i in range(17):
        nb = [j for j in range(17) if j != i]
        rad = np.zeros(112)
        for j in nb:
            rad[el[j] * 16:(el[j] + 1) * 16] += 0.25
        ang = np.zeros(1008)
        for j, k in itertools.combinations(nb, 2):
            base = angular_slot(el[j], el[k], 0, 0)
            ang[base:base + 32] += 2.0
        np.testing.assert_allclose(A[i, :112], rad, rtol=1e-9)
        np.testing.assert_allclose(A[i, 112:], ang[112:], rtol=1e-9)


def test_cutoff_membership_counts():
    # Finite cutoffs with the Gaussians and powers switched off: a pair contributes iff r < rc.
    P = Params(rc_rad=4.0, rc_ang=3.0, eta_r=0.0, eta_a=0.0, zeta=0.0)
    s = structure("gas24")
    A = oracle.aev(s, P)
    x = s.pos.astype(np.float64)
    el = [ELEM[int(z)] for z in s.Z]
    fc = lambda r, rc: 0.5 * math.cos(math.pi * r / rc) + 0.5   # pinned by test_radial_special_values
    for i in range(s.n_atoms):
        rad = np.zeros(112)
        ang = np.zeros(1008)
        near = []
        for j in range(s.n_atoms):
            r = float(np.linalg.norm(x[j] - x[i]))
            if j != i and r < 4.0:
                rad[el[j] * 16:(el[j] + 1) * 16] += 0.25 * fc(r, 4.0)
            if j != i and r < 3.0:
                near.append((j, r))
        for (j, rj), (k, rk) in itertools.combinations(near, 2):
            b = angular_slot(el[j], el[k], 0, 0)
            ang[b:b + 32] += 2 * fc(rj, 3.0) * fc(rk, 3.0)
        np.testing.assert_allclose(A[i, :112], rad, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(A[i, 112:], ang[112:], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("name", ["gas24", "box300"])
def test_invariances(name):
    s = structure(name)
    A = oracle.aev(s)
    x = s.pos.astype(np.float64)
    if not s.pbc[0]:
        y = (x - x.mean(0)) @ rot(3).T + np.array([4.0, -7.0, 1.5])
        np.testing.assert_allclose(oracle.aev(gas(s.Z, y)), A, rtol=1e-10, atol=1e-12)
    else:
        L = float(s.cell[0, 0])
        y = x + np.array([1.7, -3.1, 0.4])                      # rigid translation
        y[::3] += L * np.array([1, 0, -1])                       # lattice translations
        s2 = synth.Structures(s.Z, y, s.mol_offsets, s.cell, s.pbc)
        np.testing.assert_allclose(oracle.aev(s2), A, rtol=1e-10, atol=1e-12)
    # permutation of atoms: rows permute
    perm = np.random.default_rng(5).permutation(s.n_atoms)
    s3 = synth.Structures(s.Z[perm], x[perm], s.mol_offsets, s.cell, s.pbc)
    np.testing.assert_allclose(oracle.aev(s3), A[perm], rtol=1e-10, atol=1e-12)


def test_supercell_extensivity():
    s = structure("box300")
    L = float(s.cell[0, 0])
    x = s.pos.astype(np.float64)
    reps = [x + L * np.array(n) for n in itertools.product(range(2), repeat=3)]
    big = synth.Structures(np.tile(s.Z, 8), np.concatenate(reps), np.array([0, 8 * s.n_atoms], np.int32),
                           (s.cell * 2).astype(np.float64), s.pbc)
    A = oracle.aev(s)
    B = oracle.aev(big)
    for r in range(8):
        np.testing.assert_allclose(B[r * s.n_atoms:(r + 1) * s.n_atoms], A, rtol=1e-10, atol=1e-12)


def test_continuity_at_cutoffs():
    for rc, key in ((5.1, "rad"), (3.5, "ang")):
        vals = []
        for dr in (-1e-4, -1e-6, 1e-6):
            r = rc + dr
            if key == "rad":
                s = gas([6, 6], [[0, 0, 0], [r, 0, 0]])
                vals.append(np.abs(oracle.aev(s)[0]).max())
            else:
                s = gas([8, 1, 1], [[0, 0, 0], [r, 0, 0], [0, 1.0, 0]])
                vals.append(np.abs(oracle.aev(s)[0, 112:] - oracle.aev(gas([8, 1], [[0, 0, 0], [0, 1.0, 0]]))[0, 112:]).max())
        # the switch and its slope vanish at rc: contributions fall like dr^2
        assert vals[2] == 0.0
        assert vals[1] < 1e-10
        assert vals[0] < 1e-6


def _fd_aev(s, V, h=1e-6):
    x = s.pos.astype(np.float64)
    sp = synth.Structures(s.Z, x + h * V, s.mol_offsets, s.cell, s.pbc)
    sm = synth.Structures(s.Z, x - h * V, s.mol_offsets, s.cell, s.pbc)
    return (oracle.aev(sp) - oracle.aev(sm)) / (2 * h)


@pytest.mark.parametrize("name", ["gas24", "box300"])
def test_jvp_vjp_finite_differences(name):
    s = structure(name)
    rng = np.random.default_rng(11)
    V = rng.normal(size=(s.n_atoms, 3))
    T = oracle.aev_jvp(s, V)
    fd = _fd_aev(s, V)
    scale = np.abs(fd).max()
    assert np.abs(T - fd).max() < 1e-6 * scale
    # adjoint identity <G, J V> = <J^T G, V> and the VJP against finite differences of <G, aev>
    G = rng.normal(size=(s.n_atoms, 1008))
    grad, vir = oracle.aev_vjp(s, G)
    assert np.sum(G * T) == pytest.approx(np.sum(grad * V), rel=1e-10)
    assert np.sum(G * fd) == pytest.approx(np.sum(grad * V), rel=1e-6)
    # virial is symmetric; gas phase: W = sum_i x_i (x) (-dE/dx_i)
    assert np.allclose(vir, np.swapaxes(vir, 1, 2), rtol=1e-9, atol=1e-9 * np.abs(vir).max())
    if not s.pbc[0]:
        x = s.pos.astype(np.float64)
        np.testing.assert_allclose(vir[0], x.T @ (-grad), rtol=1e-9, atol=1e-9 * np.abs(vir).max())
    else:
        # diagonal virial = -dE/d(strain) of the linear functional <G, aev> under a homogeneous stretch
        h = 1e-6
        x = s.pos.astype(np.float64)
        for a in range(3):
            f = np.ones(3)
            out = []
            for sgn in (1, -1):
                f[a] = 1 + sgn * h
                c = s.cell.astype(np.float64).copy()
                c[0, 4 * a] *= f[a]
                st = synth.Structures(s.Z, x * f, s.mol_offsets, c, s.pbc)
                out.append(np.sum(G * oracle.aev(st)))
            dEde = (out[0] - out[1]) / (2 * h)
            assert -dEde == pytest.approx(vir[0, a, a], rel=1e-6)


# ------------------------------------------------------------------------ switching-function variants
SWITCHES = ("cosine", "polynomial", "exponential")


@pytest.mark.parametrize("p", [6.0, 4.0])
def test_polynomial_envelope_is_fixed_by_its_boundary_conditions(p):
    """The envelope 1 + a d^p + b d^(p+1) + c d^(p+2) with f(1) = f'(1) = f''(1) = 0: the three coefficients
    from a linear solve of those conditions, compared with the oracle's switch everywhere on [0, 1)."""
    A = np.array([[1.0, 1.0, 1.0], [p, p + 1, p + 2], [p * (p - 1), (p + 1) * p, (p + 2) * (p + 1)]])
    a, b, c = np.linalg.solve(A, [-1.0, 0.0, 0.0])
    P = oracle.Params(switch="polynomial", switch_p=p)
    for d in np.linspace(0.0, 0.999, 37):
        f, df = oracle.switch(d * 5.1, 5.1, P)
        want = 1 + a * d ** p + b * d ** (p + 1) + c * d ** (p + 2)
        dwant = (a * p * d ** (p - 1) + b * (p + 1) * d ** p + c * (p + 2) * d ** (p + 1)) / 5.1
        assert abs(f - want) < 1e-13 and abs(df - dwant) < 1e-12
    assert oracle.switch(5.1, 5.1, P) == (0.0, 0.0) and oracle.switch(6.0, 5.1, P) == (0.0, 0.0)


def test_exponential_switch_special_values():
    P = oracle.Params(switch="exponential")
    rc = 3.5
    assert oracle.switch(0.0, rc, P)[0] == 1.0
    f, _ = oracle.switch(rc / np.sqrt(2.0), rc, P)          # r^2 = rc^2 - r^2: exactly exp(-1)
    assert abs(f - np.exp(-1.0)) < 1e-15
    assert oracle.switch(rc * 0.99, rc, P)[0] < 1e-20        # flat to every order at the cutoff


@pytest.mark.parametrize("sw", SWITCHES)
def test_switch_derivative_and_smoothness(sw):
    P = oracle.Params(switch=sw)
    rc, h = 5.1, 1e-6
    for r in (0.3, 1.7, 2.9, 4.4, 5.0):
        fp, fm = oracle.switch(r + h, rc, P)[0], oracle.switch(r - h, rc, P)[0]
        assert abs((fp - fm) / (2 * h) - oracle.switch(r, rc, P)[1]) < 1e-8
    # value and slope go to zero at the cutoff (and, for these two, the curvature)
    f, df = oracle.switch(rc - 1e-5, rc, P)
    assert f < 1e-8 and abs(df) < 1e-3
    if sw != "cosine":
        d1, d2 = oracle.switch(rc - 2e-3, rc, P)[1], oracle.switch(rc - 1e-3, rc, P)[1]
        assert abs(d2 - d1) / 1e-3 < 1e-2


@pytest.mark.parametrize("sw", SWITCHES[1:])
def test_diatomic_radial_slot_with_switch(sw):
    P = oracle.Params(switch=sw)
    r = 2.37
    s = synth.Structures(np.array([6, 8], np.int32), np.array([[0, 0, 0], [r, 0, 0]], np.float32),
                         np.array([0, 2], np.int32), np.zeros((1, 9), np.float32), np.zeros(1, np.uint8))
    A = oracle.aev(s, P)
    r32 = float(np.float32(r))
    f = oracle.switch(r32, 5.1, P)[0]
    shifts = 0.8 + np.arange(16) * (5.1 - 0.8) / 16
    # atom 0 (C) sees one O: element 3's radial block
    np.testing.assert_allclose(A[0, 3 * 16:4 * 16], 0.25 * np.exp(-19.7 * (r32 - shifts) ** 2) * f, rtol=1e-12,
                               atol=1e-300)
    assert np.all(A[0, 112:] == 0.0)


@pytest.mark.parametrize("sw", SWITCHES[1:])
def test_forces_are_minus_energy_gradient_with_switch(sw):
    P = oracle.Params(switch=sw)
    s = structure("gas24")
    w = weights(1)
    r = oracle.energy_forces(s, w, P)
    rng = np.random.default_rng(5)
    h = 1e-4
    for i in rng.choice(s.n_atoms, 4, replace=False):
        for a in range(3):
            xp = np.asarray(s.pos, np.float64).copy()
            xm = xp.copy()
            xp[i, a] += h
            xm[i, a] -= h
            Ep = oracle.energy_forces(synth.Structures(s.Z, xp, s.mol_offsets, s.cell, s.pbc), w, P).energy[0]
            Em = oracle.energy_forces(synth.Structures(s.Z, xm, s.mol_offsets, s.cell, s.pbc), w, P).energy[0]
            assert abs(-(Ep - Em) / (2 * h) - r.forces[i, a]) < 1e-6 * max(1.0, abs(r.forces[i, a]))
