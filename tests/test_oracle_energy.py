"""Pins of the oracle's networks, energies, forces, virials and loss gradients.

Library special cases: the per-element networks against torch.nn.Linear + torch.nn.CELU
in float64; finite differences for forces and weight gradients; conservation laws
(sum of forces, torque, virial symmetry); extensivity and batch-composition invariance
(paper section II.A: structures in a batch never interact)."""
import itertools

import numpy as np
import pytest
import torch

import oracle
from paper_2405_01491_b300 import synth
from conftest import structure, weights

ELEM = {1: 0, 6: 1, 7: 2, 8: 3, 9: 4, 16: 5, 17: 6}


def torch_net(w, m, e):
    net = torch.nn.Sequential(torch.nn.Linear(1008, 256), torch.nn.CELU(0.1), torch.nn.Linear(256, 192),
                              torch.nn.CELU(0.1), torch.nn.Linear(192, 160), torch.nn.CELU(0.1),
                              torch.nn.Linear(160, 1)).double()
    with torch.no_grad():
        for li, (W, b) in enumerate([(w.W1, w.b1), (w.W2, w.b2), (w.W3, w.b3)]):
            net[2 * li].weight.copy_(torch.from_numpy(W[m, e].astype(np.float64)))
            net[2 * li].bias.copy_(torch.from_numpy(b[m, e].astype(np.float64)))
        net[6].weight.copy_(torch.from_numpy(w.w4[m, e].astype(np.float64))[None])
        net[6].bias.fill_(float(w.b4[m, e]))
    return net


def test_networks_match_torch_nn():
    w = weights(2)
    rng = np.random.default_rng(0)
    Z = np.array([1, 6, 7, 8, 9, 16, 17, 1, 6, 8], np.int32)
    A = rng.uniform(0, 1.5, size=(10, 1008))
    y, G = oracle.network_energies(A, Z, w)
    for i, z in enumerate(Z):
        x = torch.tensor(A[i:i + 1], requires_grad=True)
        tot = 0
        for m in range(2):
            out = torch_net(w, m, ELEM[int(z)])(x)[0, 0]
            assert float(out.detach()) == pytest.approx(y[i, m], rel=1e-12, abs=1e-14)
            tot = tot + out / 2
        gx, = torch.autograd.grad(tot, x)
        # torch's CELU backward carries alpha in single precision (about 1e-8 relative error)
        np.testing.assert_allclose(G[i], gx[0].numpy(), rtol=1e-6, atol=1e-7 * np.abs(G[i]).max())


def test_isolated_atoms_energy_is_network_at_zero():
    w = weights(2)
    # atoms 20 A apart: every AEV entry is zero, so E = mean over members of net(0)
    Z = np.array([6, 8, 17], np.int32)
    s = synth.Structures(Z, np.array([[0, 0, 0], [20, 0, 0], [0, 20, 0]], np.float32),
                         np.array([0, 3], np.int32), np.zeros((1, 9), np.float32), np.zeros(1, np.uint8))
    r = oracle.energy_forces(s, w)
    want = sum(float(torch_net(w, m, ELEM[int(z)])(torch.zeros(1, 1008, dtype=torch.float64))) / 2
               for z in Z for m in range(2))
    assert r.energy[0] == pytest.approx(want, rel=1e-12)
    assert np.all(r.forces == 0)


def _energy(s, w, x):
    return oracle.energy_forces(synth.Structures(s.Z, x, s.mol_offsets, s.cell, s.pbc), w).energy


@pytest.mark.parametrize("name,M", [("gas24", 2), ("box300", 1)])
def test_forces_are_minus_energy_gradient(name, M):
    s = structure(name)
    w = weights(M)
    r = oracle.energy_forces(s, w)
    x = s.pos.astype(np.float64)
    rng = np.random.default_rng(2)
    for _ in range(2):
        V = rng.normal(size=x.shape)
        h = 1e-5
        fd = (_energy(s, w, x + h * V) - _energy(s, w, x - h * V)).sum() / (2 * h)
        assert -np.sum(r.forces * V) == pytest.approx(fd, rel=1e-6, abs=1e-9)
    np.testing.assert_allclose(r.forces.sum(0), 0, atol=1e-10)
    vir = r.virial[0]
    np.testing.assert_allclose(vir, vir.T, atol=1e-9 * max(1, np.abs(vir).max()))
    if not s.pbc[0]:
        torque = np.cross(x, r.forces).sum(0)
        np.testing.assert_allclose(torque, 0, atol=1e-9)


def test_batch_composition_invariance():
    b = structure("batch64")
    w = weights(1)
    rb = oracle.energy_forces(b, w)
    for m in (0, 17, 63):
        one = b.molecule(m)
        r1 = oracle.energy_forces(one, w)
        a0, a1 = b.mol_offsets[m], b.mol_offsets[m + 1]
        assert r1.energy[0] == pytest.approx(rb.energy[m], rel=1e-12, abs=1e-12)
        np.testing.assert_allclose(r1.forces, rb.forces[a0:a1], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(r1.virial[0], rb.virial[m], rtol=1e-10, atol=1e-12)


def test_supercell_energy_is_extensive():
    s = structure("box300")
    w = weights(1)
    L = float(s.cell[0, 0])
    x = s.pos.astype(np.float64)
    big = synth.Structures(np.tile(s.Z, 8), np.concatenate([x + L * np.array(n) for n in itertools.product(range(2), repeat=3)]),
                           np.array([0, 8 * s.n_atoms], np.int32), (s.cell * 2).astype(np.float64), s.pbc)
    r = oracle.energy_forces(s, w)
    rb = oracle.energy_forces(big, w)
    assert rb.energy[0] == pytest.approx(8 * r.energy[0], rel=1e-10)
    np.testing.assert_allclose(rb.forces[:s.n_atoms], r.forces, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(rb.virial[0], 8 * r.virial[0], rtol=1e-9, atol=1e-9)


def test_loss_weight_gradients_finite_differences():
    b = structure("batch64").molecule(3)
    b2 = synth.concat([b, structure("batch64").molecule(5)])
    w = weights(2)
    E_ref, F_ref = synth.batch_targets(b2, seed=9)
    L, E, F, grads = oracle.loss_and_weight_grads(b2, w, E_ref, F_ref)
    r = oracle.energy_forces(b2, w)
    np.testing.assert_allclose(E, r.energy, rtol=1e-12)
    np.testing.assert_allclose(F, r.forces, rtol=1e-10, atol=1e-12)
    rng = np.random.default_rng(4)
    names = ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")
    for trial in range(2):
        D = {k: rng.normal(size=getattr(w, k).shape) for k in names}
        # CELU'' jumps at 0 (0 vs 1/alpha), so the force loss is only C^1 in the weights and the central
        # difference error is O(h) wherever a pre-activation crosses zero: use tiny steps in float64.
        h = 1e-7 if trial == 0 else 2e-7

        def Lat(sgn):
            wp = synth.Weights(*(getattr(w, k).astype(np.float64) + sgn * h * D[k] for k in names))
            return oracle.loss_and_weight_grads(b2, wp, E_ref, F_ref)[0]

        fd = (Lat(1) - Lat(-1)) / (2 * h)
        an = sum(float(np.sum(grads[k] * D[k])) for k in names)
        assert an == pytest.approx(fd, rel=1e-6)


def test_velocity_verlet_conserves_energy_and_is_time_reversible():
    """Pins of the reference integrator: with a small step the total energy of an isolated molecule is
    conserved to second order in dt, and running back from the end (velocities negated) returns the
    starting positions (velocity Verlet is time reversible)."""
    s = structure("gas24")
    w = weights(1)
    rng = np.random.default_rng(8)
    v0 = rng.normal(scale=0.003, size=(s.n_atoms, 3))
    el = oracle.elements(s.Z)
    m = np.asarray([oracle.MASS[int(e)] for e in el])[:, None]
    kin = lambda v: 0.5 * np.sum(m * v * v) / oracle.ACCEL   # kcal/mol

    def drift(dt):
        E, x, v, F = oracle.velocity_verlet(s, w, v0, 21, dt)
        e0 = E[0, 0] + kin(v0)
        e1 = E[-1, 0] + kin(v)
        return abs(e1 - e0), x, v

    d1, x1, v1 = drift(0.2)
    d2, _, _ = drift(0.1)
    assert d2 < d1 / 2.5          # second-order integrator: halving dt cuts the error about 4x
    back = synth.Structures(s.Z, x1, s.mol_offsets, s.cell, s.pbc)
    _, x0, _, _ = oracle.velocity_verlet(back, w, -v1, 21, 0.2)
    np.testing.assert_allclose(x0, s.pos.astype(np.float64), atol=1e-9)


def test_celu_kink_deltas_are_one_sided_gradient_jumps():
    """Put one pre-activation exactly on the CELU kink by shifting its bias, then the loss gradients
    just above and just below it (float64 autograd) differ by the jump celu_kink_deltas predicts."""
    s = structure("gas24")
    base = weights(1)
    names = ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")

    class W64:
        n_members = 1

    def with_bias(layer, e, u, value):
        w = W64()
        for k in names:
            setattr(w, k, np.array(getattr(base, k), np.float64))
        getattr(w, f"b{layer}")[0, e, u] = value
        return w

    E_ref, F_ref = synth.batch_targets(s)
    el = oracle.elements(s.Z)
    A = oracle.aev(s)
    checked = 0
    for layer, e in [(1, 1), (2, 0), (3, 3)]:
        rows = np.nonzero(el == e)[0]
        W1, b1, W2, b2, W3, b3, _, _ = oracle._layers(base, 0, e)
        h = A[rows]
        for W, b in [(W1, b1), (W2, b2), (W3, b3)][:layer]:
            z = h @ W.T + b
            h = oracle.celu(z)
        # moving the row nearest the kink onto it keeps every other row of the unit on its side
        for u in range(z.shape[1]):
            ri = int(np.argmin(np.abs(z[:, u])))
            if np.min(np.abs(np.delete(z[:, u], ri) - z[ri, u]), initial=1.0) < 1e-3:
                continue
            b0 = float([b1, b2, b3][layer - 1][u]) - z[ri, u]
            eps = 1e-9
            lo, hi = with_bias(layer, e, u, b0 - eps), with_bias(layer, e, u, b0 + eps)
            g_lo = oracle.loss_and_weight_grads(s, lo, E_ref, F_ref)[3]
            g_hi = oracle.loss_and_weight_grads(s, hi, E_ref, F_ref)[3]
            found = [d for (m, ee, l, atom, uu, d) in oracle.celu_kink_deltas(s, lo, E_ref, F_ref)
                     if (m, ee, l, atom, uu) == (0, e, layer, int(rows[ri]), u)]
            assert len(found) == 1
            d = found[0]
            jump = sum(np.linalg.norm(d[k]) for k in names)
            assert jump > 0
            for k in names:
                np.testing.assert_allclose(g_hi[k][0, e] - g_lo[k][0, e], d[k], rtol=0, atol=1e-6 * jump)
                other = np.delete(g_hi[k] - g_lo[k], e, axis=1)
                assert np.abs(other).max() <= 1e-6 * jump
            checked += 1
            break
    assert checked == 3
