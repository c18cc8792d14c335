"""Variants of the descriptor (section II.A switching functions; Appendix A angular resources) on the GPU,
through the C ABI, against the float64 oracle with the same tolerances as the ANI path."""
import numpy as np
import pytest

import oracle
from paper_2405_01491_b300 import synth
from conftest import structure, weights

pytestmark = pytest.mark.gpu
E_TOL_PER_ATOM = 1e-4
F_TOL = 1e-3


@pytest.fixture(scope="module")
def fnn():
    import torch
    assert torch.cuda.is_available()
    from paper_2405_01491_b300 import fnn as f
    return f


@pytest.mark.parametrize("sw", ["polynomial", "exponential"])
@pytest.mark.parametrize("name,skin", [("gas24", 0.0), ("water216", 1.0), ("batch64", 0.5)])
def test_switch_variants_aev_and_tangent(fnn, sw, name, skin):
    import torch
    s = structure(name)
    P = oracle.Params(switch=sw)
    ctx = fnn.Context(1, skin=skin, switch=sw)
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    A = fnn.aev(ctx, ds, nl).cpu().numpy()
    fnn.check(ctx)
    want = oracle.aev(s, P)
    assert np.abs(A - want).max() <= 2e-5 * np.abs(want).max() + 1e-6
    V = np.random.default_rng(7).standard_normal((s.n_atoms, 3)).astype(np.float32)
    T = fnn.aev_jvp(ctx, ds, nl, torch.from_numpy(V).cuda()).cpu().numpy()
    fnn.check(ctx)
    Tw = oracle.aev_jvp(s, V, P)
    assert np.abs(T - Tw).max() <= 1e-4 * np.abs(Tw).max() + 1e-6


@pytest.mark.parametrize("sw", ["polynomial", "exponential"])
@pytest.mark.parametrize("name,M,precision", [("gas24", 1, "fp32"), ("water216", 2, "fp32x3"),
                                              ("box1500", 1, "fp32x3")])
def test_switch_variants_energy_forces(fnn, sw, name, M, precision):
    s = structure(name)
    P = oracle.Params(switch=sw)
    ctx = fnn.Context(M, skin=0.5, switch=sw)
    fnn.load_weights(ctx, weights(M))
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    E, F, W = fnn.energy_forces(ctx, ds, nl, precision)
    fnn.check(ctx)
    r = oracle.energy_forces(s, weights(M), P)
    n = np.maximum(np.diff(s.mol_offsets), 1)
    assert (np.abs(E.cpu().numpy() - r.energy) / n).max() <= E_TOL_PER_ATOM
    assert np.abs(F.cpu().numpy() - r.forces).max() <= F_TOL
    scale = max(1.0, np.abs(r.virial).max())
    assert np.abs(W.cpu().numpy().reshape(r.virial.shape) - r.virial).max() <= 1e-4 * scale


@pytest.mark.parametrize("name,skin,sw", [("gas24", 0.0, "cosine"), ("water216", 1.0, "cosine"),
                                          ("batch64", 0.5, "polynomial"), ("box1500", 0.0, "exponential"),
                                          ("box1100", 0.0, "cosine")])
def test_crate_angular_and_vjp_parity(fnn, name, skin, sw):
    import torch
    s = structure(name)
    P = oracle.Params(switch=sw)
    rng = np.random.default_rng(11)
    V = (rng.standard_normal((7, 8, 32)) / 4).astype(np.float32)
    G = rng.standard_normal((s.n_atoms, 4, 32)).astype(np.float32)
    ctx = fnn.Context(1, skin=skin, switch=sw)
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    Vd, Gd = torch.from_numpy(V).cuda(), torch.from_numpy(G).cuda()
    g = fnn.crate_angular(ctx, ds, nl, Vd).cpu().numpy()
    gx, gV = fnn.crate_angular_vjp(ctx, ds, nl, Vd, Gd)
    fnn.check(ctx)
    gw, gxw, gVw = oracle.crate_angular(s, V, P, G=G)
    assert np.abs(g - gw).max() <= 2e-5 * np.abs(gw).max() + 1e-6
    assert np.abs(gx.cpu().numpy() - gxw).max() <= 1e-4 * np.abs(gxw).max() + 1e-5
    assert np.abs(gV.cpu().numpy() - gVw).max() <= 1e-4 * np.abs(gVw).max() + 1e-5
