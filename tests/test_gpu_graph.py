"""CUDA-graph replay of the step (fnn_graph_*), through the C ABI.

A replay runs the same kernels on the same buffers as the eager calls, so energies (fixed-order
float64 sums) are bitwise equal to an eager step on the same positions; forces are summed with
atomics, so they agree within float32 rounding (1e-5 kcal/mol/A here).  A replay reads the
positions in place: moving the atoms and replaying gives the eager result at the new positions."""
import numpy as np
import pytest

import oracle
from conftest import structure, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fnn():
    import torch
    assert torch.cuda.is_available()
    from paper_2405_01491_b300 import fnn as f
    return f


def _setup(fnn, name, M, skin=0.0):
    s = structure(name)
    ctx = fnn.Context(M, skin=skin)
    fnn.load_weights(ctx, weights(M))
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    return s, ctx, ds, nl


def _eager(fnn, torch, ctx, ds, nl, precision, stream):
    with torch.cuda.stream(stream):
        fnn.build_neighbors(ctx, ds, nl, stream=stream)
        E, F, W = fnn.energy_forces(ctx, ds, nl, precision, stream=stream)
    fnn.check(ctx, stream=stream)
    return E.cpu().numpy(), F.cpu().numpy(), W.cpu().numpy()


@pytest.mark.parametrize("name,M,precision", [("water216", 8, "fp32x3"), ("box300", 2, "bf16"),
                                              ("batch64", 1, "fp32"), ("box1500", 2, "fp8")])
def test_replay_equals_eager(fnn, name, M, precision):
    import torch
    s, ctx, ds, nl = _setup(fnn, name, M)
    g = fnn.Graph(ctx, ds, nl, precision)
    assert g.kernels > 10
    for _ in range(3):
        g.launch()
    fnn.check(ctx, stream=g.stream)
    Eg, Fg, Wg = g.E.cpu().numpy(), g.F.cpu().numpy(), g.W.cpu().numpy()
    Ee, Fe, We = _eager(fnn, torch, ctx, ds, nl, precision, g.stream)
    np.testing.assert_array_equal(Eg, Ee)
    np.testing.assert_allclose(Fg, Fe, rtol=0, atol=1e-5)
    np.testing.assert_allclose(Wg, We, rtol=1e-9, atol=1e-6)
    if precision in ("fp32", "fp32x3"):
        r = oracle.energy_forces(s, weights(M))
        n = np.maximum(np.diff(s.mol_offsets), 1)
        assert (np.abs(Eg - r.energy) / n).max() <= 1e-4
        assert np.abs(Fg - r.forces).max() <= 1e-3
    g.close()


def test_replay_reads_positions_in_place(fnn):
    """Move every atom by a seeded displacement (in the same buffer) and replay: the result is the
    eager step at the new positions, and the float64 oracle's there."""
    import torch
    s, ctx, ds, nl = _setup(fnn, "water216", 2)
    g = fnn.Graph(ctx, ds, nl, "fp32x3")
    g.launch()
    E0 = g.E.cpu().numpy().copy()
    d = np.random.default_rng(5).normal(scale=0.05, size=(s.n_atoms, 3)).astype(np.float32)
    with torch.cuda.stream(g.stream):
        ds.pos[:, :3] += torch.from_numpy(d).cuda()
        g.launch()
    fnn.check(ctx, stream=g.stream)
    Eg, Fg = g.E.cpu().numpy(), g.F.cpu().numpy()
    assert not np.array_equal(Eg, E0)
    Ee, Fe, _ = _eager(fnn, torch, ctx, ds, nl, "fp32x3", g.stream)
    np.testing.assert_array_equal(Eg, Ee)
    np.testing.assert_allclose(Fg, Fe, rtol=0, atol=1e-5)
    moved = type(s)(s.Z, ds.pos[:, :3].cpu().numpy(), s.mol_offsets, s.cell, s.pbc)
    r = oracle.energy_forces(moved, weights(2))
    assert np.abs(Eg - r.energy).max() / s.n_atoms <= 1e-4
    assert np.abs(Fg - r.forces).max() <= 1e-3


def test_graph_without_rebuild_and_stream_rules(fnn):
    import torch
    s, ctx, ds, nl = _setup(fnn, "gas24", 1)
    g = fnn.Graph(ctx, ds, nl, "fp32x3", rebuild=False)
    g.launch()
    fnn.check(ctx, stream=g.stream)
    Ee, _, _ = _eager(fnn, torch, ctx, ds, nl, "fp32x3", g.stream)
    np.testing.assert_array_equal(g.E.cpu().numpy(), Ee)
    assert g.kernels < fnn.Graph(ctx, ds, nl, "fp32x3", rebuild=True).kernels
    # the legacy default stream cannot be captured
    with pytest.raises(fnn.FnnError):
        fnn.Graph(ctx, ds, nl, "fp32x3", stream=torch.cuda.default_stream())


def test_host_entry_point_replays_repeated_calls(fnn):
    """fnn_energy_forces_host replays a graph from the second call of the same shape on: results equal
    the first (eager) call's, and follow new positions."""
    s = structure("box300")
    ctx = fnn.Context(2)
    fnn.load_weights(ctx, weights(2))
    outs = [fnn.energy_forces_host(ctx, s, "fp32x3") for _ in range(4)]
    for E, F, W in outs[1:]:
        np.testing.assert_array_equal(E, outs[0][0])
        np.testing.assert_allclose(F, outs[0][1], rtol=0, atol=1e-5)
    moved = type(s)(s.Z, (s.pos + np.float32(0.03)).astype(np.float32), s.mol_offsets, s.cell, s.pbc)
    E2, F2, _ = fnn.energy_forces_host(ctx, moved, "fp32x3")
    r = oracle.energy_forces(moved, weights(2))
    assert np.abs(E2 - r.energy).max() / s.n_atoms <= 1e-4
    assert np.abs(F2 - r.forces).max() <= 1e-3


def test_host_entry_point_after_weight_reload(fnn):
    """The entry point's recorded graph is dropped when the context's buffers are reallocated: after a
    weight reload the next call evaluates the new networks (a fresh context and the oracle agree)."""
    s = structure("box300")
    ctx = fnn.Context(2)
    fnn.load_weights(ctx, weights(2))
    for _ in range(4):   # the second call records the graph, the later ones replay it
        fnn.energy_forces_host(ctx, s, "fp32x3")
    from paper_2405_01491_b300 import synth
    w2 = synth.xavier_weights(2, seed=9)
    fnn.load_weights(ctx, w2)
    E, F, _ = fnn.energy_forces_host(ctx, s, "fp32x3")
    fresh = fnn.Context(2)
    fnn.load_weights(fresh, w2)
    Ef, Ff, _ = fnn.energy_forces_host(fresh, s, "fp32x3")
    np.testing.assert_array_equal(E, Ef)
    np.testing.assert_allclose(F, Ff, rtol=0, atol=1e-5)
    r = oracle.energy_forces(s, w2)
    assert np.abs(E - r.energy).max() / s.n_atoms <= 1e-4
    assert np.abs(F - r.forces).max() <= 1e-3


def test_graph_refuses_replay_after_reallocation(fnn):
    """A recorded graph references the context's buffers: after a weight reload its launch returns
    FNN_E_STATE (nothing runs) and a newly recorded graph evaluates the new networks."""
    s, ctx, ds, nl = _setup(fnn, "water216", 2)
    g = fnn.Graph(ctx, ds, nl, "fp32x3")
    g.launch()
    fnn.check(ctx, stream=g.stream)
    from paper_2405_01491_b300 import synth
    w2 = synth.xavier_weights(2, seed=11)
    fnn.load_weights(ctx, w2)
    with pytest.raises(fnn.FnnError):
        g.launch()
    g.close()
    g2 = fnn.Graph(ctx, ds, nl, "fp32x3")
    g2.launch()
    fnn.check(ctx, stream=g2.stream)
    r = oracle.energy_forces(s, w2)
    assert np.abs(g2.E.cpu().numpy() - r.energy).max() / s.n_atoms <= 1e-4
    g2.close()
