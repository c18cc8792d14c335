"""The fused AEV -> first-layer kernel (FNN_BF16_FUSED): the BF16 form's arithmetic with each 64-row tile of
AEV rows built in shared memory as the first layer's tensor-core operand (section II.E).

Against the unfused BF16 form it differs only in where the bf16 AEV lives and in the tile height of the
first product, so energies and forces agree to the order of FP32 sums (the force scatter's atomics):
per-atom energy within 1e-6 kcal/mol, forces within 1e-4 kcal/mol/A.  Against the float64 oracle it is
held to the BF16 form's bounds (per-atom energy 1e-2 kcal/mol, RMS force error 3% of the RMS force)."""
import numpy as np
import pytest

import oracle
from paper_2405_01491_b300 import synth
from conftest import structure, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fnn():
    import torch
    assert torch.cuda.is_available()
    from paper_2405_01491_b300 import fnn as f
    return f


def _run(fnn, s, M, precisions, skin=0.0):
    ctx = fnn.Context(M, skin=skin)
    fnn.load_weights(ctx, weights(M))
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    out = {}
    for p in precisions:
        E, F, W = fnn.energy_forces(ctx, ds, nl, p)
        fnn.check(ctx, p)
        out[p] = (E.cpu().numpy(), F.cpu().numpy(), W.cpu().numpy())
    return out


def _agree(s, a, b):
    n_mol_atoms = np.maximum(np.diff(s.mol_offsets), 1)
    dE = float((np.abs(a[0] - b[0]) / n_mol_atoms).max())
    dF = float(np.abs(a[1] - b[1]).max()) if s.n_atoms else 0.0
    return dE, dF


def _ragged_tiles():
    """Structures whose element segments end at every offset within a 64-row tile: one atom of a rare
    element, segments of 1..63 rows and of more than 128, a single-atom structure, an empty one."""
    rng = np.random.default_rng(71)
    parts = [synth.random_molecule(rng, n) for n in (1, 3, 17, 40, 63)]
    parts.append(synth.mix_box(900, (900 / 0.1) ** (1 / 3), seed=72, fractions=synth.MIX7))
    parts.append(synth.Structures(np.zeros(0, np.int32), np.zeros((0, 3), np.float32), np.array([0, 0], np.int32),
                                  np.zeros((1, 9), np.float32), np.zeros(1, np.uint8)))
    return synth.concat(parts, "ragged_tiles")


CASES = [("box1500", 2, 0.0), ("batch64", 1, 0.5), ("water216", 8, 1.0), ("boxes3", 1, 0.0), ("ragged", 3, 0.0)]


@pytest.mark.parametrize("name,M,skin", CASES)
def test_fused_matches_unfused_bf16(fnn, name, M, skin):
    s = _ragged_tiles() if name == "ragged" else structure(name)
    out = _run(fnn, s, M, ["bf16", "bf16_fused"], skin)
    dE, dF = _agree(s, out["bf16"], out["bf16_fused"])
    print(f"fused vs bf16 {name} M={M}: max|dE|/atom={dE:.2e} max|dF|={dF:.2e}")
    assert dE <= 1e-6 and dF <= 1e-4, (dE, dF)


@pytest.mark.parametrize("name,M", [("box1500", 2), ("batch64", 1), ("water216", 8)])
def test_fused_error_against_oracle(fnn, name, M):
    s = structure(name)
    E, F, W = _run(fnn, s, M, ["bf16_fused"])["bf16_fused"]
    r = oracle.energy_forces(s, weights(M))
    n_mol_atoms = np.maximum(np.diff(s.mol_offsets), 1)
    dE = float((np.abs(E - r.energy) / n_mol_atoms).max())
    rel = float(np.sqrt(np.mean((F - r.forces) ** 2) / np.mean(r.forces ** 2)))
    print(f"bf16_fused {name}: max|dE|/atom={dE:.2e} max|dF|={np.abs(F - r.forces).max():.2e} rms rel F={rel:.2e}")
    assert dE <= 1e-2 and rel <= 3e-2


def test_fused_full_box_against_oracle(fnn):
    """The 23,558-atom box with the 8-member ensemble, in the launch configuration the benchmark times: the
    fused form against the oracle (BF16 bounds) and against the unfused BF16 form."""
    s = structure("mix23558")
    out = _run(fnn, s, 8, ["bf16", "bf16_fused"])
    dE, dF = _agree(s, out["bf16"], out["bf16_fused"])
    assert dE <= 1e-6 and dF <= 1e-4, (dE, dF)
    r = oracle.energy_forces(s, weights(8))
    E, F, _ = out["bf16_fused"]
    rel = float(np.sqrt(np.mean((F - r.forces) ** 2) / np.mean(r.forces ** 2)))
    assert abs(E[0] - r.energy[0]) / s.n_atoms <= 1e-2 and rel <= 3e-2


def test_fused_graph_replay_matches_eager(fnn):
    """One step (list rebuild + fused evaluation) captured as a CUDA graph and replayed gives the eager result."""
    s = structure("box1500")
    M = 2
    ctx = fnn.Context(M)
    fnn.load_weights(ctx, weights(M))
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    E0, F0, _ = fnn.energy_forces(ctx, ds, nl, "bf16_fused")
    E0, F0 = E0.cpu().numpy(), F0.cpu().numpy()
    g = fnn.Graph(ctx, ds, nl, "bf16_fused")
    for _ in range(3):
        g.launch()
    g.stream.synchronize()
    fnn.check(ctx, "graph")
    np.testing.assert_allclose(g.E.cpu().numpy(), E0, rtol=0, atol=1e-6 * s.n_atoms)
    assert np.abs(g.F.cpu().numpy() - F0).max() <= 1e-4


def test_fused_form_in_md_and_serving(fnn):
    """The fused form drives device MD (graph blocks with conditional rebuilds) and the server like the unfused
    BF16 form: the same energies along 12 steps of the water box, within the force scatter's rounding."""
    import torch
    s = structure("water216")
    v0 = synth.maxwell_boltzmann(s.Z, 300.0, seed=7)
    runs = {}
    for form in ("bf16", "bf16_fused"):
        ctx = fnn.Context(1, skin=1.0)
        fnn.load_weights(ctx, weights(1))
        ds = fnn.DeviceSystem.from_structures(s)
        vel = torch.zeros((s.n_atoms, 4), dtype=torch.float32)
        vel[:, :3] = torch.from_numpy(v0)
        vel = vel.cuda()
        nl = fnn.NeighborList(ctx)
        stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            E, _ = fnn.md_run(ctx, ds, vel, nl, form, 12, 0.5, 4, stream=stream)
        fnn.check(ctx, "md_run", stream=stream)
        srv = fnn.Server(ctx, 8 << 30, form, rebuild_every=4)
        r = srv.poll(srv.submit(s, v0, 12, 0.5), timeout_s=120)
        srv.close()
        runs[form] = (E.cpu().numpy()[:, 0], r["energies"])
    for k in range(2):
        d = np.abs(runs["bf16"][k] - runs["bf16_fused"][k]).max() / s.n_atoms
        assert d <= 1e-6, (k, d)
