"""Device-resident velocity Verlet and the continuous-batching server, through the C ABI.

MD: trajectories of the FP32-accurate forms against the float64 velocity-Verlet oracle (per-step
energies within the FP32 energy tolerance per atom, final positions within 1e-4 A).
Serving: each structure's result is the same alone and in a mixed batch (energies within the FP32
energy tolerance per atom, positions within 1e-4 A), under budget-limited admission."""
import time

import numpy as np
import pytest

import oracle
from paper_2405_01491_b300 import synth
from conftest import structure, weights

pytestmark = pytest.mark.gpu
E_TOL_PER_ATOM = 1e-4


@pytest.fixture(scope="module")
def fnn():
    import torch
    assert torch.cuda.is_available()
    from paper_2405_01491_b300 import fnn as f
    return f


def _velocities(s, seed):
    return synth.maxwell_boltzmann(s.Z, 300.0, seed=seed)


def _md_gpu(fnn, s, v0, M, precision, n_steps, dt, skin=1.0, rebuild=10, side_stream=False):
    """fnn_md_run; on a side stream whole blocks of `rebuild` steps run as replays of one CUDA graph."""
    import torch
    ctx = fnn.Context(M, skin=skin)
    fnn.load_weights(ctx, weights(M))
    ds = fnn.DeviceSystem.from_structures(s)
    vel = torch.zeros((s.n_atoms, 4), dtype=torch.float32)
    vel[:, :3] = torch.from_numpy(v0)
    vel = vel.cuda()
    nl = fnn.NeighborList(ctx)
    stream = torch.cuda.Stream() if side_stream else None
    torch.cuda.synchronize()
    with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
        E, F = fnn.md_run(ctx, ds, vel, nl, precision, n_steps, dt, rebuild, stream=stream)
    fnn.check(ctx, "md_run", stream=stream)
    return E.cpu().numpy(), ds.pos[:, :3].cpu().numpy(), vel[:, :3].cpu().numpy(), F.cpu().numpy()


@pytest.mark.parametrize("name,M,precision,skin,rebuild,graph", [("gas24", 1, "fp32", 0.0, 1, False),
                                                                 ("gas24", 2, "fp32x3", 1.0, 5, True),
                                                                 ("water216", 1, "fp32x3", 1.0, 10, False),
                                                                 ("water216", 2, "fp32x3", 1.0, 3, True)])
def test_md_matches_oracle_velocity_verlet(fnn, name, M, precision, skin, rebuild, graph):
    s = structure(name)
    v0 = _velocities(s, 3)
    n, dt = 20, 0.5
    E, x, v, F = _md_gpu(fnn, s, v0, M, precision, n, dt, skin, rebuild, side_stream=graph)
    Er, xr, vr, Fr = oracle.velocity_verlet(s, weights(M), v0, n, dt)
    assert np.abs(E - Er).max() / s.n_atoms <= E_TOL_PER_ATOM
    assert np.abs(x - xr).max() <= 1e-4
    assert np.abs(F - Fr).max() <= 1e-3


def _mix():
    rng = np.random.default_rng(21)
    parts = [structure("gas24"), synth.random_molecule(rng, 40), synth.random_molecule(rng, 700, periodic=True),
             structure("water216"), synth.random_molecule(rng, 9), synth.random_molecule(rng, 150)]
    steps = [12, 7, 10, 15, 3, 9]
    return parts, steps


def test_serving_result_is_the_same_alone_and_in_the_mix(fnn):
    M = 1
    parts, steps = _mix()
    vels = [_velocities(p, 30 + k) for k, p in enumerate(parts)]
    # every structure alone (one server, one structure at a time)
    alone = []
    ctx = fnn.Context(M, skin=1.0)
    fnn.load_weights(ctx, weights(M))
    srv = fnn.Server(ctx, 8 << 30, "fp32x3", rebuild_every=5)
    for p, v, k in zip(parts, vels, steps):
        t = srv.submit(p, v, k, 0.5)
        alone.append(srv.poll(t, timeout_s=120))
    srv.close()
    # all together, submitted while the first ones are running
    ctx2 = fnn.Context(M, skin=1.0)
    fnn.load_weights(ctx2, weights(M))
    srv2 = fnn.Server(ctx2, 8 << 30, "fp32x3", rebuild_every=5)
    tickets = []
    for p, v, k in zip(parts, vels, steps):
        tickets.append(srv2.submit(p, v, k, 0.5))
        time.sleep(0.002)
    mixed = [srv2.poll(t, timeout_s=120) for t in tickets]
    st = srv2.stats()
    srv2.close()
    assert st["status"] == 0 and st["max_batch_atoms"] > max(p.n_atoms for p in parts)   # really batched
    for p, a, b, k in zip(parts, alone, mixed, steps):
        assert a is not None and b is not None
        assert a["n_steps_done"] == k and b["n_steps_done"] == k
        assert np.abs(a["energies"] - b["energies"]).max() / p.n_atoms <= E_TOL_PER_ATOM
        assert np.abs(a["pos"] - b["pos"]).max() <= 1e-4


def test_serving_matches_md_run(fnn):
    s = structure("water216")
    v0 = _velocities(s, 5)
    E, x, v, F = _md_gpu(fnn, s, v0, 1, "fp32x3", 12, 0.5, 1.0, 5)
    ctx = fnn.Context(1, skin=1.0)
    fnn.load_weights(ctx, weights(1))
    srv = fnn.Server(ctx, 8 << 30, "fp32x3", rebuild_every=5)
    r = srv.poll(srv.submit(s, v0, 12, 0.5), timeout_s=120)
    srv.close()
    assert np.abs(r["energies"] - E[:, 0]).max() / s.n_atoms <= E_TOL_PER_ATOM
    assert np.abs(r["pos"] - x).max() <= 1e-4


def test_serving_admission_budget_and_poll(fnn):
    ctx = fnn.Context(1, skin=1.0)
    fnn.load_weights(ctx, weights(1))
    parts, steps = _mix()
    per_atom = 40_000
    # a budget that holds only about one large structure at a time: everything still completes, later
    # structures wait in the queue
    srv = fnn.Server(ctx, 800 * per_atom, "bf16", rebuild_every=5)
    assert srv.stats()["bytes_per_atom"] < per_atom
    tickets = [srv.submit(p, None, k, 0.5) for p, k in zip(parts, steps)]
    t0 = time.perf_counter()
    early = srv.poll(tickets[-1], timeout_s=0.0)     # pending (None) or done, but never blocks
    assert time.perf_counter() - t0 < 0.5
    res = [srv.poll(t, timeout_s=120) for t in tickets[:-1]] + [early or srv.poll(tickets[-1], timeout_s=120)]
    assert all(r is not None and r["n_steps_done"] == k for r, k in zip(res, steps))
    assert max(r["queue_ms"] for r in res) > 0.0
    # a structure larger than the whole budget is refused at submission
    big = synth.random_molecule(np.random.default_rng(2), 2000, periodic=True)
    with pytest.raises(fnn.FnnError):
        srv.submit(big, None, 1, 0.5)
    srv.close()
