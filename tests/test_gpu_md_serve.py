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


def _md_ex(fnn, s, v0, M, precision, n, dt, skin, rebuild, side_stream=True, **kw):
    """fnn_md_run_ex with counters and the kinetic history; on a side stream blocks run as graph replays."""
    import torch
    ctx = fnn.Context(M, skin=skin)
    fnn.load_weights(ctx, weights(M))
    ds = fnn.DeviceSystem.from_structures(s)
    vel = torch.zeros((s.n_atoms, 4), dtype=torch.float32)
    vel[:, :3] = torch.from_numpy(np.asarray(v0, np.float32))
    vel = vel.cuda()
    nl = fnn.NeighborList(ctx)
    stream = torch.cuda.Stream() if side_stream else None
    torch.cuda.synchronize()
    with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
        E, K, F, cnt = fnn.md_run_ex(ctx, ds, vel, nl, precision, n, dt, rebuild, kinetic=True, counters=True,
                                     stream=stream, **kw)
    fnn.check(ctx, "md_run_ex", stream=stream)
    return (E.cpu().numpy(), K.cpu().numpy(), ds.pos[:, :3].cpu().numpy(), vel[:, :3].cpu().numpy(),
            F.cpu().numpy(), cnt)


@pytest.mark.parametrize("name,M,precision,rebuild,graph", [("gas24", 1, "fp32", 1, False),
                                                            ("water216", 1, "fp32x3", 5, True)])
def test_langevin_matches_oracle_baoab(fnn, name, M, precision, rebuild, graph):
    s = structure(name)
    v0 = _velocities(s, 4)
    n, dt, T, gamma, seed = 20, 0.5, 300.0, 0.02, 0x5eed_0001_0002
    E, K, x, v, F, cnt = _md_ex(fnn, s, v0, M, precision, n, dt, 1.0, rebuild, graph, integrator="langevin",
                                temperature_K=T, friction_per_fs=gamma, seed=seed, step0=1000)
    Er, Kr, xr, vr, Fr = oracle.langevin_baoab(s, weights(M), v0, n, dt, T, gamma, seed, step0=1000)
    assert np.abs(E - Er).max() / s.n_atoms <= E_TOL_PER_ATOM
    assert np.abs(K - Kr).max() / s.n_atoms <= E_TOL_PER_ATOM
    assert np.abs(x - xr).max() <= 1e-4 and np.abs(v - vr).max() <= 1e-5
    assert np.abs(F - Fr).max() <= 1e-3
    assert cnt["graph_blocks"] == ((n - rebuild) // rebuild if graph else 0)
    # friction and noise did act: the trajectory differs from velocity Verlet's
    Ev, xv, _, _ = oracle.velocity_verlet(s, weights(M), v0, n, dt)
    assert np.abs(xv - xr).max() > 1e-3


def test_skin_guard_rebuilds_inside_graph_blocks_and_matches_oracle(fnn):
    s = structure("water216")
    v0 = _velocities(s, 6)
    n, dt, skin, rebuild = 40, 1.5, 0.3, 10
    E, K, x, v, F, cnt = _md_ex(fnn, s, v0, 1, "fp32x3", n, dt, skin, rebuild, True)
    # atoms move ~0.05 A per step: the 0.15 A half-skin is crossed within every block of 10 steps
    assert cnt["graph_blocks"] == 3 and cnt["guard_rebuilds"] > 3
    assert cnt["rebuilds"] > n // rebuild + 3
    Er, xr, vr, Fr = oracle.velocity_verlet(s, weights(1), v0, n, dt)
    assert np.abs(E[:, 0] - Er[:, 0]).max() / s.n_atoms <= E_TOL_PER_ATOM
    assert np.abs(x - xr).max() <= 1e-4 and np.abs(F - Fr).max() <= 1e-3
    assert abs(K[-1, 0] - oracle.kinetic_energies(s, vr)[0]) / s.n_atoms <= E_TOL_PER_ATOM


def test_serving_skin_guard_matches_oracle(fnn):
    s = structure("gas24")
    v0 = _velocities(s, 8)
    n, dt = 24, 1.5
    ctx = fnn.Context(1, skin=0.2)
    fnn.load_weights(ctx, weights(1))
    srv = fnn.Server(ctx, 8 << 30, "fp32x3", rebuild_every=10)
    r = srv.poll(srv.submit(s, v0, n, dt), timeout_s=120)
    st = srv.stats()
    srv.close()
    assert st["guard_rebuilds"] > 0
    Er, xr, vr, Fr = oracle.velocity_verlet(s, weights(1), v0, n, dt)
    assert np.abs(r["energies"] - Er[:, 0]).max() / s.n_atoms <= E_TOL_PER_ATOM
    assert np.abs(r["pos"] - xr).max() <= 1e-4


def test_water_box_1000_steps_matches_oracle_every_100_steps(fnn):
    """The periodic water box under NVE for 1000 steps of 0.5 fs (8-member ensemble, FP32X3, skin 1 A, list
    rebuilt every 10 steps and by the guard): run as ten continued runs of 100 steps, the oracle evaluated
    at the GPU's positions after each (energy per atom within 1e-4, forces within 1e-3)."""
    import torch
    s = structure("water216")
    M = 8
    ctx = fnn.Context(M, skin=1.0)
    fnn.load_weights(ctx, weights(M))
    ds = fnn.DeviceSystem.from_structures(s)
    vel = torch.zeros((s.n_atoms, 4), dtype=torch.float32)
    vel[:, :3] = torch.from_numpy(_velocities(s, 2))
    vel = vel.cuda()
    nl = fnn.NeighborList(ctx)
    stream = torch.cuda.Stream()
    worst_e = worst_f = 0.0
    for chunk in range(10):
        with torch.cuda.stream(stream):
            # 101 evaluations: the first repeats the previous chunk's last position (no drift after it)
            E, K, F, cnt = fnn.md_run_ex(ctx, ds, vel, nl, "fp32x3", 101, 0.5, 10, kinetic=True, counters=True,
                                         stream=stream)
        fnn.check(ctx, "md chunk", stream=stream)
        st = synth.Structures(s.Z, ds.pos[:, :3].cpu().numpy(), s.mol_offsets, s.cell, s.pbc)
        r = oracle.energy_forces(st, weights(M))
        worst_e = max(worst_e, abs(float(E[-1, 0]) - r.energy[0]) / s.n_atoms)
        worst_f = max(worst_f, float(np.abs(F.cpu().numpy() - r.forces).max()))
        assert cnt["graph_blocks"] == 9
    assert worst_e <= E_TOL_PER_ATOM and worst_f <= 1e-3


@pytest.mark.parametrize("name,P,n,rebuild,graph", [("gas24", 4, 8, 3, False), ("water216", 8, 20, 5, True)])
def test_rpmd_matches_oracle(fnn, name, P, n, rebuild, graph):
    import torch
    s = structure(name)
    rng = np.random.default_rng(12)
    x0 = (np.asarray(s.pos, np.float64)[None] + 0.02 * rng.standard_normal((P, s.n_atoms, 3))).astype(np.float32)
    v0 = np.stack([_velocities(s, 50 + b) for b in range(P)]).astype(np.float32)
    ctx = fnn.Context(1, skin=1.0)
    fnn.load_weights(ctx, weights(1))
    ds = fnn.bead_system(s, x0)
    vel = torch.zeros((P * s.n_atoms, 4), dtype=torch.float32)
    vel[:, :3] = torch.from_numpy(v0.reshape(-1, 3))
    vel = vel.cuda()
    nl = fnn.NeighborList(ctx)
    stream = torch.cuda.Stream() if graph else None
    torch.cuda.synchronize()
    with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
        E, H, F, cnt = fnn.rpmd_run(ctx, ds, vel, nl, "fp32x3", P, n, 0.5, 300.0, rebuild, counters=True,
                                    stream=stream)
    fnn.check(ctx, "rpmd", stream=stream)
    Er, Hr, xr, vr, Fr = oracle.rpmd(s, weights(1), P, x0.astype(np.float64), v0.astype(np.float64), n, 0.5, 300.0)
    assert np.abs(E.cpu().numpy() - Er).max() / s.n_atoms <= E_TOL_PER_ATOM
    assert np.abs(H.cpu().numpy() - Hr).max() / (P * s.n_atoms) <= E_TOL_PER_ATOM
    x = ds.pos[:, :3].cpu().numpy().reshape(P, s.n_atoms, 3)
    assert np.abs(x - xr).max() <= 1e-4
    assert np.abs(F.cpu().numpy().reshape(P, s.n_atoms, 3) - Fr).max() <= 1e-3
    assert cnt["graph_blocks"] == ((n - rebuild) // rebuild if graph else 0)
