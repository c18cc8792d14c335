"""Failure detection on the GPU path, without faulting the GPU.

Every failure here is made on the host (bad inputs, an out-of-range request) or by a device wait with a
time limit that a test makes run out (a scan tile that never publishes its sum).  Each test checks the
status the host reads back and that the context (or the server) stays usable afterwards."""
import ctypes

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


def _stream_ptr():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_bounded_lookback_wait_gives_up_and_context_stays_usable(fnn):
    ctx = fnn.Context(1)
    fnn.load_weights(ctx, weights(1))
    assert fnn.lib.fnn_selftest_lookback(ctx.h, 0, _stream_ptr()) == 0
    assert fnn.sync(ctx) == (0, 0)                   # the scan itself is right
    assert fnn.lib.fnn_selftest_lookback(ctx.h, 1, _stream_ptr()) == 0
    code, tile = fnn.sync(ctx)
    assert code == -6 and tile in (1, 2)             # a successor of the withheld tile gave up waiting
    assert fnn.sync(ctx) == (0, 0)                   # cleared
    # the same context still evaluates correctly
    s = structure("gas24")
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    E, F, _ = fnn.energy_forces(ctx, ds, nl, "fp32")
    fnn.check(ctx)
    r = oracle.energy_forces(s, weights(1))
    assert abs(float(E.cpu()[0]) - r.energy[0]) / s.n_atoms <= E_TOL_PER_ATOM


def test_nonfinite_coordinate_is_reported_with_its_atom(fnn):
    s = structure("box300")
    ctx = fnn.Context(1)
    pos = s.pos.copy()
    pos[57, 1] = np.nan
    bad = synth.Structures(s.Z, pos, s.mol_offsets, s.cell, s.pbc)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, fnn.DeviceSystem.from_structures(bad), nl)
    assert fnn.sync(ctx) == (-7, 57)
    # the list of the good atoms is still the oracle's (the bad atom has no pairs), and a clean build follows
    fnn.build_neighbors(ctx, fnn.DeviceSystem.from_structures(s), nl, checked=True)
    row_ptr, nbr, shift = fnn.nlist_export(nl, s.n_atoms)
    assert len(nbr) == len(oracle.neighbors(s, 5.1)[0])


def _crowded_centre(n_shell=70, radius=3.0):
    """A carbon at the origin with n_shell hydrogens spread evenly (Fibonacci sphere) on a shell: only the
    carbon has more than 64 neighbours within the 3.5 A angular cutoff."""
    k = np.arange(n_shell) + 0.5
    phi = np.arccos(1 - 2 * k / n_shell)
    th = np.pi * (1 + 5 ** 0.5) * k
    shell = radius * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    pos = np.vstack([np.zeros((1, 3)), shell]).astype(np.float32) + 10.0
    Z = np.array([6] + [1] * n_shell, np.int32)
    return synth.Structures(Z, pos, np.array([0, len(Z)], np.int32), np.zeros((1, 9), np.float32),
                            np.zeros(1, np.uint8))


def test_angular_neighbour_limit_is_reported_with_its_atom(fnn):
    s = _crowded_centre()
    d = np.linalg.norm(s.pos[:, None] - s.pos[None], axis=-1)
    n_ang = ((d < 3.5).sum(1) - 1)
    assert n_ang[0] > 64 and n_ang[1:].max() <= 64
    ctx = fnn.Context(1)
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    fnn.aev(ctx, ds, nl)
    assert fnn.sync(ctx) == (-4, -1)                 # info = -(atom + 1)
    # with 60 shell atoms the same centre is within the limit and matches the oracle
    s2 = _crowded_centre(60)
    ds2 = fnn.DeviceSystem.from_structures(s2)
    fnn.build_neighbors(ctx, ds2, nl, checked=True)
    A = fnn.aev(ctx, ds2, nl).cpu().numpy()
    fnn.check(ctx)
    want = oracle.aev(s2)
    assert np.abs(A - want).max() <= 2e-5 * np.abs(want).max() + 1e-6


def test_overlapping_structure_offsets_are_rejected(fnn):
    s = structure("box300")
    N = s.n_atoms
    ctx = fnn.Context(1)
    nl = fnn.NeighborList(ctx)
    # offsets that are consistent structure by structure but overlap ([0, N) twice): every structure is
    # dropped, the call reports FNN_E_INVALID and writes no list entries
    cell = np.repeat(s.cell, 3, 0)
    pbc = np.repeat(s.pbc, 3)
    over = synth.Structures(s.Z, s.pos, np.array([0, N, 0, N], np.int32), cell, pbc)
    fnn.build_neighbors(ctx, fnn.DeviceSystem.from_structures(over), nl)
    code, _ = fnn.sync(ctx)
    assert code == -1
    assert fnn.nlist_nnz(nl) == 0
    fnn.build_neighbors(ctx, fnn.DeviceSystem.from_structures(s), nl, checked=True)
    assert fnn.nlist_nnz(nl) == len(oracle.neighbors(s, 5.1)[0])


def test_serving_rejects_bad_requests_and_isolates_a_failing_structure(fnn):
    rng = np.random.default_rng(23)
    good = [structure("gas24"), synth.random_molecule(rng, 40), synth.random_molecule(rng, 600, periodic=True)]
    vels = [synth.maxwell_boltzmann(p.Z, 300.0, seed=40 + k) for k, p in enumerate(good)]
    steps = [8, 6, 7]
    ctx = fnn.Context(1, skin=1.0)
    fnn.load_weights(ctx, weights(1))
    srv = fnn.Server(ctx, 8 << 30, "fp32x3", rebuild_every=1)
    g = structure("gas24")
    # rejected at submission, before reaching the shared batch
    badZ = synth.Structures(g.Z.copy(), g.pos, g.mol_offsets, g.cell, g.pbc)
    badZ.Z[3] = 26
    nanp = synth.Structures(g.Z, g.pos.copy(), g.mol_offsets, g.cell, g.pbc)
    nanp.pos[5, 0] = np.inf
    p600 = good[2]
    small = synth.Structures(p600.Z, p600.pos, p600.mol_offsets, np.diag([12.0, 30.0, 30.0]).reshape(1, 9)
                             .astype(np.float32), p600.pbc)
    skew = synth.Structures(p600.Z, p600.pos, p600.mol_offsets, p600.cell.copy(), p600.pbc)
    skew.cell[0, 1] = 0.5
    for bad, code in ((badZ, -2), (nanp, -7), (small, -3), (skew, -3)):
        with pytest.raises(fnn.FnnError) as e:
            srv.submit(bad, None, 3, 0.5)
        assert e.value.code == code
    # a structure that turns non-finite while running (its atoms thrown to infinity by a huge step) fails
    # its own ticket only; the others run in the same batch steps and give their results alone
    doomed = synth.random_molecule(rng, 9)
    tickets = [srv.submit(p, v, k, 0.5) for p, v, k in zip(good[:2], vels[:2], steps[:2])]
    t_doomed = srv.submit(doomed, np.full((9, 3), 1e6, np.float32), 5, 1e35)
    tickets.append(srv.submit(good[2], vels[2], steps[2], 0.5))
    with pytest.raises(fnn.FnnError) as e:
        srv.poll(t_doomed, timeout_s=120)
    assert e.value.code == -7
    mixed = [srv.poll(t, timeout_s=120) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["status"] == 0 and st["failed"] == 1
    ctx2 = fnn.Context(1, skin=1.0)
    fnn.load_weights(ctx2, weights(1))
    srv2 = fnn.Server(ctx2, 8 << 30, "fp32x3", rebuild_every=1)
    alone = [srv2.poll(srv2.submit(p, v, k, 0.5), timeout_s=120) for p, v, k in zip(good, vels, steps)]
    srv2.close()
    for p, a, b, k in zip(good, alone, mixed, steps):
        assert b is not None and b["n_steps_done"] == k
        assert np.abs(a["energies"] - b["energies"]).max() / p.n_atoms <= E_TOL_PER_ATOM
        assert np.abs(a["pos"] - b["pos"]).max() <= 1e-4


def test_small_build_reports_bad_inputs(fnn):
    """The one-block build of small systems (at most 256 atoms) makes the same checks as the cell-list build."""
    s = structure("gas24")
    ctx = fnn.Context(1)
    nl = fnn.NeighborList(ctx)
    pos = s.pos.copy()
    pos[9, 2] = np.nan
    fnn.build_neighbors(ctx, fnn.DeviceSystem.from_structures(synth.Structures(s.Z, pos, s.mol_offsets, s.cell,
                                                                                 s.pbc)), nl)
    assert fnn.sync(ctx) == (-7, 9)
    Z = s.Z.copy()
    Z[4] = 26
    fnn.build_neighbors(ctx, fnn.DeviceSystem.from_structures(synth.Structures(Z, s.pos, s.mol_offsets, s.cell,
                                                                                 s.pbc)), nl)
    assert fnn.sync(ctx) == (-2, 4)
    over = synth.Structures(s.Z, s.pos, np.array([0, 24, 0, 24], np.int32), np.zeros((3, 9), np.float32),
                            np.zeros(3, np.uint8))
    fnn.build_neighbors(ctx, fnn.DeviceSystem.from_structures(over), nl)
    assert fnn.sync(ctx)[0] == -1 and fnn.nlist_nnz(nl) == 0
    nl_small = fnn.NeighborList(ctx, capacity=50)
    fnn.build_neighbors(ctx, fnn.DeviceSystem.from_structures(s), nl_small)
    code, info = fnn.sync(ctx)
    assert code == -4 and info == len(oracle.neighbors(s, 5.1)[0])
