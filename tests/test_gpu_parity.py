"""Parity of the CUDA path (through the C ABI) with the float64 oracle.

Neighbour lists: bit-exact (same set of (i, j, shift)).  AEVs: float32 against float64,
|d| <= 2e-5 * max|AEV| + 1e-6.  Energies and forces of the FP32 form: |dE| / n_atoms(mol)
<= 1e-4 kcal/mol and max |dF| <= 1e-3 kcal/mol/A (the stated FP32 tolerances).
Virials: 1e-4 of the largest entry (at least 1)."""
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


def gpu_list(fnn, s, skin=0.0):
    ctx = fnn.Context(1, skin=skin)
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    row_ptr, nbr, shift = fnn.nlist_export(nl, s.n_atoms)
    ei = np.repeat(np.arange(s.n_atoms), np.diff(row_ptr))
    return ctx, ds, nl, (ei, nbr, shift)


def as_set(ei, ej, es):
    return set(zip(ei.tolist(), ej.tolist(), map(tuple, es.tolist())))


@pytest.mark.parametrize("name,skin", [("gas24", 0.0), ("water216", 1.0), ("box300", 0.0), ("box1500", 1.0),
                                       ("box1100", 0.0), ("batch64", 0.0), ("mix23558", 0.0), ("mix23558", 1.0)])
def test_neighbor_list_bit_exact(fnn, name, skin):
    s = structure(name)
    _, _, _, got = gpu_list(fnn, s, skin)
    want = oracle.neighbors(s, 5.1 + skin)
    assert len(got[0]) == len(want[0])
    assert as_set(*got) == as_set(*want)


def test_neighbor_edge_cases(fnn):
    rng = np.random.default_rng(3)
    parts = []
    # empty structure, single atom, two atoms on one axis (zero extent on two axes)
    parts.append(synth.Structures(np.zeros(0, np.int32), np.zeros((0, 3), np.float32), np.array([0, 0], np.int32),
                                  np.zeros((1, 9), np.float32), np.zeros(1, np.uint8)))
    parts.append(synth.Structures(np.array([6], np.int32), np.zeros((1, 3), np.float32), np.array([0, 1], np.int32),
                                  np.zeros((1, 9), np.float32), np.zeros(1, np.uint8)))
    parts.append(synth.Structures(np.array([1, 8], np.int32), np.array([[0, 0, 0], [0, 0, 4.0]], np.float32),
                                  np.array([0, 2], np.int32), np.zeros((1, 9), np.float32), np.zeros(1, np.uint8)))
    # small periodic box (L = 11.4 A: 2 cells per axis); some atoms outside the primary cell
    small = synth.random_molecule(rng, 150, periodic=True)
    small.pos[::4] += np.float32(small.cell[0, 0]) * np.array([1, -2, 0], np.float32)
    parts.append(small)
    # sparse gas cluster spread far apart (the cell budget clamps the grid)
    far = synth.random_molecule(rng, 40)
    far.pos *= np.float32(25.0)
    parts.append(far)
    # pairs placed at r = 5.1 give or take one float32 ulp of the coordinates (predicate band)
    x = np.array([[10.0, 10.0, 10.0], [15.1, 10.0, 10.0], [10.0, 15.100001, 10.0], [10.0, 10.0, 15.099999]], np.float32)
    parts.append(synth.Structures(np.array([6, 6, 1, 8], np.int32), x, np.array([0, 4], np.int32),
                                  np.zeros((1, 9), np.float32), np.zeros(1, np.uint8)))
    b = synth.concat(parts)
    _, _, _, got = gpu_list(fnn, b)
    want = oracle.neighbors(b, 5.1)
    assert as_set(*got) == as_set(*want)


def test_status_codes(fnn):
    s = structure("box300")
    ctx = fnn.Context(1)
    # species outside the table
    bad = synth.Structures(s.Z.copy(), s.pos, s.mol_offsets, s.cell, s.pbc)
    bad.Z[7] = 26
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, fnn.DeviceSystem.from_structures(bad), nl)
    assert fnn.sync(ctx) == (-2, 7)
    # cell edge <= 2 (rc + skin)
    cell = np.zeros((1, 9), np.float32)
    cell[0, [0, 4, 8]] = 10.0
    tiny = synth.Structures(s.Z, s.pos, s.mol_offsets, cell, s.pbc)
    fnn.build_neighbors(ctx, fnn.DeviceSystem.from_structures(tiny), nl)
    assert fnn.sync(ctx)[0] == -3
    # capacity overflow reports the entries needed
    nl2 = fnn.NeighborList(ctx, capacity=100)
    ds = fnn.DeviceSystem.from_structures(s)
    fnn.build_neighbors(ctx, ds, nl2)
    code, info = fnn.sync(ctx)
    assert code == -4 and info == len(oracle.neighbors(s, 5.1)[0])
    assert fnn.sync(ctx) == (0, 0)   # cleared
    # offsets that leave atoms outside every structure
    short = synth.Structures(s.Z, s.pos, np.array([0, s.n_atoms - 5], np.int32), s.cell, s.pbc)
    fnn.build_neighbors(ctx, fnn.DeviceSystem.from_structures(short), nl)
    assert fnn.sync(ctx)[0] == -1


@pytest.mark.parametrize("name", ["gas24", "water216", "box300", "batch64", "box1100", "mix23558"])
def test_aev_parity(fnn, name):
    s = structure(name)
    ctx, ds, nl, _ = gpu_list(fnn, s, skin=0.5)
    A = fnn.aev(ctx, ds, nl).cpu().numpy()
    fnn.check(ctx)
    want = oracle.aev(s)
    tol = 2e-5 * np.abs(want).max() + 1e-6
    assert np.abs(A - want).max() <= tol


def _energy_case(fnn, s, M, skin=0.0, precision="fp32"):
    w = weights(M)
    ctx = fnn.Context(M, skin=skin)
    fnn.load_weights(ctx, w)
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    E, F, W = fnn.energy_forces(ctx, ds, nl, precision)
    fnn.check(ctx)
    return ctx, ds, nl, E.cpu().numpy(), F.cpu().numpy(), W.cpu().numpy()


def _compare(s, r, E, F, W):
    n_mol_atoms = np.maximum(np.diff(s.mol_offsets), 1)
    dE = np.abs(E - r.energy) / n_mol_atoms
    dF = np.abs(F - r.forces).max() if s.n_atoms else 0.0
    assert dE.max() <= E_TOL_PER_ATOM, dE.max()
    assert dF <= F_TOL, dF
    scale = max(1.0, np.abs(r.virial).max())
    assert np.abs(W.reshape(r.virial.shape) - r.virial).max() <= 1e-4 * scale


FP32_FORMS = ["fp32", "fp32x3"]   # SIMT FFMA, and the three-term bf16 split on tensor cores


@pytest.mark.parametrize("precision", FP32_FORMS)
@pytest.mark.parametrize("name,M,skin", [("gas24", 1, 0.0), ("water216", 8, 1.0), ("box1500", 2, 0.0),
                                         ("box1100", 1, 0.0), ("batch64", 1, 0.5)])
def test_energy_forces_fp32_parity(fnn, name, M, skin, precision):
    s = structure(name)
    _, _, _, E, F, W = _energy_case(fnn, s, M, skin, precision=precision)
    r = oracle.energy_forces(s, weights(M))
    _compare(s, r, E, F, W)


@pytest.mark.parametrize("precision", FP32_FORMS)
def test_energy_forces_several_large_structures(fnn, precision):
    """A batch of three periodic boxes (700, 2600 and 1500 atoms): each structure's energy is a float64 sum
    over several slices of atoms, finished by whichever slice ends last, for all three at once."""
    s = structure("boxes3")
    _, _, _, E, F, W = _energy_case(fnn, s, 2, precision=precision)
    r = oracle.energy_forces(s, weights(2))
    _compare(s, r, E, F, W)


def test_neighbor_rows_sorted_by_element(fnn):
    """Rows of at most 128 entries come out sorted by neighbour element, stable within an element
    (the order the AEV kernels stage in one pass); the set is the oracle's."""
    for name, skin in (("box1500", 1.0), ("batch64", 0.0), ("mix23558", 0.0)):
        s = structure(name)
        _, _, nl, got = gpu_list(fnn, s, skin)
        assert as_set(*got) == as_set(*oracle.neighbors(s, 5.1 + skin))
        row_ptr, nbr, _ = fnn.nlist_export(nl, s.n_atoms)
        Z = np.asarray(s.Z)
        elem_of = {1: 0, 6: 1, 7: 2, 8: 3, 9: 4, 16: 5, 17: 6}
        e = np.array([elem_of[int(z)] for z in Z])[nbr]
        lens = np.diff(row_ptr)
        assert lens.max() <= 128, lens.max()
        for i in range(s.n_atoms):
            ei = e[row_ptr[i]:row_ptr[i + 1]]
            assert np.all(np.diff(ei) >= 0), (name, i, ei)


@pytest.mark.parametrize("precision", FP32_FORMS)
def test_energy_forces_fp32_full_size(fnn, precision):
    """The 23,558-atom periodic box with the 8-member ensemble, in the launch configuration the benchmark times."""
    s = structure("mix23558")
    _, _, _, E, F, W = _energy_case(fnn, s, 8, precision=precision)
    r = oracle.energy_forces(s, weights(8))
    _compare(s, r, E, F, W)


def test_host_entry_point_matches_device_path(fnn):
    s = structure("batch64")
    ctx, ds, nl, E, F, W = _energy_case(fnn, s, 1)
    Eh, Fh, Wh = fnn.energy_forces_host(ctx, s, "fp32")
    np.testing.assert_allclose(Eh, E, rtol=0, atol=1e-9)
    np.testing.assert_allclose(Fh, F, rtol=0, atol=1e-5)


def test_neighbor_list_deterministic(fnn):
    s = structure("box1500")
    ctx = fnn.Context(1)
    ds = fnn.DeviceSystem.from_structures(s)
    outs = []
    for _ in range(2):
        nl = fnn.NeighborList(ctx)
        fnn.build_neighbors(ctx, ds, nl, checked=True)
        outs.append(fnn.nlist_export(nl, s.n_atoms))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def _form_errors(s, r, E, F):
    n_mol_atoms = np.maximum(np.diff(s.mol_offsets), 1)
    dE = float((np.abs(E - r.energy) / n_mol_atoms).max())
    dF = float(np.abs(F - r.forces).max())
    rel = float(np.sqrt(np.mean((F - r.forces) ** 2) / np.mean(r.forces ** 2)))
    return dE, dF, rel


@pytest.mark.parametrize("name,M", [("box1500", 2), ("batch64", 1), ("water216", 8)])
def test_energy_forces_bf16_error(fnn, name, M):
    """BF16 tensor-core networks: no stated tolerance, so the error is reported and held to bounds
    derived from bf16 rounding (8-bit mantissa, relative 2^-8 per operand): per-atom energy error
    below 1e-2 kcal/mol and RMS force error below 3% of the RMS force."""
    s = structure(name)
    _, _, _, E, F, W = _energy_case(fnn, s, M, precision="bf16")
    r = oracle.energy_forces(s, weights(M))
    dE, dF, rel = _form_errors(s, r, E, F)
    print(f"bf16 {name}: max|dE|/atom={dE:.2e} max|dF|={dF:.2e} rms rel F={rel:.2e}")
    assert dE <= 1e-2 and rel <= 3e-2


def test_bf16_and_fp32_forms_agree_on_the_full_box(fnn):
    s = structure("mix23558")
    _, _, _, E32, F32, _ = _energy_case(fnn, s, 8, precision="fp32")
    _, _, _, E16, F16, _ = _energy_case(fnn, s, 8, precision="bf16")
    rel = np.sqrt(np.mean((F16 - F32) ** 2) / np.mean(F32 ** 2))
    assert abs(E16[0] - E32[0]) / s.n_atoms <= 1e-2 and rel <= 3e-2


@pytest.mark.parametrize("name,M", [("box1500", 2), ("batch64", 1), ("water216", 8)])
def test_energy_forces_fp8_error(fnn, name, M):
    """FP8 (e4m3, per-layer scaling) networks: no stated tolerance, so the error is reported and held
    to the BF16 bounds scaled by the ratio of the formats' spacings (3-bit against 7-bit stored
    mantissa: 16x): per-atom energy error below 0.16 kcal/mol, RMS force error below 48% of the RMS force."""
    s = structure(name)
    _, _, _, E, F, W = _energy_case(fnn, s, M, precision="fp8")
    r = oracle.energy_forces(s, weights(M))
    dE, dF, rel = _form_errors(s, r, E, F)
    print(f"fp8 {name}: max|dE|/atom={dE:.2e} max|dF|={dF:.2e} rms rel F={rel:.2e}")
    assert dE <= 0.16 and rel <= 0.48


def test_fp8_calibration_on_another_system(fnn):
    """Scales calibrated on one system serve another; recalibrating on the evaluated system gives the
    self-calibrated result exactly (the scales are a pure function of the calibration system)."""
    s, other = structure("box1500"), structure("box300")
    M = 2
    ctx = fnn.Context(M)
    fnn.load_weights(ctx, weights(M))
    ds, do = fnn.DeviceSystem.from_structures(s), fnn.DeviceSystem.from_structures(other)
    nl, no = fnn.NeighborList(ctx), fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, do, no, checked=True)
    fnn.calibrate_fp8(ctx, do, no)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    E1, F1, _ = fnn.energy_forces(ctx, ds, nl, "fp8")
    fnn.calibrate_fp8(ctx, ds, nl)
    E2, F2, _ = fnn.energy_forces(ctx, ds, nl, "fp8")
    fnn.check(ctx)
    _, _, _, E3, F3, _ = _energy_case(fnn, s, M, precision="fp8")
    np.testing.assert_array_equal(E2.cpu().numpy(), E3)
    r = oracle.energy_forces(s, weights(M))
    for E, F in ((E1, F1), (E2, F2)):
        dE, _, rel = _form_errors(s, r, E.cpu().numpy(), F.cpu().numpy())
        assert dE <= 0.16 and rel <= 0.48


def test_fp8_and_fp32_forms_agree_on_the_full_box(fnn):
    s = structure("mix23558")
    _, _, _, E32, F32, _ = _energy_case(fnn, s, 8, precision="fp32")
    _, _, _, E8, F8, _ = _energy_case(fnn, s, 8, precision="fp8")
    rel = np.sqrt(np.mean((F8 - F32) ** 2) / np.mean(F32 ** 2))
    print(f"fp8 mix23558: |dE|/atom={abs(E8[0] - E32[0]) / s.n_atoms:.2e} rms rel F={rel:.2e}")
    assert abs(E8[0] - E32[0]) / s.n_atoms <= 0.16 and rel <= 0.48


@pytest.mark.parametrize("M,precision", [(1, "fp32"), (1, "fp32x3"), (2, "fp32x3")])
def test_small_system_path_matches_oracle(fnn, M, precision):
    """Systems of at most 256 atoms (atoms x members at most 256) take the one-block list build and the single
    cooperative evaluation kernel: the same list set and the oracle's energies, forces and virials."""
    rng = np.random.default_rng(61)
    parts = [structure("gas24"), synth.random_molecule(rng, 8), synth.random_molecule(rng, 40)]
    if M == 1:
        parts.append(synth.random_molecule(rng, 150, periodic=True))
    s = synth.concat(parts, "small")
    assert s.n_atoms * M <= 256
    w = weights(M)
    ctx = fnn.Context(M, skin=0.5)
    fnn.load_weights(ctx, w)
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.profile_read(ctx)
    fnn.profile_enable(ctx, True)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    E, F, W = fnn.energy_forces(ctx, ds, nl, precision)
    fnn.check(ctx)
    fnn.profile_enable(ctx, False)
    names = set(fnn.profile_read(ctx))
    assert {"small_build", "small_eval"} <= names, names
    row_ptr, nbr, shift = fnn.nlist_export(nl, s.n_atoms)
    ei = np.repeat(np.arange(s.n_atoms), np.diff(row_ptr))
    assert as_set(ei, nbr, shift) == as_set(*oracle.neighbors(s, 5.6))
    # rows (all under 128 entries here) sorted by neighbour element
    el = oracle.elements(s.Z)
    for i in range(s.n_atoms):
        e = el[nbr[row_ptr[i]:row_ptr[i + 1]]]
        assert np.all(np.diff(e) >= 0)
    r = oracle.energy_forces(s, w)
    _compare(s, r, E.cpu().numpy(), F.cpu().numpy(), W.cpu().numpy())
    # energies are deterministic: a second evaluation gives the same bits
    E2, _, _ = fnn.energy_forces(ctx, ds, nl, precision)
    fnn.check(ctx)
    np.testing.assert_array_equal(E2.cpu().numpy(), E.cpu().numpy())
