"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This module only draws numbers: structures (species, positions, cells), random
model parameters and request streams. It holds none of the method's arithmetic
(no neighbour search, no symmetry functions, no network evaluation) and imports
neither the oracle nor the CUDA binding, so both sides can consume its output
without sharing code.

Workloads (the paper's water boxes and ANI-2x weights are not available, so
these stand in for their shapes and densities; paper section V.E):

* ``gas24``      24-atom gas-phase cluster (10 H, 8 C, 3 N, 3 O) in a 6 A cube.
* ``water216``   216 rigid H2O in an 18.64 A periodic cube (1.0 g/cm^3).
* ``mix23558``   23,558-atom periodic mixture in a 62.2 A cube (0.1 atoms/A^3).
* ``batch4096``  4096 gas-phase molecules of 8..64 atoms (ragged batch).
* request stream: Poisson arrivals of molecules / boxes, log-uniform sizes.

Positions are float32 (the precision the CUDA path consumes); every consumer
widens the same float32 values.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Atomic numbers of the seven elements the model knows, in table order.
Z_TABLE = (1, 6, 7, 8, 9, 16, 17)
D_MIN = 0.95          # minimum pair distance of every synthetic structure, A
GAS_DENSITY = 0.111   # atoms / A^3 used to size gas-phase cubes (24 atoms / 6^3 A^3)
PBC_DENSITY = 0.1     # atoms / A^3 used to size periodic cubes
# composition of the ragged batch and the request stream (H C N O F S Cl)
MIX7 = (0.50, 0.30, 0.07, 0.08, 0.02, 0.02, 0.01)

# layer widths of every per-element network: AEV length -> 256 -> 192 -> 160 -> 1
LAYER_DIMS = (1008, 256, 192, 160, 1)


@dataclasses.dataclass
class Structures:
    """A ragged batch of structures, concatenated (paper section II.A batching).

    Z           int32  [N]        atomic numbers
    pos         float32[N, 3]     Cartesian positions, A
    mol_offsets int32  [n_mol+1]  atoms of molecule m are [mol_offsets[m], mol_offsets[m+1])
    cell        float32[n_mol, 9] row-major cell vectors (row a = lattice vector a); zero when not periodic
    pbc         uint8  [n_mol]    1 = periodic (minimum image), 0 = gas phase
    """
    Z: np.ndarray
    pos: np.ndarray
    mol_offsets: np.ndarray
    cell: np.ndarray
    pbc: np.ndarray
    name: str = ""

    @property
    def n_atoms(self) -> int:
        return int(self.Z.shape[0])

    @property
    def n_mol(self) -> int:
        return int(self.mol_offsets.shape[0] - 1)

    def molecule(self, m: int) -> "Structures":
        a, b = int(self.mol_offsets[m]), int(self.mol_offsets[m + 1])
        return Structures(self.Z[a:b].copy(), self.pos[a:b].copy(),
                          np.array([0, b - a], np.int32), self.cell[m:m + 1].copy(),
                          self.pbc[m:m + 1].copy(), f"{self.name}[{m}]")


def concat(parts: list["Structures"], name: str = "") -> Structures:
    """Concatenate structures into one ragged batch."""
    sizes = [p.n_atoms for p in parts]
    offs = np.zeros(len(parts) + 1, np.int64)
    offs[1:] = np.cumsum([p.n_atoms for p in parts])
    # each part may itself hold several molecules
    mol_offsets = [0]
    base = 0
    for p in parts:
        mol_offsets.extend((p.mol_offsets[1:] + base).tolist())
        base += p.n_atoms
    del sizes
    return Structures(
        np.concatenate([p.Z for p in parts]).astype(np.int32),
        np.concatenate([p.pos for p in parts]).astype(np.float32),
        np.asarray(mol_offsets, np.int32),
        np.concatenate([p.cell for p in parts]).astype(np.float32),
        np.concatenate([p.pbc for p in parts]).astype(np.uint8),
        name,
    )


def _counts_largest_remainder(n: int, fractions) -> np.ndarray:
    f = np.asarray(fractions, np.float64)
    f = f / f.sum()
    raw = f * n
    base = np.floor(raw).astype(np.int64)
    rem = n - int(base.sum())
    order = np.argsort(-(raw - base), kind="stable")
    base[order[:rem]] += 1
    return base


def _place_min_distance(rng: np.random.Generator, n: int, box: float, periodic: bool,
                        d_min: float = D_MIN, max_rounds: int = 10000) -> np.ndarray:
    """Uniform points in a cube with every pair at least d_min apart.

    All points are drawn at once; while any pair is closer than d_min, the
    higher-indexed point of each offending pair is redrawn (a parallel form of
    random sequential addition).  Distances use the minimum image when periodic.
    """
    from scipy.spatial import cKDTree

    x = rng.uniform(0.0, box, size=(n, 3))
    for _ in range(max_rounds):
        xf = x.astype(np.float32).astype(np.float64)
        if periodic:
            xf = np.mod(xf, box)
            tree = cKDTree(xf, boxsize=box * (1 + 1e-12))
        else:
            tree = cKDTree(xf)
        pairs = tree.query_pairs(d_min * (1 + 1e-6), output_type="ndarray")
        if pairs.shape[0] == 0:
            return x.astype(np.float32)
        bad = np.unique(np.max(pairs, axis=1))
        x[bad] = rng.uniform(0.0, box, size=(bad.shape[0], 3))
    raise RuntimeError("could not place points at the requested minimum distance")


def random_molecule(rng: np.random.Generator, n: int, fractions=MIX7, periodic: bool = False,
                    name: str = "") -> Structures:
    """One molecule (gas cube of density 0.111) or periodic box (density 0.1), species iid."""
    Z = np.asarray(Z_TABLE, np.int32)[rng.choice(7, size=n, p=np.asarray(fractions) / np.sum(fractions))]
    if periodic:
        L = (n / PBC_DENSITY) ** (1.0 / 3.0)
        pos = _place_min_distance(rng, n, L, True)
        cell = np.zeros((1, 9), np.float32)
        cell[0, [0, 4, 8]] = np.float32(L)
        pbc = np.ones(1, np.uint8)
    else:
        L = (n / GAS_DENSITY) ** (1.0 / 3.0)
        pos = _place_min_distance(rng, n, L, False)
        cell = np.zeros((1, 9), np.float32)
        pbc = np.zeros(1, np.uint8)
    return Structures(Z, pos, np.array([0, n], np.int32), cell, pbc, name)


def gas24(seed: int = 1) -> Structures:
    """24-atom gas cluster: 10 H, 8 C, 3 N, 3 O, uniform in a 6 A cube, d_min 0.95."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Z = np.array([1] * 10 + [6] * 8 + [7] * 3 + [8] * 3, np.int32)
    Z = Z[rng.permutation(24)]
    pos = _place_min_distance(rng, 24, 6.0, False)
    return Structures(Z, pos, np.array([0, 24], np.int32), np.zeros((1, 9), np.float32),
                      np.zeros(1, np.uint8), "gas24")


def water216(seed: int = 2, n_side: int = 6, L: float = 18.64) -> Structures:
    """216 rigid waters (O-H 0.9572 A, HOH 104.52 deg) on a 6^3 lattice, random orientations."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = L / n_side
    r_oh, ang = 0.9572, math.radians(104.52)
    # body frame: O at origin, H's in the xy plane symmetric about x
    h1 = np.array([r_oh * math.cos(ang / 2), r_oh * math.sin(ang / 2), 0.0])
    h2 = np.array([r_oh * math.cos(ang / 2), -r_oh * math.sin(ang / 2), 0.0])
    pos, Z = [], []
    for ix in range(n_side):
        for iy in range(n_side):
            for iz in range(n_side):
                o = (np.array([ix, iy, iz]) + 0.5) * a
                q = rng.normal(size=4)
                q /= np.linalg.norm(q)
                w, x, y, z = q
                R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                              [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                              [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
                pos += [o, o + R @ h1, o + R @ h2]
                Z += [8, 1, 1]
    n = len(Z)
    cell = np.zeros((1, 9), np.float32)
    cell[0, [0, 4, 8]] = np.float32(L)
    return Structures(np.asarray(Z, np.int32), np.asarray(pos, np.float32), np.array([0, n], np.int32),
                      cell, np.ones(1, np.uint8), "water216")


def mix_box(n: int = 23558, L: float = 62.2, seed: int = 3,
            fractions=(0.50, 0.30, 0.08, 0.10, 0.0, 0.02, 0.0)) -> Structures:
    """Periodic mixture; species counts by largest remainder, shuffled; d_min 0.95 (min image)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = _counts_largest_remainder(n, fractions)
    Z = np.repeat(np.asarray(Z_TABLE, np.int32), counts)
    Z = Z[rng.permutation(n)]
    pos = _place_min_distance(rng, n, L, True)
    cell = np.zeros((1, 9), np.float32)
    cell[0, [0, 4, 8]] = np.float32(L)
    return Structures(Z, pos, np.array([0, n], np.int32), cell, np.ones(1, np.uint8), f"mix{n}")


def mix23558(seed: int = 3) -> Structures:
    """23,558 atoms (H 11,779, C 7,067, N 1,885, O 2,356, S 471) in a 62.2 A periodic cube."""
    return mix_box(23558, 62.2, seed)


def ragged_batch(n_mol: int = 4096, n_lo: int = 8, n_hi: int = 64, seed: int = 4) -> Structures:
    """n_mol gas-phase molecules with atom counts uniform in [n_lo, n_hi], species iid MIX7."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = rng.integers(n_lo, n_hi + 1, size=n_mol)
    parts = [random_molecule(rng, int(s), MIX7, False) for s in sizes]
    return concat(parts, f"batch{n_mol}")


def batch_targets(s: Structures, seed: int = 4):
    """Seeded regression targets: E* ~ N(0,1)*n_atoms per molecule, F* ~ N(0,1) per component."""
    rng = np.random.Generator(np.random.PCG64([seed, 7]))
    n = np.diff(s.mol_offsets).astype(np.float64)
    E = rng.normal(size=s.n_mol) * n
    F = rng.normal(size=(s.n_atoms, 3))
    return E, F


# ----------------------------------------------------------------------------- model parameters

@dataclasses.dataclass
class Weights:
    """Per-member, per-element network parameters (float32).

    W1 [M,7,256,1008] b1 [M,7,256]   W2 [M,7,192,256] b2 [M,7,192]
    W3 [M,7,160,192]  b3 [M,7,160]   w4 [M,7,160]     b4 [M,7]
    Row-major, W[out, in] (a layer computes z = W @ x + b).
    """
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray
    w4: np.ndarray
    b4: np.ndarray

    @property
    def n_members(self) -> int:
        return int(self.W1.shape[0])

    def member(self, m: int) -> "Weights":
        return Weights(*(getattr(self, f.name)[m:m + 1].copy() for f in dataclasses.fields(self)))


def xavier_weights(n_members: int, seed: int = 0, dims=LAYER_DIMS, n_elements: int = 7) -> Weights:
    """Seeded Xavier-uniform weights, W ~ U(+-sqrt(6/(fan_in+fan_out))), b ~ U(+-1/sqrt(fan_in)).

    Each (member, element, layer) draws from its own PCG64 stream keyed by
    (seed, member, element, layer), so member m of an M-member set equals member m
    of any larger set drawn with the same seed.
    """
    M, E = n_members, n_elements
    d = dims
    out = Weights(np.empty((M, E, d[1], d[0]), np.float32), np.empty((M, E, d[1]), np.float32),
                  np.empty((M, E, d[2], d[1]), np.float32), np.empty((M, E, d[2]), np.float32),
                  np.empty((M, E, d[3], d[2]), np.float32), np.empty((M, E, d[3]), np.float32),
                  np.empty((M, E, d[3]), np.float32), np.empty((M, E), np.float32))
    Ws = (out.W1, out.W2, out.W3, out.w4)
    bs = (out.b1, out.b2, out.b3, out.b4)
    for m in range(M):
        for e in range(E):
            for layer in range(4):
                fi, fo = d[layer], d[layer + 1]
                rng = np.random.Generator(np.random.PCG64([seed, m, e, layer]))
                lim = math.sqrt(6.0 / (fi + fo))
                W = rng.uniform(-lim, lim, size=(fo, fi))
                b = rng.uniform(-1.0 / math.sqrt(fi), 1.0 / math.sqrt(fi), size=fo)
                if layer < 3:
                    Ws[layer][m, e] = W
                    bs[layer][m, e] = b
                else:
                    Ws[3][m, e] = W[0]
                    bs[3][m, e] = b[0]
    return out


# ----------------------------------------------------------------------------- dynamics inputs

# masses (amu) in table order H C N O F S Cl
MASSES = (1.008, 12.011, 14.007, 15.999, 18.998, 32.06, 35.45)
KB_KCAL = 0.0019872041  # kcal/mol/K


def maxwell_boltzmann(Z: np.ndarray, T: float = 300.0, seed: int = 0) -> np.ndarray:
    """Seeded Maxwell-Boltzmann velocities in A/fs (kcal/mol, amu units), zero net momentum."""
    rng = np.random.Generator(np.random.PCG64([seed, 11]))
    m = np.asarray([MASSES[Z_TABLE.index(int(z))] for z in Z], np.float64)
    # kT/m in kcal/mol/amu -> (A/fs)^2 : 1 kcal/mol/amu = 4.184e-4 A^2/fs^2
    sigma = np.sqrt(KB_KCAL * T / m * 4.184e-4)
    v = rng.normal(size=(Z.shape[0], 3)) * sigma[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    return v.astype(np.float32)


@dataclasses.dataclass
class Request:
    arrival_s: float
    structure: Structures
    velocities: np.ndarray
    n_steps: int
    dt_fs: float


def request_sizes(rng: np.random.Generator, n: int, lo: int = 8, hi: int = 20000) -> np.ndarray:
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))).astype(np.int64)


def _pool_member(args) -> Structures:
    seed, k, n, pbc_above = args
    rng = np.random.Generator(np.random.PCG64([seed, 1, k]))
    return random_molecule(rng, int(n), MIX7, periodic=bool(n > pbc_above), name=f"req{k}")


def request_pool(n_pool: int = 4096, seed: int = 5, lo: int = 8, hi: int = 20000,
                 pbc_above: int = 500, workers: int = 1) -> list[Structures]:
    """Pool of request structures: log-uniform sizes, MIX7 composition, PBC above 500 atoms.  Structure k is
    drawn from its own stream (seed, 1, k), so the pool is the same whether it is built serially or by
    `workers` spawned processes."""
    rng = np.random.Generator(np.random.PCG64([seed, 1]))
    sizes = request_sizes(rng, n_pool, lo, hi)
    jobs = [(seed, k, int(n), pbc_above) for k, n in enumerate(sizes)]
    if workers <= 1:
        return [_pool_member(j) for j in jobs]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    # largest first, so the long placements start early; results come back in pool order
    order = sorted(range(len(jobs)), key=lambda k: -jobs[k][2])
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        built = list(ex.map(_pool_member, [jobs[k] for k in order], chunksize=8))
    out = [None] * len(jobs)
    for k, b in zip(order, built):
        out[k] = b
    return out


def poisson_stream(pool: list[Structures], rate_hz: float = 2000.0, duration_s: float = 60.0,
                   seed: int = 5, n_steps: int = 10, dt_fs: float = 0.5) -> list[Request]:
    """Open-loop Poisson arrivals drawing structures uniformly from the pool."""
    rng = np.random.Generator(np.random.PCG64([seed, 2]))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        k = int(rng.integers(len(pool)))
        s = pool[k]
        out.append(Request(t, s, maxwell_boltzmann(s.Z, 300.0, seed=len(out)), n_steps, dt_fs))
    return out
