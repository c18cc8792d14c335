"""Float64 CPU oracle for the ANI-style energy / force path (FeNNol, arXiv 2405.01491).

TEST INFRASTRUCTURE ONLY.  This package may be imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; the
product (``paper_2405_01491_b300``) never imports it, and it imports nothing
from the product.  The only inputs both sides share are the seeded arrays from
``paper_2405_01491_b300.synth`` (a module that holds none of the method's
arithmetic).

Layout:
  fnn_oracle.c   neighbour graph, AEV, AEV vector-Jacobian and Jacobian-vector
                 products, in plain C, float64, one loop per definition.
  this module    ctypes glue, the per-element networks and the energy / force /
                 virial / loss assembly in numpy float64 (matrix products are
                 the only library primitive used).

Paper passages followed:
  * neighbour graph and batching: section II.A (GraphGenerator, GraphFilter,
    GraphAngularExtension; concatenated batches with a batch index).
  * switching function (cosine) and radial Gaussian basis: sections II.A, II.B.
  * ANI AEV + species-dependent networks + per-structure energy sum and forces
    by differentiation: section II.E (ANI flow diagram) and section II.B
    (neural networks, ChemicalNet).
  * angular basis Theta_n = (1/2 + cos(theta - theta_n)/2)^zeta over unordered
    neighbour pairs {jk}: Appendix A (angular resources).
  * energy/force MSE loss with per-atom energy normalisation: section IV.
Readings of unstated details (ANI-2x constants, prefactors, 0.95 damping,
shift grids, slot order, CELU activation) are listed in the design notes.
Parity of every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(HERE, "fnn_oracle.c")

N_AEV = 1008
N_RAD = 112
ELEMENT_OF_Z = {1: 0, 6: 1, 7: 2, 8: 3, 9: 4, 16: 5, 17: 6}
CELU_ALPHA = 0.1


@dataclass(frozen=True)
class Params:
    """ANI-2x symmetry-function constants (the model the paper benchmarks, section V.E)."""
    rc_rad: float = 5.1
    rc_ang: float = 3.5
    eta_r: float = 19.7
    eta_a: float = 12.5
    zeta: float = 14.1
    shf_r0: float = 0.8
    shf_a0: float = 0.8
    switch: str = "cosine"   # switching function (section II.A): "cosine", "polynomial" or "exponential"
    switch_p: float = 6.0    # exponent of the polynomial envelope


SWITCH_KIND = {"cosine": 0, "polynomial": 1, "exponential": 2}


class _CParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("rc_rad", "rc_ang", "eta_r", "eta_a", "zeta", "shf_r0", "shf_a0",
                                               "sw_kind", "sw_p")]


class _CGraph(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("n_mol", ctypes.c_int32),
                ("mol_offsets", ctypes.c_void_p), ("Z", ctypes.c_void_p),
                ("pos", ctypes.c_void_p), ("cell", ctypes.c_void_p), ("pbc", ctypes.c_void_p),
                ("nnz", ctypes.c_int64), ("ei", ctypes.c_void_p), ("ej", ctypes.c_void_p),
                ("es", ctypes.c_void_p)]


def build(force: bool = False) -> str:
    """Compile fnn_oracle.c (gcc, -O2, OpenMP, no FP contraction) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_neighbors.restype = ctypes.c_int64
        _lib.oracle_neighbors.argtypes = [ctypes.c_int32, ctypes.c_int32] + [ctypes.c_void_p] * 4 + \
            [ctypes.c_double, ctypes.c_int64] + [ctypes.c_void_p] * 3
        for f in ("oracle_aev", "oracle_aev_vjp", "oracle_aev_jvp"):
            getattr(_lib, f).restype = ctypes.c_int
        _lib.oracle_aev.argtypes = [ctypes.c_void_p] * 3
        _lib.oracle_aev_vjp.argtypes = [ctypes.c_void_p] * 5
        _lib.oracle_aev_jvp.argtypes = [ctypes.c_void_p] * 4
        _lib.oracle_switch.restype = None
        _lib.oracle_switch.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                       ctypes.c_void_p]
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _sys_arrays(s):
    Z = np.ascontiguousarray(s.Z, np.int32)
    # float32 inputs widen exactly; float64 inputs (finite-difference pins) pass through
    pos = np.ascontiguousarray(s.pos, np.float64).reshape(-1, 3)
    mo = np.ascontiguousarray(s.mol_offsets, np.int32)
    cell = np.ascontiguousarray(s.cell, np.float64).reshape(-1, 9)
    pbc = np.ascontiguousarray(s.pbc, np.uint8)
    return Z, pos, mo, cell, pbc


class OracleError(RuntimeError):
    pass


def neighbors(s, R: float):
    """Directed pairs within R (section II.A): arrays i, j (int32) and shift n (int8 [nnz,3]), sorted by (i, j)."""
    Z, pos, mo, cell, pbc = _sys_arrays(s)
    L = lib()
    n = L.oracle_neighbors(s.n_atoms, s.n_mol, _p(mo), _p(pos), _p(cell), _p(pbc), float(R), 0, None, None, None)
    if n < 0:
        raise OracleError(f"oracle_neighbors failed with status {n}")
    ei = np.empty(n, np.int32)
    ej = np.empty(n, np.int32)
    es = np.empty((n, 3), np.int8)
    n2 = L.oracle_neighbors(s.n_atoms, s.n_mol, _p(mo), _p(pos), _p(cell), _p(pbc), float(R), n,
                            _p(ei), _p(ej), _p(es))
    assert n2 == n
    return ei, ej, es


class Graph:
    """The rc_rad neighbour graph of a structure batch, kept alive for the C calls."""

    def __init__(self, s, params: Params = Params()):
        self.s = s
        self.params = params
        self.arrays = _sys_arrays(s)
        self.ei, self.ej, self.es = neighbors(s, params.rc_rad)
        Z, pos, mo, cell, pbc = self.arrays
        self.c = _CGraph(s.n_atoms, s.n_mol, _p(mo), _p(Z), _p(pos), _p(cell), _p(pbc),
                         self.ei.shape[0], _p(self.ei), _p(self.ej), _p(self.es))
        self.cp = _c_params(params)


def _c_params(params: Params) -> _CParams:
    return _CParams(*(getattr(params, f) for f in ("rc_rad", "rc_ang", "eta_r", "eta_a", "zeta", "shf_r0", "shf_a0")),
                    float(SWITCH_KIND[params.switch]), float(params.switch_p))


def switch(r: float, rc: float, params: Params = Params()):
    """The switching function of params at distance r for cutoff rc: (value, derivative)."""
    f, df = ctypes.c_double(), ctypes.c_double()
    lib().oracle_switch(ctypes.byref(_c_params(params)), float(r), float(rc), ctypes.byref(f), ctypes.byref(df))
    return f.value, df.value


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def aev(s, params: Params = Params(), graph: Graph | None = None) -> np.ndarray:
    """AEV [N, 1008] float64: 112 radial slots (element-major, 16 shifts) + 28 x 32 angular slots."""
    g = graph or Graph(s, params)
    out = np.empty((s.n_atoms, N_AEV), np.float64)
    _check(lib().oracle_aev(ctypes.byref(g.c), ctypes.byref(g.cp), _p(out)), "oracle_aev")
    return out


def aev_vjp(s, G: np.ndarray, params: Params = Params(), graph: Graph | None = None):
    """dE/dx [N,3] and virial [n_mol,3,3] from G = dE/dAEV [N,1008]."""
    g = graph or Graph(s, params)
    G = np.ascontiguousarray(G, np.float64)
    grad = np.empty((s.n_atoms, 3), np.float64)
    vir = np.empty((s.n_mol, 3, 3), np.float64)
    _check(lib().oracle_aev_vjp(ctypes.byref(g.c), ctypes.byref(g.cp), _p(G), _p(grad), _p(vir)), "oracle_aev_vjp")
    return grad, vir


def aev_jvp(s, V: np.ndarray, params: Params = Params(), graph: Graph | None = None) -> np.ndarray:
    """Directional derivative of the AEV [N,1008] along the displacement field V [N,3]."""
    g = graph or Graph(s, params)
    V = np.ascontiguousarray(V, np.float64)
    out = np.empty((s.n_atoms, N_AEV), np.float64)
    _check(lib().oracle_aev_jvp(ctypes.byref(g.c), ctypes.byref(g.cp), _p(V), _p(out)), "oracle_aev_jvp")
    return out


# ----------------------------------------------------------------------------- networks (numpy, float64)

def celu(z, a=CELU_ALPHA):
    """CELU(z) = z for z > 0, a (exp(z/a) - 1) otherwise."""
    return np.where(z > 0, z, a * np.expm1(np.minimum(z, 0.0) / a))


def dcelu(z, a=CELU_ALPHA):
    return np.where(z > 0, 1.0, np.exp(np.minimum(z, 0.0) / a))


def d2celu(z, a=CELU_ALPHA):
    return np.where(z > 0, 0.0, np.exp(np.minimum(z, 0.0) / a) / a)


def elements(Z) -> np.ndarray:
    try:
        return np.asarray([ELEMENT_OF_Z[int(z)] for z in Z], np.int64)
    except KeyError as exc:
        raise OracleError(f"species outside the element table: {exc}") from None


def _layers(w, m, e):
    f64 = lambda a: np.asarray(a, np.float64)
    return (f64(w.W1[m, e]), f64(w.b1[m, e]), f64(w.W2[m, e]), f64(w.b2[m, e]),
            f64(w.W3[m, e]), f64(w.b3[m, e]), f64(w.w4[m, e]), float(w.b4[m, e]))


def network_energies(A: np.ndarray, Z, w):
    """Atomic outputs y [N, M] of the per-element networks 1008-256-192-160-1 (CELU, linear output),
    and dY/dAEV averaged over members: G [N, 1008] = (1/M) sum_m dy_m/daev."""
    el = elements(Z)
    N, M = A.shape[0], w.n_members
    y = np.zeros((N, M))
    G = np.zeros((N, N_AEV))
    for e in range(7):
        rows = np.nonzero(el == e)[0]
        if rows.size == 0:
            continue
        x = A[rows]
        for m in range(M):
            W1, b1, W2, b2, W3, b3, w4, b4 = _layers(w, m, e)
            z1 = x @ W1.T + b1
            h1 = celu(z1)
            z2 = h1 @ W2.T + b2
            h2 = celu(z2)
            z3 = h2 @ W3.T + b3
            h3 = celu(z3)
            y[rows, m] = h3 @ w4 + b4
            g3 = w4[None, :] * dcelu(z3)
            g2 = (g3 @ W3) * dcelu(z2)
            g1 = (g2 @ W2) * dcelu(z1)
            G[rows] += (g1 @ W1) / M
    return y, G


@dataclass
class Result:
    energy: np.ndarray      # [n_mol] float64
    forces: np.ndarray      # [N, 3]
    virial: np.ndarray      # [n_mol, 3, 3]
    atomic: np.ndarray      # [N] member-averaged atomic energies
    aev: np.ndarray         # [N, 1008]


def energy_forces(s, w, params: Params = Params()) -> Result:
    """E_mol = (1/M) sum_m sum_{i in mol} y_im; F = -dE/dx; virial = -sum_edges d (x) dE/dd (section II.E, V.A)."""
    g = Graph(s, params)
    A = aev(s, params, g)
    y, G = network_energies(A, s.Z, w)
    e_atom = y.mean(axis=1)
    mol = np.repeat(np.arange(s.n_mol), np.diff(s.mol_offsets))
    E = np.zeros(s.n_mol)
    np.add.at(E, mol, e_atom)
    grad, vir = aev_vjp(s, G, params, g)
    return Result(E, -grad, vir, e_atom, A)


# ----------------------------------------------------------------------------- training loss (section IV)

FORCE_WEIGHT = 0.99
ENERGY_WEIGHT = 0.01


def loss_and_weight_grads(s, w, E_ref: np.ndarray, F_ref: np.ndarray, params: Params = Params()):
    """L = 0.99 mean_{i,c} (F - F*)^2 + 0.01 mean_mol ((E - E*) / n_mol)^2 and dL/dtheta.

    The networks are differentiated with float64 torch autograd on the CPU (a
    library primitive); the AEV enters through the oracle's own Jacobian-vector
    product: dL_F/dtheta = d/dtheta <-J_aev v, dE/dAEV(theta)>, v = dL/dF.
    Returns (L, E, F, grads) with grads a dict of arrays shaped like the weights.
    """
    import torch

    g = Graph(s, params)
    A = aev(s, params, g)
    el = elements(s.Z)
    N, M = s.n_atoms, w.n_members
    names = ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")
    th = {k: torch.tensor(np.asarray(getattr(w, k), np.float64), requires_grad=True) for k in names}
    At = torch.tensor(A, requires_grad=True)
    y = torch.zeros((N, M), dtype=torch.float64)
    ys = []
    for e in range(7):
        rows = np.nonzero(el == e)[0]
        if rows.size == 0:
            continue
        x = At[rows]
        for m in range(M):
            # CELU from elementary ops (torch's fused CELU backward carries alpha in single precision)
            cel = lambda z: torch.where(z > 0, z, CELU_ALPHA * torch.expm1(torch.clamp(z, max=0.0) / CELU_ALPHA))
            h = cel(x @ th["W1"][m, e].T + th["b1"][m, e])
            h = cel(h @ th["W2"][m, e].T + th["b2"][m, e])
            h = cel(h @ th["W3"][m, e].T + th["b3"][m, e])
            ys.append((rows, m, h @ th["w4"][m, e] + th["b4"][m, e]))
    for rows, m, v in ys:
        y = y.index_put((torch.as_tensor(rows), torch.full((rows.size,), m)), v)
    e_atom = y.mean(dim=1)
    mol = torch.as_tensor(np.repeat(np.arange(s.n_mol), np.diff(s.mol_offsets)))
    E = torch.zeros(s.n_mol, dtype=torch.float64).index_add(0, mol, e_atom)
    G = torch.autograd.grad(E.sum(), At, create_graph=True)[0]           # dE/dAEV(theta)
    grad_x, _ = aev_vjp(s, G.detach().numpy(), params, g)
    F = -grad_x
    n_mol_atoms = np.diff(s.mol_offsets).astype(np.float64)
    LF = FORCE_WEIGHT * np.mean((F - F_ref) ** 2)
    LE_t = ENERGY_WEIGHT * torch.mean(((E - torch.as_tensor(E_ref)) / torch.as_tensor(n_mol_atoms)) ** 2)
    v = FORCE_WEIGHT * 2.0 * (F - F_ref) / F.size                        # dL/dF
    t = aev_jvp(s, v, params, g)                                         # J_aev v
    surrogate = LE_t + torch.sum(torch.as_tensor(-t) * G)                # d/dtheta of this = dL/dtheta
    gr = torch.autograd.grad(surrogate, [th[k] for k in names])
    L = float(LE_t.detach()) + LF
    return L, E.detach().numpy(), F, {k: gk.numpy() for k, gk in zip(names, gr)}


def celu_kink_deltas(s, w, E_ref: np.ndarray, F_ref: np.ndarray, band: float = 2e-5,
                     params: Params = Params()):
    """Pre-activations at the CELU kink and what each does to dL/dtheta.

    The force term of the loss (section IV) differentiates dE/dAEV once more, so its parameter
    gradient holds CELU''(z), which is 0 for z > 0 and exp(z/alpha)/alpha below: a jump of
    1/alpha at z = 0.  An evaluation whose pre-activation z is within its rounding error of 0
    may take either side, and both results are gradients of the loss (one-sided limits).
    For every pre-activation with |z| <= band * (sum_j |W_uj h_j| + |b_u|) this returns
    (m, e, layer, atom, unit, deltas): deltas[name] [shape of the weight's (m, e) block] is the
    change of the gradient when that one entry takes the other side.  With zd the tangent of z along
    J dL/dF and gb = d(-<J dL/dF, dE/dAEV>)/dhd at the entry, the other side changes
    dL/dz there by -/+ (1/alpha) CELU'(z) zd gb (minus when z <= 0: the term leaves); that
    change flows down the layers below through W^T and CELU' alone (linear in it)."""
    g = Graph(s, params)
    r = energy_forces(s, w, params)
    v = FORCE_WEIGHT * 2.0 * (r.forces - F_ref) / r.forces.size
    T = aev_jvp(s, v, params, g)
    A = r.aev
    el = elements(s.Z)
    M = w.n_members
    out = []
    for e in range(7):
        rows = np.nonzero(el == e)[0]
        if rows.size == 0:
            continue
        for m in range(M):
            W1, b1, W2, b2, W3, b3, w4, _ = _layers(w, m, e)
            Ws, bs = (W1, W2, W3), (b1, b2, b3)
            h, hd, z, mag = [A[rows]], [T[rows]], [], []
            for W, b in zip(Ws, bs):
                zl = h[-1] @ W.T + b
                z.append(zl)
                mag.append(np.abs(h[-1]) @ np.abs(W).T + np.abs(b))
                hd.append(dcelu(zl) * (hd[-1] @ W.T))
                h.append(celu(zl))
            # gb_l = dPhi/dhd_l, Phi's tangent part -<t, G> = -(1/M) sum w4 . hd_3
            gb = [None, None, None]
            gb[2] = np.broadcast_to(-w4 / M, hd[3].shape)
            gb[1] = (dcelu(z[2]) * gb[2]) @ W3
            gb[0] = (dcelu(z[1]) * gb[1]) @ W2
            for l in range(3):
                rr, uu = np.nonzero(np.abs(z[l]) <= band * mag[l])
                for ri, u in zip(rr, uu):
                    zv = z[l][ri, u]
                    d_gz = (1.0 if zv > 0 else -1.0) / CELU_ALPHA * hd[l + 1][ri, u] * gb[l][ri, u]
                    deltas = {k: np.zeros(np.shape(getattr(w, k))[2:]) for k in ("W1", "b1", "W2", "b2", "W3",
                                                                                 "b3", "w4", "b4")}
                    gz = np.zeros(Ws[l].shape[0])
                    gz[u] = d_gz
                    for k in range(l, -1, -1):
                        deltas[f"W{k + 1}"] += np.outer(gz, h[k][ri])
                        deltas[f"b{k + 1}"] += gz
                        if k > 0:
                            gz = dcelu(z[k - 1][ri]) * (gz @ Ws[k])
                    out.append((m, e, l + 1, int(rows[ri]), int(u), deltas))
    return out


# ----------------------------------------------------------------------------- dynamics (section V.D)

# atomic masses (amu), element order H C N O F S Cl
MASS = {0: 1.008, 1: 12.011, 2: 14.007, 3: 15.999, 4: 18.998, 5: 32.06, 6: 35.45}
ACCEL = 4.184e-4   # (kcal/mol/A) / amu in A/fs^2


def velocity_verlet(s, w, v0, n_steps: int, dt: float, params: Params = Params()):
    """NVE velocity Verlet, the integrator of the paper's native MD engine for NVE runs (section V.D):
    n_steps force evaluations at x_0 .. x_{n-1}; between evaluations
    v <- v + a dt/2, x <- x + v dt, then after the next evaluation v <- v + a dt/2.
    Returns (energies [n_steps, n_mol], final positions, final velocities v_{n-1}, final forces)."""
    el = elements(s.Z)
    m = np.asarray([MASS[int(e)] for e in el])[:, None]
    x = np.asarray(s.pos, np.float64).copy()
    v = np.asarray(v0, np.float64).copy()
    energies = []
    F = None
    for k in range(n_steps):
        st = type(s)(s.Z, x, s.mol_offsets, s.cell, s.pbc)
        r = energy_forces(st, w, params)
        energies.append(r.energy)
        a = r.forces / m * ACCEL
        if k > 0:
            v = v + 0.5 * dt * a          # completes the previous step's velocity
        F = r.forces
        if k < n_steps - 1:
            v = v + 0.5 * dt * a
            x = x + dt * v
    return np.asarray(energies), x, v, F


# ---------------------------------------------------------------------------------------------- Langevin
KB_KCAL = 0.0019872041   # Boltzmann constant, kcal/mol/K


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox-4x32-10, the counter-based generator of Salmon, Moraes, Dror and Shaw (SC 2011): ten rounds,
    each forming the two 64-bit products of counter words 0 and 2 with the multipliers 0xD2511F53 and
    0xCD9E8D57 and mixing their halves with words 1, 3 and the round key; the key advances between rounds
    by the Weyl constants 0x9E3779B9 and 0xBB67AE85.  ctr: uint32 [n, 4]; key: two uint32 words."""
    c = np.asarray(ctr, np.uint64).copy()
    k0, k1 = np.uint64(int(key[0]) & 0xffffffff), np.uint64(int(key[1]) & 0xffffffff)
    mask = np.uint64(0xffffffff)
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(0x9E3779B9)) & mask
            k1 = (k1 + np.uint64(0xBB67AE85)) & mask
        p0 = c[:, 0] * np.uint64(0xD2511F53)
        p1 = c[:, 2] * np.uint64(0xCD9E8D57)
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c = np.stack([hi1 ^ c[:, 1] ^ k0, lo1, hi0 ^ c[:, 3] ^ k1, lo0], axis=1)
    return c.astype(np.uint32)


def langevin_noise(n_atoms: int, t: int, seed: int) -> np.ndarray:
    """Three standard normal numbers per atom for noise step t: the Philox block of counter
    (atom, t mod 2^32, t >> 32, 0) and key (seed mod 2^32, seed >> 32), each word w turned into
    u = (floor(w / 256) + 1/2) / 2^24 in (0, 1), then the Box-Muller transform of (u0, u1) and (u2, u3)
    (the sine of the second pair unused).  Returns float64 [n_atoms, 3]."""
    ctr = np.zeros((n_atoms, 4), np.uint64)
    ctr[:, 0] = np.arange(n_atoms)
    ctr[:, 1] = t & 0xffffffff
    ctr[:, 2] = (t >> 32) & 0xffffffff
    w = philox4x32_10(ctr, (seed & 0xffffffff, (seed >> 32) & 0xffffffff)).astype(np.float64)
    u = (np.floor(w / 256.0) + 0.5) / 2.0 ** 24
    r0 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r1 = np.sqrt(-2.0 * np.log(u[:, 2]))
    return np.stack([r0 * np.cos(2 * np.pi * u[:, 1]), r0 * np.sin(2 * np.pi * u[:, 1]),
                     r1 * np.cos(2 * np.pi * u[:, 3])], axis=1)


def kinetic_energies(s, v) -> np.ndarray:
    """Per-structure kinetic energy sum_i m_i |v_i|^2 / 2 in kcal/mol (v in A/fs, masses in amu)."""
    m = np.asarray([MASS[int(e)] for e in elements(s.Z)])
    ke = 0.5 * m * np.sum(np.asarray(v, np.float64) ** 2, axis=1) / ACCEL
    off = np.asarray(s.mol_offsets)
    return np.array([ke[off[i]:off[i + 1]].sum() for i in range(len(off) - 1)])


def langevin_baoab(s, w, v0, n_steps: int, dt: float, temperature: float, gamma: float, seed: int,
                   step0: int = 0, params: Params = Params()):
    """Langevin dynamics by the BAOAB splitting (Leimkuhler and Matthews 2013), the integrator of the paper's
    native engine for Langevin runs (section V.D).  n_steps force evaluations at x_0 .. x_{n-1}; after
    evaluation k: B (v += a dt/2, completing step k-1 when k > 0), then, unless k is the last: B, A
    (x += v dt/2), O (v = c1 v + c2 sqrt(kB T / m) xi with c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2), xi
    from langevin_noise at noise step step0 + k), A.  gamma = 0 is velocity Verlet.
    Returns (potential energies [n, n_mol], kinetic energies of v_k [n, n_mol], final x, final v, final F)."""
    el = elements(s.Z)
    m = np.asarray([MASS[int(e)] for e in el])[:, None]
    x = np.asarray(s.pos, np.float64).copy()
    v = np.asarray(v0, np.float64).copy()
    c1 = np.exp(-gamma * dt)
    c2 = np.sqrt(1.0 - c1 * c1)
    sig = np.sqrt(KB_KCAL * temperature * ACCEL / m)
    energies, kinetic = [], []
    F = None
    for k in range(n_steps):
        st = type(s)(s.Z, x, s.mol_offsets, s.cell, s.pbc)
        r = energy_forces(st, w, params)
        energies.append(r.energy)
        a = r.forces / m * ACCEL
        if k > 0:
            v = v + 0.5 * dt * a
        kinetic.append(kinetic_energies(s, v))
        F = r.forces
        if k < n_steps - 1:
            v = v + 0.5 * dt * a
            x = x + 0.5 * dt * v
            v = c1 * v + c2 * sig * langevin_noise(s.n_atoms, step0 + k, seed)
            x = x + 0.5 * dt * v
    return np.asarray(energies), np.asarray(kinetic), x, v, F


# ------------------------------------------------------------------------- CRATE angular resource (App. A)
CRATE_NB = 8       # triplet radial basis functions B~_a
CRATE_DA = 32      # channels d_a of D_ij
CRATE_NT = 4       # angular basis functions Theta_n = cos(n theta), n = 0..3


def _switch_torch(r, rc, params: Params):
    """The switching function of params (section II.A) in torch float64, for the autograd of the CRATE
    resource; it is compared point by point with the C oracle's switch in the pins."""
    import torch
    inside = r < rc
    rr = torch.where(inside, r, torch.zeros_like(r))
    if params.switch == "polynomial":
        p, d = params.switch_p, rr / rc
        f = 1 - 0.5 * (p + 1) * (p + 2) * d ** p + p * (p + 2) * d ** (p + 1) - 0.5 * p * (p + 1) * d ** (p + 2)
    elif params.switch == "exponential":
        f = torch.exp(-rr * rr / ((rc - rr) * (rc + rr)))
    else:
        f = 0.5 * torch.cos(np.pi * rr / rc) + 0.5
    return torch.where(inside, f, torch.zeros_like(f))


def crate_triplets(ei: np.ndarray):
    """Unordered pairs {p, q}, p < q, of the directed edges that share their centre atom (edges sorted by
    centre): the triplets (i, j, k) of Appendix A's sum over {jk}."""
    P, Q = [], []
    starts = np.flatnonzero(np.r_[True, ei[1:] != ei[:-1]]) if len(ei) else np.zeros(0, np.int64)
    ends = np.r_[starts[1:], len(ei)]
    for a, b in zip(starts, ends):
        p, q = np.triu_indices(b - a, 1)
        P.append(p + a)
        Q.append(q + a)
    if not P:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(P).astype(np.int64), np.concatenate(Q).astype(np.int64)


def crate_angular(s, V, params: Params = Params(), G=None):
    """The angular resource of CRATE's first interaction layer (Appendix A, angular resources):
        D_ij[c] = f~(r_ij) sum_a B~_a(r_ij) V[e(j), a, c],   B~_a(r) = exp(-eta_a (r - A_a)^2),
        g_i[n, c] = sum_{j<k} Theta_n(theta_jik) D_ij[c] D_ik[c],   Theta_n = cos(n theta),
    over neighbours within rc_ang (the triplet cutoff), A_a = shf_a0 + a (rc_ang - shf_a0) / 8, f~ the switch
    at rc_ang.  The neighbour embedding depends on the neighbour's element only (layer 1), so the product of
    the species table and the trainable tensor W_ang enters as one tensor V [7, 8, 32].  cos(n theta) is
    evaluated as the Chebyshev polynomial T_n(cos theta) (equal for every theta, smooth at 0 and pi).
    Returns g [N, 4, 32]; with G = dL/dg given, also (dL/dx [N, 3], dL/dV [7, 8, 32]) by float64 autograd."""
    import torch
    Z, pos, mo, cell, pbc = _sys_arrays(s)
    ei, ej, es = neighbors(s, params.rc_ang)
    x = torch.tensor(pos, dtype=torch.float64, requires_grad=G is not None)
    Vt = torch.tensor(np.asarray(V, np.float64), requires_grad=G is not None)
    mol = np.repeat(np.arange(s.n_mol), np.diff(mo))
    L = np.zeros((s.n_atoms, 3))
    for m in range(s.n_mol):
        if pbc[m]:
            L[mo[m]:mo[m + 1]] = cell[m, [0, 4, 8]]
    sh = torch.tensor(es.astype(np.float64) * L[ei], dtype=torch.float64)
    d = x[torch.from_numpy(ej.astype(np.int64))] - x[torch.from_numpy(ei.astype(np.int64))] + sh
    r = torch.sqrt((d * d).sum(1))
    shifts = torch.tensor(params.shf_a0 + np.arange(CRATE_NB) * (params.rc_ang - params.shf_a0) / CRATE_NB)
    B = torch.exp(-params.eta_a * (r[:, None] - shifts[None, :]) ** 2)
    el = torch.from_numpy(elements(Z)[ej].astype(np.int64))
    D = _switch_torch(r, params.rc_ang, params)[:, None] * torch.einsum("pa,pac->pc", B, Vt[el])
    p, q = crate_triplets(ei)
    p, q = torch.from_numpy(p), torch.from_numpy(q)
    c = (d[p] * d[q]).sum(1) / (r[p] * r[q])
    T = torch.stack([torch.ones_like(c), c, 2 * c * c - 1, (4 * c * c - 3) * c], 1)
    g = torch.zeros((s.n_atoms, CRATE_NT, CRATE_DA), dtype=torch.float64)
    g = g.index_add(0, torch.from_numpy(ei.astype(np.int64))[p], T[:, :, None] * (D[p] * D[q])[:, None, :])
    if G is None:
        return g.detach().numpy()
    gx, gV = torch.autograd.grad(g, (x, Vt), grad_outputs=torch.tensor(np.asarray(G, np.float64)),
                                 allow_unused=True)
    gx = torch.zeros_like(x) if gx is None else gx
    gV = torch.zeros_like(Vt) if gV is None else gV
    return g.detach().numpy(), gx.numpy(), gV.numpy()


# -------------------------------------------------------------------------------- RPMD (section V.D)
HBAR_KCAL_FS = 15.178736   # reduced Planck constant in kcal/mol fs (1.054571817e-34 J s, N_A, 4184 J/kcal)


def rpmd_normal_modes(P: int):
    """Orthogonal matrix C [bead j, mode k] of the free ring polymer (real Fourier basis): k = 0 the centroid
    1/sqrt(P); 0 < k < P/2 sqrt(2/P) cos(2 pi j k / P); k = P/2 (-1)^j / sqrt(P); P/2 < k sqrt(2/P) sin(2 pi j k / P).
    Returns C and the mode frequencies in units of omega_P: 2 sin(k pi / P)."""
    j = np.arange(P)[:, None]
    k = np.arange(P)[None, :]
    C = np.where(k == 0, 1.0 / np.sqrt(P), 0.0)
    C = C + np.where((k > 0) & (2 * k < P), np.sqrt(2.0 / P) * np.cos(2 * np.pi * j * k / P), 0.0)
    C = C + np.where((2 * k == P), (-1.0) ** j / np.sqrt(P), 0.0)
    C = C + np.where(2 * k > P, np.sqrt(2.0 / P) * np.sin(2 * np.pi * j * k / P), 0.0)
    return C, 2.0 * np.sin(np.arange(P) * np.pi / P)


def rpmd(s, w, P: int, x0, v0, n_steps: int, dt: float, temperature: float, params: Params = Params()):
    """Ring-polymer molecular dynamics (Habershon et al. 2013; the paper's NQE method of section V.D): P replicas
    (beads) of the structure s, bead b's positions x[b] and velocities v[b] ([P, N, 3]); the physical forces of
    all beads from one batched evaluation (the beads as P structures of one batch), and the free ring polymer,
    whose springs 1/2 m omega_P^2 |x_b - x_(b+1)|^2 (omega_P = P kB T / hbar) couple neighbouring beads, propagated
    exactly in its normal modes.  After evaluation k: v += a dt/2 (completing step k-1 when k > 0; then the
    Hamiltonian of the ring polymer at step k is recorded), and unless k is the last: v += a dt/2, then each mode
    q~_k = sum_j C_jk x_j evolves for dt as a harmonic oscillator of frequency omega_P 2 sin(k pi / P) (the centroid
    freely).  Returns (bead potential energies [n_steps, P], Hamiltonian [n_steps], x, v, F [P, N, 3])."""
    el = elements(s.Z)
    m = np.asarray([MASS[int(e)] for e in el])[None, :, None]
    N = s.n_atoms
    x = np.asarray(x0, np.float64).reshape(P, N, 3).copy()
    v = np.asarray(v0, np.float64).reshape(P, N, 3).copy()
    C, wk = rpmd_normal_modes(P)
    wP = P * KB_KCAL * temperature / HBAR_KCAL_FS
    om = wk * wP
    batch = lambda xx: type(s)(np.tile(s.Z, P), xx.reshape(P * N, 3), np.arange(P + 1, dtype=np.int32) * N,
                               np.repeat(np.asarray(s.cell, np.float64).reshape(1, 9), P, 0), np.repeat(s.pbc, P))
    energies, hamilton = [], []
    F = None
    for k in range(n_steps):
        r = energy_forces(batch(x), w, params)
        energies.append(r.energy.copy())
        F = r.forces.reshape(P, N, 3)
        a = F / m * ACCEL
        if k > 0:
            v = v + 0.5 * dt * a
        kin = 0.5 * np.sum(m * v * v) / ACCEL
        spring = 0.5 * np.sum(m * (wP ** 2) * (x - np.roll(x, -1, axis=0)) ** 2) / ACCEL
        hamilton.append(kin + spring + r.energy.sum())
        if k < n_steps - 1:
            v = v + 0.5 * dt * a
            q = np.einsum("jk,jnc->knc", C, x)
            p = np.einsum("jk,jnc->knc", C, v)
            qn, pn = q.copy(), p.copy()
            for kk in range(P):
                if om[kk] == 0.0:
                    qn[kk] = q[kk] + dt * p[kk]
                else:
                    cs, sn = np.cos(om[kk] * dt), np.sin(om[kk] * dt)
                    qn[kk] = cs * q[kk] + sn / om[kk] * p[kk]
                    pn[kk] = -om[kk] * sn * q[kk] + cs * p[kk]
            x = np.einsum("jk,knc->jnc", C, qn)
            v = np.einsum("jk,knc->jnc", C, pn)
    return np.asarray(energies), np.asarray(hamilton), x, v, F
