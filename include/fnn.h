/*
 * fnn.h -- C ABI of the B300 (sm_103a) ANI-style energy / force library.
 *
 * The operation (FeNNol, arXiv 2405.01491, section II.E and Fig. ani_diagram):
 * species (atomic numbers) and coordinates of a batch of concatenated
 * structures, with a per-structure atom count and optional periodic cell
 * (section II.A), go in; per-structure energies, per-atom forces and
 * per-structure virials come out (the energy_and_forces_and_virial call of
 * section V.A).  Inside: cell-list neighbour search (the O(N) replacement of
 * the all-pairs GraphGenerator, section II.A / V.E), ANI radial + angular
 * AEVs (sections II.B, II.E, Appendix A), per-element networks
 * 1008-256-192-160-1 with CELU (section II.B, ChemicalNet), the per-structure
 * energy sum, and the analytic adjoint F = -dE/dx (the paper uses jax.grad).
 *
 * Conventions shared by every call:
 *   - Units: A, kcal/mol, kcal/mol/A.
 *   - Every array argument is owned by the caller; opaque handles are owned
 *     by the library and released by their *_destroy call.
 *   - "device" pointers are CUDA global-memory pointers on the context's
 *     device; "host" pointers are ordinary (pinned or pageable) host memory.
 *   - A stream argument is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Calls that take a stream are asynchronous and
 *     stream-ordered: argument errors are returned at once, while conditions
 *     detected by the kernels (bad species, too-small cell, capacity
 *     overflow, non-finite results) are posted to a sticky per-context status
 *     that fnn_sync() returns and clears.  Results written by a call whose
 *     kernels posted an error are unspecified.
 *   - Batches: atoms of structure m are [mol_offsets[m], mol_offsets[m+1]);
 *     structures never interact (section II.A batch index).
 *   - Periodic structures use the minimum image convention, orthorhombic
 *     cells only, every edge longer than 2 * (rc_rad + skin).
 *   - Elements: H C N O F S Cl (Z = 1 6 7 8 9 16 17), AEV length 1008
 *     (112 radial: element-major x 16 shifts; 896 angular: 28 element pairs
 *     x 8 radial shifts x 4 angle sections).  These sizes are compiled in.
 *   - Per-atom limits of the AEV kernels: at most 160 neighbours within
 *     rc_rad and 64 within rc_ang (FNN_E_CAPACITY, info = -(atom + 1)).
 */
#ifndef FNN_H
#define FNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fnn_ctx fnn_ctx;
typedef struct fnn_nlist fnn_nlist;

typedef enum {
  FNN_OK = 0,
  FNN_PENDING = 1,
  FNN_E_INVALID = -1,   /* bad argument (NULL, negative size, inconsistent offsets) */
  FNN_E_SPECIES = -2,   /* atomic number outside the element table; info = atom */
  FNN_E_CELL = -3,      /* periodic cell not orthorhombic or an edge <= 2 (rc_rad + skin); info = structure */
  FNN_E_CAPACITY = -4,  /* neighbour list larger than its capacity; info = entries needed */
  FNN_E_OOM = -5,       /* device allocation failed */
  FNN_E_TIMEOUT = -6,   /* a bounded device wait gave up */
  FNN_E_NONFINITE = -7, /* non-finite coordinate (info = atom) or energy (info = -(structure + 1)) */
  FNN_E_CUDA = -8,      /* a CUDA runtime call failed; see fnn_last_error */
  FNN_E_STATE = -9      /* call out of order (e.g. no weights loaded) */
} fnn_status;

typedef enum {
  FNN_FP32 = 0, /* network GEMMs in FP32 (SIMT FFMA), FP32 accumulation */
  FNN_BF16 = 1, /* network GEMMs in BF16 on tcgen05 tensor cores, FP32 accumulation */
  FNN_FP8 = 2,  /* network GEMMs in FP8 e4m3 with per-layer scales, FP32 accumulation */
  FNN_FP32X3 = 3, /* FP32-accurate network GEMMs on tcgen05 tensor cores: every operand split into
                    bf16 hi + lo, products hi*hi + hi*lo + lo*hi accumulated in FP32 (relative error
                    of a product about 2^-16, within the FP32 tolerances of the energies and forces) */
  FNN_BF16_FUSED = 4 /* the FNN_BF16 arithmetic with the AEV and the first layer in one kernel (section
                    II.E): each 64-row tile of species-sorted AEV rows is built in shared memory as bf16 and
                    is the A operand of the first layer's tcgen05 products; the AEV never reaches global
                    memory.  Energies and forces equal FNN_BF16's up to the order of FP32 sums. */
} fnn_precision;

/* Symmetry-function constants and ensemble size.  fnn_config_default() fills
 * the ANI-2x values of the paper's benchmark model (section V.E). */
typedef struct {
  double rc_rad;      /* radial cutoff, A (5.1) */
  double rc_ang;      /* angular cutoff, A (3.5) */
  double eta_rad;     /* radial Gaussian width, 1/A^2 (19.7) */
  double eta_ang;     /* angular radial Gaussian width, 1/A^2 (12.5) */
  double zeta;        /* angular exponent (14.1) */
  double shift_rad0;  /* first radial shift, A (0.8); shifts are shift_rad0 + k (rc_rad - shift_rad0) / 16 */
  double shift_ang0;  /* first angular radial shift, A (0.8); shifts shift_ang0 + m (rc_ang - shift_ang0) / 8 */
  double skin;        /* neighbour-list skin, A; list radius = rc_rad + skin (0 = exact list) */
  int32_t n_members;  /* ensemble size M, 1..8; the energy is the member average */
  int32_t switch_kind;/* switching function of both cutoffs (section II.A), fnn_switch; 0 = cosine */
  double switch_p;    /* exponent p of the polynomial envelope (> 0; 6 by default) */
} fnn_config;

/* Switching functions f(r) for r < rc (0 from rc on), d = r / rc (section II.A processing modules):
 *   FNN_SWITCH_COSINE       cos(pi d) / 2 + 1/2                                   (ANI)
 *   FNN_SWITCH_POLYNOMIAL   1 - (p+1)(p+2)/2 d^p + p(p+2) d^(p+1) - p(p+1)/2 d^(p+2)  (Gasteiger et al. 2020)
 *   FNN_SWITCH_EXPONENTIAL  exp(-r^2 / ((rc - r)(rc + r)))                        (SpookyNet) */
typedef enum { FNN_SWITCH_COSINE = 0, FNN_SWITCH_POLYNOMIAL = 1, FNN_SWITCH_EXPONENTIAL = 2 } fnn_switch;

/* Network parameters, float32, host memory, row-major W[out][in]:
 * W1 [M][7][256][1008], b1 [M][7][256], W2 [M][7][192][256], b2 [M][7][192],
 * W3 [M][7][160][192], b3 [M][7][160], w4 [M][7][160], b4 [M][7]. */
typedef struct {
  int32_t n_members;
  const float *W1, *b1, *W2, *b2, *W3, *b3, *w4, *b4;
} fnn_weights;

/* A batch of structures, all device pointers, caller-owned. */
typedef struct {
  int32_t n_atoms;            /* N >= 0 */
  int32_t n_mol;              /* >= 1 */
  const int32_t *mol_offsets; /* [n_mol + 1], mol_offsets[0] = 0, non-decreasing, last = N */
  const int32_t *Z;           /* [N] atomic numbers */
  const float *pos;           /* [N][4] x, y, z, (w ignored), A; 16-byte aligned */
  const float *cell;          /* [n_mol][9] row vectors, or NULL when no structure is periodic */
  const uint8_t *pbc;         /* [n_mol] 1 = periodic, or NULL = none periodic */
} fnn_system;

/* Fill *cfg with the ANI-2x constants, skin 0, M = 1 and the cosine switch (p = 6). */
void fnn_config_default(fnn_config *cfg);

/* Create a context on the current CUDA device.  Returns FNN_E_INVALID for
 * out-of-range constants (cutoffs <= 0, rc_ang > rc_rad, M outside 1..8, an unknown
 * switch_kind, switch_p <= 0). */
fnn_status fnn_create(fnn_ctx **ctx, const fnn_config *cfg);
fnn_status fnn_destroy(fnn_ctx *ctx);

/* Copy network parameters to the device (and derive the transposed, BF16 and
 * FP8 forms).  Exactly one of path (a file written by the Python binding's
 * save_weights: magic "FNNW", int32 version 1, int32 M, then the eight float32
 * arrays in the order above, little-endian) and host is non-NULL.
 * host->n_members must equal the context's M.  Synchronous. */
fnn_status fnn_load_weights(fnn_ctx *ctx, const char *path, const fnn_weights *host);

/* Neighbour-list handle.  capacity = number of directed entries it can hold
 * (0 = size from the first system: 160 entries per atom). */
fnn_status fnn_nlist_create(fnn_ctx *ctx, fnn_nlist **nl, int64_t capacity);
fnn_status fnn_nlist_destroy(fnn_nlist *nl);
/* Grow the entry capacity (and the per-atom arrays) ahead of use; synchronous. */
fnn_status fnn_nlist_reserve(fnn_nlist *nl, int32_t n_atoms, int32_t n_mol, int64_t capacity);

/*
 * Directed neighbour list within R = rc_rad + skin (section II.A): entry (i, j, n)
 * for every ordered pair of distinct atoms of the same structure with
 * |x_j - x_i + n L|^2 < R^2, n the minimum-image shift (0 when not periodic).
 * The membership test is the float64 predicate d = (x_j - x_i) + n L per axis,
 * d2 = (dx*dx + dy*dy) + dz*dz, d2 < R*R, rounded to nearest without
 * contraction; the kernels prefilter in float32 and re-test a band around R in
 * float64, so the set is bit-exact with that predicate.  Cell lists: counting
 * sort of atoms into cells of edge >= R, then a warp per atom scans the 27
 * surrounding cells (ballot + popc compaction, prefix-sum row offsets).
 * Row order: a row of at most 128 entries is sorted by neighbour element
 * (H, C, N, O, F, S, Cl), stable within an element; a longer row is in cell
 * traversal order.  Either order is deterministic.
 * Also records the species-sorted atom order used by fnn_energy_forces.
 * Asynchronous on stream; overflow posts FNN_E_CAPACITY (info = entries needed).
 */
fnn_status fnn_build_neighbors(fnn_ctx *ctx, const fnn_system *sys, fnn_nlist *nl, void *stream);

/* Number of entries of the last build (synchronises the list's stream). */
fnn_status fnn_nlist_nnz(fnn_nlist *nl, int64_t *nnz);

/* Copy the last list to HOST buffers in CSR form: row_ptr [N+1] (int32), nbr [nnz]
 * (int32 neighbour index), shift [nnz][3] (int8).  Synchronous.  Returns
 * FNN_E_CAPACITY with *nnz set when cap < nnz. */
fnn_status fnn_nlist_export(fnn_nlist *nl, int32_t *row_ptr, int32_t *nbr, int8_t *shift, int64_t cap,
                            int64_t *nnz);

/* AEVs [N][1008] float32 (device, caller-owned, 16-byte aligned: FNN_E_INVALID otherwise) from a list
 * built for sys.
 * Radial slot e*16+k = sum over neighbours j of element e within rc_rad of
 * 1/4 exp(-eta_rad (r - R_k)^2) fc(r); angular slot 112 + p*32 + m*4 + s = sum
 * over unordered neighbour pairs {j,k} within rc_ang with element pair p of
 * 2 ((1 + cos(theta' - theta_s))/2)^zeta exp(-eta_ang ((r_ij + r_ik)/2 - A_m)^2)
 * fc(r_ij) fc(r_ik), theta' = acos(0.95 cos theta_ijk); fc the context's switching function
 * (cos(pi r/rc)/2 + 1/2 by default) with the cutoff of the term.
 * Asynchronous. */
fnn_status fnn_aev(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, float *aev, void *stream);

/* Tangent of the AEVs along a displacement field: T [N][1008] = (dAEV/dx) . V with V [N][3] (device,
 * float32): for every slot, the directional derivative of the symmetry function above (chain rule
 * through r_ij, r_ik and cos theta_ijk).  The force term of a training loss needs it (section IV:
 * dL_F/dtheta = -d/dtheta <T(dL/dF), dE/dAEV(theta)>).  Asynchronous. */
fnn_status fnn_aev_jvp(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *V, float *T, void *stream);

/* Energies E [n_mol] (float64, device), forces F [N][3] (float32, device) and,
 * when virial != NULL, virials [n_mol][9] (float64, device, W = -sum over
 * directed entries of d (x) dE_i/dd, = sum_i x_i (x) F_i for a gas-phase
 * structure).  E_m = (1/M) sum_members sum_{i in m} y_i, F = -dE/dx by the
 * analytic adjoint of the networks and the AEV.  Asynchronous. */
fnn_status fnn_energy_forces(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, fnn_precision prec,
                             double *E, float *F, double *virial, void *stream);

/* FP8 form (FNN_FP8): e4m3 operands on the tensor cores with per-layer scaling.  Every weight block
 * (member, element, layer) is scaled by amax/448 at load (the transposed first layer, whose
 * reduction runs over all members, by one scale per element); every activation tensor of a layer
 * (AEV, h1, h2 and the three backward tensors) by one scale, 2 amax/448, measured by an FP32
 * evaluation of sys here.  Conversions round to nearest and saturate.  Synchronises the stream.  An
 * FP8 call on a context that was never calibrated (or whose weights were reloaded) calibrates on its
 * own system first. */
fnn_status fnn_calibrate_fp8(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, void *stream);

/* The same computation from HOST arrays: copies the inputs to library-owned
 * device buffers, rebuilds the neighbour list, evaluates, copies E [n_mol],
 * F [N][3] and (optional) virial [n_mol][9] back to the host arrays, and
 * synchronises.  Z [N] int32, pos [N][3] float32, mol_offsets [n_mol+1],
 * cell [n_mol][9] or NULL, pbc [n_mol] or NULL.  Returns the sticky status. */
fnn_status fnn_energy_forces_host(fnn_ctx *ctx, int32_t n_atoms, int32_t n_mol, const int32_t *mol_offsets,
                                  const int32_t *Z, const float *pos, const float *cell, const uint8_t *pbc,
                                  fnn_precision prec, double *E, float *F, double *virial, void *stream);

/* Parameter gradients, float32, device, same layout as fnn_weights (caller-owned, ACCUMULATED into:
 * zero them first). */
typedef struct {
  float *W1, *b1, *W2, *b2, *W3, *b3, *w4, *b4;
} fnn_grads;

/*
 * Gradient of a training loss L(E, F) with respect to the network parameters (section IV: force
 * and energy terms), given dL/dE [n_mol] (float64, device) and dL/dF [N][3] (float32, device, atom
 * order) at the current parameters:
 *   dL/dtheta = dL/dE . dE/dtheta - d/dtheta <J v, dE/dAEV>,  v = dL/dF,  J = dAEV/dx,
 * the second term by a forward-mode tangent of the networks along J v (fnn_aev_jvp) and one reverse
 * sweep over the primal and tangent activations.  prec: FNN_FP32 (SIMT FP32 throughout) or FNN_BF16
 * (every product on the tensor cores with bf16 operands and FP32 accumulation, the weight gradients
 * as products over each element's rows); others give FNN_E_INVALID.  The list must be built for
 * sys.  Adds into g (zero it first).  Asynchronous on stream.
 */
fnn_status fnn_param_grads(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, fnn_precision prec,
                           const double *dLdE, const float *dLdF, const fnn_grads *g, void *stream);

/*
 * One step as a CUDA graph: fnn_build_neighbors (when rebuild != 0) then fnn_energy_forces, recorded on
 * stream (not the legacy default stream) after one eager step that sizes every buffer (and
 * calibrates the FP8 form), then instantiated.  The system's device arrays, the list and the outputs
 * are bound by address: a replay reads their contents at replay time (new positions in the same
 * buffer are fine; a different atom count or structure layout needs a new graph).  A replay cannot
 * grow a list: an overflow posts FNN_E_CAPACITY (read with fnn_sync); reserve and recreate.  The
 * eager step's device status is returned (and cleared) by create.  Synchronous.
 */
typedef struct fnn_graph fnn_graph;
fnn_status fnn_graph_create(fnn_ctx *ctx, const fnn_system *sys, fnn_nlist *nl, fnn_precision prec, double *E,
                            float *F, double *virial, int32_t rebuild, void *stream, fnn_graph **graph);
/* Replay on stream (asynchronous).  FNN_E_STATE (nothing launched) once the context has reallocated a
 * buffer the graph references since it was recorded: weights reloaded, or a larger system evaluated
 * on the context; record a new graph then. */
fnn_status fnn_graph_launch(fnn_graph *graph, void *stream);
/* Kernel launches one replay performs. */
fnn_status fnn_graph_kernels(const fnn_graph *graph, int64_t *kernels);
fnn_status fnn_graph_destroy(fnn_graph *graph);

/* Synchronise the stream, return and clear the sticky device status; *info
 * (optional) receives its detail (entries needed for FNN_E_CAPACITY, the
 * offending atom for FNN_E_SPECIES, ...). */
fnn_status fnn_sync(fnn_ctx *ctx, void *stream, int64_t *info);

/*
 * NVE velocity Verlet on the device: fnn_md_run_ex with FNN_MD_NVE, the skin guard on, no kinetic
 * history and no counters (asynchronous).  The list is rebuilt before evaluations 0, rebuild_every, ...
 * and early whenever an atom has moved more than skin/2 since the last rebuild.
 */
fnn_status fnn_md_run(fnn_ctx *ctx, const fnn_system *sys, float *pos, float *vel, fnn_nlist *nl, fnn_precision prec,
                      int32_t n_steps, double dt_fs, int32_t rebuild_every, double *E_hist, float *F, void *stream);

/*
 * Device-resident molecular dynamics (the native engine of section V.D): n_steps force evaluations at
 * x_0 .. x_{n-1} of the system whose positions are pos.  After evaluation k every atom does
 *   k > 0:     v += a dt/2  (completes step k-1; K_hist[k] is the kinetic energy of this v)
 *   k < n-1:   v += a dt/2, then
 *              FNN_MD_NVE:      x += v dt                                         (velocity Verlet)
 *              FNN_MD_LANGEVIN: x += v dt/2, v = c1 v + c2 sqrt(kB T/m) xi, x += v dt/2   (BAOAB)
 * a = F/m (masses H 1.008 C 12.011 N 14.007 O 15.999 F 18.998 S 32.06 Cl 35.45 amu; 1 kcal/mol/A/amu
 * = 4.184e-4 A/fs^2), c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2), kB = 0.0019872041 kcal/mol/K.  xi: for
 * atom i at noise step t = step0 + k, the Philox-4x32-10 block of counter (i, t mod 2^32, t >> 32, 0)
 * and key (seed mod 2^32, seed >> 32) gives words w0..w3, u_j = (floor(w_j / 256) + 1/2) / 2^24, and
 * xi = (sqrt(-2 ln u0) cos 2 pi u1, sqrt(-2 ln u0) sin 2 pi u1, sqrt(-2 ln u2) cos 2 pi u3).
 * Neighbour list: rebuilt before evaluation 0, whenever rebuild_every evaluations have passed since the
 * last rebuild, and (skin_guard != 0) before any evaluation at which some atom lies more than skin/2
 * from its position at the last rebuild (the context's skin; with skin 0 any motion rebuilds).  The
 * decision is taken on the device; on a stream other than the legacy default stream, whole blocks of
 * rebuild_every steps after the first run as replays of one CUDA graph whose rebuilds are conditional
 * nodes.  pos, vel: device [N][4] (w unused), updated in place.  E_hist: device [n_steps][n_mol]
 * float64 potential energies, or NULL.  K_hist: device [n_steps][n_mol] float64 kinetic energies (kcal/mol),
 * or NULL.  F: device [N][3], the forces of the last evaluation.  counters: host, or NULL; when given the
 * call synchronises the stream and fills it.  Otherwise asynchronous.
 */
typedef enum { FNN_MD_NVE = 0, FNN_MD_LANGEVIN = 1 } fnn_md_integrator;
typedef struct {
  int32_t n_steps;          /* force evaluations */
  double dt_fs;             /* time step, fs */
  int32_t rebuild_every;    /* the list is rebuilt at least every this many evaluations (>= 1) */
  int32_t skin_guard;       /* 1: also rebuild early when an atom moved more than skin/2 */
  int32_t integrator;       /* fnn_md_integrator */
  double temperature_K;     /* Langevin bath temperature */
  double friction_per_fs;   /* Langevin friction gamma (> 0), 1/fs */
  uint64_t seed;            /* Langevin noise key */
  uint64_t step0;           /* noise counter of evaluation 0 (continue a run with step0 + n_steps) */
} fnn_md_options;
typedef struct {
  int32_t rebuilds;          /* list builds, the first included */
  int32_t guard_rebuilds;    /* of them, forced early by the skin guard */
  int32_t graph_blocks;      /* blocks of rebuild_every steps that ran as graph replays */
  double max_displacement;   /* largest displacement from the last rebuild seen by a rebuild decision, A */
} fnn_md_counters;
fnn_status fnn_md_run_ex(fnn_ctx *ctx, const fnn_system *sys, float *pos, float *vel, fnn_nlist *nl,
                         fnn_precision prec, const fnn_md_options *opt, double *E_hist, double *K_hist, float *F,
                         fnn_md_counters *counters, void *stream);

/*
 * Ring-polymer molecular dynamics (the NQE method of section V.D): P replicas (beads) of one structure, whose
 * potential energies and forces come from one batched evaluation -- the beads are the P structures of the
 * system `beads` (n_mol = P, each of n_atoms / P atoms, bead b's atom i at b n + i, identical species and
 * cells; periodic beads use the minimum image each).  The free ring polymer, springs 1/2 m wP^2 |x_b - x_(b+1)|^2
 * with wP = P kB T / hbar (hbar = 15.178736 kcal/mol fs), is propagated exactly in its normal modes
 * q~_k = sum_j C_jk x_j (C: the real Fourier basis, 1/sqrt(P); sqrt(2/P) cos(2 pi j k / P) for 0 < k < P/2;
 * (-1)^j / sqrt(P) for k = P/2; sqrt(2/P) sin(2 pi j k / P) above), mode k a harmonic oscillator of frequency
 * 2 wP sin(k pi / P) (the centroid free).  After evaluation k: v += a dt/2 (completing step k-1; H_hist[k] =
 * the ring-polymer Hamiltonian: bead kinetic + spring + potential energies), and unless k is the last:
 * v += a dt/2 and the exact free-ring-polymer step for dt.  The list schedule and skin guard are those of
 * fnn_md_run_ex (the guard on a bound of the displacement: 3 times its largest component squared).
 * pos, vel: device [P n][4].  E_hist: device [n_steps][P] bead energies, or NULL.  H_hist: device [n_steps]
 * float64, or NULL.  F: device [P n][3], the last evaluation's forces.  counters as for fnn_md_run_ex.
 */
#define FNN_RPMD_MAX_BEADS 32
typedef struct {
  int32_t n_beads;          /* P, 1..FNN_RPMD_MAX_BEADS */
  int32_t n_steps;
  double dt_fs;
  double temperature_K;     /* sets the spring constant (> 0) */
  int32_t rebuild_every;
  int32_t skin_guard;
} fnn_rpmd_options;
fnn_status fnn_rpmd_run(fnn_ctx *ctx, const fnn_system *beads, float *pos, float *vel, fnn_nlist *nl,
                        fnn_precision prec, const fnn_rpmd_options *opt, double *E_hist, double *H_hist, float *F,
                        fnn_md_counters *counters, void *stream);

/*
 * Continuous-batching MD service.  A scheduler thread keeps a ragged batch of
 * structures on the device and advances all of them one velocity-Verlet step per batch step (one
 * neighbour-list/AEV/network/adjoint pass over the whole batch; the shared list is rebuilt when the
 * batch changes, every rebuild_every steps, and early when an atom of any structure has moved more
 * than skin/2 since the last rebuild); between batch steps it retires
 * finished structures and admits queued requests, in arrival order, while the batch's estimated
 * device memory stays within hbm_budget_bytes.  A structure's results do not depend on the rest of
 * the batch.  The server uses ctx (weights, constants, skin) exclusively while it exists: make no
 * other calls on that context meanwhile.
 */
typedef struct fnn_server fnn_server;

typedef struct {
  int32_t n_atoms;
  const int32_t *Z;     /* host [n] atomic numbers */
  const float *pos;     /* host [n][3] */
  const float *vel;     /* host [n][3] A/fs, or NULL = at rest */
  const float *cell;    /* host [9] orthorhombic cell (periodic, minimum image), or NULL = gas phase */
  int32_t n_steps;      /* force evaluations (MD steps) */
  double dt_fs;         /* time step */
} fnn_request;

typedef struct {
  double *energies;     /* host [n_steps] energy after each evaluation, or NULL */
  float *pos, *vel, *forces;  /* host [n][3] final state, or NULL */
  double latency_ms;    /* completion minus submission */
  double queue_ms;      /* admission minus submission */
  int32_t n_steps_done;
} fnn_result;

typedef struct {
  int64_t atom_evals;       /* atoms evaluated, summed over batch steps */
  int64_t batch_steps;
  int64_t admitted;
  int64_t max_batch_atoms;
  int64_t pending;          /* requests waiting for admission */
  double bytes_per_atom;    /* the admission estimate */
  double host_ms;           /* scheduler time spent retiring and re-laying out the batch */
  double step_ms;           /* scheduler time spent in batch steps (GPU work, waited for) */
  int64_t failed;           /* requests failed alone by their own structure's device-detected error */
  int64_t rebuilds;         /* batch neighbour-list builds */
  int64_t guard_rebuilds;   /* of them, forced early by the skin guard (an atom moved more than skin/2) */
} fnn_serve_counters;

fnn_status fnn_serve_create(fnn_server **srv, fnn_ctx *ctx, size_t hbm_budget_bytes, fnn_precision prec,
                            int32_t rebuild_every);
/* Copies the request; never blocks on the GPU.  Rejected at once, before it can reach the shared batch:
 * FNN_E_OOM when the structure alone exceeds the budget, FNN_E_SPECIES for an atomic number outside the
 * table, FNN_E_NONFINITE for a non-finite position or velocity, FNN_E_CELL for a cell that is not
 * orthorhombic or has an edge <= 2 (rc_rad + skin), FNN_E_INVALID for n_steps < 0.  A structure whose own
 * atoms raise a device-detected error later (a non-finite coordinate or energy, an atom beyond the AEV
 * neighbour limits) leaves the batch and its ticket's poll returns that error; the other requests go on. */
fnn_status fnn_serve_submit(fnn_server *srv, const fnn_request *req, uint64_t *ticket);
/* FNN_OK and the result (copied into the caller's buffers) once the request is done; FNN_PENDING if it
 * is not done within timeout_us (0 = do not wait).  A ticket's result can be taken once. */
fnn_status fnn_serve_poll(fnn_server *srv, uint64_t ticket, fnn_result *res, int64_t timeout_us);
fnn_status fnn_serve_stats(fnn_server *srv, fnn_serve_counters *stats);
/* Finishes every admitted and queued request, then releases the server. */
fnn_status fnn_serve_destroy(fnn_server *srv);

/*
 * Allocation-free neighbour list (no counterpart in the paper).
 *
 * For callers that may not allocate device memory themselves or through this
 * library -- for example code running inside a host framework that hands out
 * all device memory from its own pool, or a latency-sensitive loop in which
 * cudaMalloc/cudaFree would synchronise the device and stall other streams.
 * Builds the same directed list as fnn_build_neighbors (the same predicate and
 * cell traversal, in a two-pass count/fill form; rows of at most 128 entries
 * sorted by neighbour element, longer rows in traversal order, as there) for at
 * most FNN_STATIC_MAX_ATOMS atoms in at most FNN_STATIC_MAX_MOL structures, with
 * list radius R, and needs no context.  All scratch lives in one array of
 * 423,280 bytes compiled into the library, which every GPU that loads the
 * library keeps until the process exits; the call itself allocates nothing.
 *   sys      device system, as for fnn_build_neighbors.
 *   row_ptr  device int32 [N+1] (caller-owned), CSR row offsets.
 *   nbr      device int32 [cap], neighbour indices.
 *   shift4   device int8 [cap][4], 4-byte aligned: image shift x, y, z and a zero byte.
 *   nnz      host; receives the number of entries (also when it exceeds cap).
 * Returns FNN_E_CAPACITY at once, touching nothing, when n_atoms or n_mol is
 * above the limit; FNN_E_CAPACITY after the build when nnz > cap (entries
 * beyond cap are not written); otherwise the device status (FNN_E_SPECIES,
 * FNN_E_CELL, FNN_E_INVALID for inconsistent offsets, ...); FNN_E_CUDA when a
 * CUDA call fails, after waiting for the work the call had already queued.
 * Synchronises the stream before returning, so it must not be called while
 * the stream (or, in global capture mode, any stream) is being captured.
 * The array's device address is looked up (cudaGetSymbolAddress, with the
 * device current) by the first call in each CUDA context of a device, and
 * again after that context is reset.  Every call shares the one array per
 * device: calls that overlap on the GPU (several streams or threads at once)
 * race and corrupt each other's lists; each call clears the parts that must
 * start at zero.
 */
#define FNN_STATIC_MAX_ATOMS 8192
#define FNN_STATIC_MAX_MOL 256
fnn_status fnn_build_neighbors_static(const fnn_system *sys, double R, int32_t *row_ptr, int32_t *nbr, int8_t *shift4,
                                      int64_t cap, int64_t *nnz, void *stream);

/*
 * CRATE angular resource of the first interaction layer (Appendix A, angular resources), over the
 * neighbours within rc_ang of a list built for sys:
 *   D_ij[c] = f~(r_ij) sum_a B~_a(r_ij) V[e(j)][a][c],   B~_a(r) = exp(-eta_ang (r - A_a)^2),
 *   g_i[n][c] = sum over unordered neighbour pairs {j, k} of cos(n theta_jik) D_ij[c] D_ik[c],
 * a < FNN_CRATE_NB radial functions on the angular shifts A_a = shift_ang0 + a (rc_ang - shift_ang0) / 8,
 * n < FNN_CRATE_NT (the Fourier angular basis, cos(n theta) evaluated as a Chebyshev polynomial of
 * cos theta), c < FNN_CRATE_DA channels, f~ the context's switching function at rc_ang, e(j) the element
 * index (H C N O F S Cl = 0..6).  V [7][8][32] float32 (device): the product of the layer's neighbour
 * embedding table (a row per element) and its trainable tensor W_ang, contracted over the embedding.
 * g: device [N][4][32] float32, written.  At most 64 neighbours within rc_ang per atom (FNN_E_CAPACITY,
 * info = -(atom + 1); that atom's row is zero).  Asynchronous.
 */
#define FNN_CRATE_NB 8
#define FNN_CRATE_DA 32
#define FNN_CRATE_NT 4
fnn_status fnn_crate_angular(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *V, float *g,
                             void *stream);
/* Vector-Jacobian product of fnn_crate_angular: with G = dL/dg [N][4][32] (device), grad_x [N][3] = dL/dx and
 * (when grad_V != NULL) grad_V [7][8][32] = dL/dV, both device float32 and overwritten.  Asynchronous. */
fnn_status fnn_crate_angular_vjp(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *V,
                                 const float *G, float *grad_x, float *grad_V, void *stream);

/* Instrumentation (no counterpart in the paper; the tracing the benchmark reads).
 * fnn_profile_enable: while on, every kernel this context launches is bracketed
 * by CUDA events on its own stream (a few microseconds of host work per launch).
 * fnn_profile_read: synchronises the device, then returns per kernel name
 * (names: cap x 48 chars) the summed device milliseconds and launch counts
 * since the previous read; *count = number of distinct kernels.
 * fnn_launch_count: kernels launched by this context since creation. */
fnn_status fnn_profile_enable(fnn_ctx *ctx, int on);
fnn_status fnn_profile_read(fnn_ctx *ctx, char *names, double *ms, int64_t *launches, int32_t cap, int32_t *count);
fnn_status fnn_launch_count(const fnn_ctx *ctx, int64_t *n);

/* Self-test of the device-side wait limits (no counterpart in the paper; failure detection).  Runs the
 * neighbour build's single-pass prefix scan (decoupled look-back, whose every wait on a predecessor
 * tile gives up after about a second of clock cycles and posts FNN_E_TIMEOUT) over a library-owned
 * array of 3 x 2048 ones.  withhold != 0 makes the first tile never publish its sum, so the other
 * tiles' waits run out: the next fnn_sync returns FNN_E_TIMEOUT, nothing reads the scan's result, and
 * the context stays usable.  withhold == 0 checks the scan's result (FNN_E_INVALID if wrong).
 * Asynchronous on stream. */
fnn_status fnn_selftest_lookback(fnn_ctx *ctx, int32_t withhold, void *stream);

/* Text of the last host-side error of this context (never NULL). */
const char *fnn_last_error(const fnn_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* FNN_H */
