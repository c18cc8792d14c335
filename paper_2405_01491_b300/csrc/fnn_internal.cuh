// Internal definitions shared by the CUDA translation units of libfnn.
// Nothing here is part of the C ABI (include/fnn.h is).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fnn.h"

namespace fnn {

// ---------------------------------------------------------------------------------------- sizes
constexpr int NE = 7;                       // elements H C N O F S Cl
constexpr int NSR = 16;                     // radial shifts
constexpr int NSA = 8;                      // angular radial shifts
constexpr int NSZ = 4;                      // angle sections
constexpr int NRAD = NE * NSR;              // 112
constexpr int NPAIR = NE * (NE + 1) / 2;    // 28
constexpr int NAEV = NRAD + NPAIR * NSA * NSZ;  // 1008
constexpr int H1 = 256, H2 = 192, H3 = 160; // hidden widths
constexpr int MAXM = 8;                     // ensemble members
constexpr int ROW_TILE = 128;               // species segments are padded to this many rows
// neighbour rows of at most PAIR_STRIDE entries (every row of a usual density) are stored sorted by
// neighbour element, stable within an element; longer rows are in traversal order
constexpr int PAIR_STRIDE = 128;
constexpr int RAD_CAP = 160;                // neighbours within rc_rad handled per atom
// systems of at most this many atoms (in at most SMALL_BUILD_MOL structures) have their list built by one
// block (k_small_build), and the FP32 forms evaluated by one kernel of thread-block clusters when atoms x
// members is at most SMALL_EVAL_ROWS (fnn_energy_forces)
constexpr int SMALL_BUILD_ATOMS = 256, SMALL_BUILD_MOL = 256, SMALL_EVAL_ROWS = 256;
constexpr int ANG_CAP = 64;                 // neighbours within rc_ang handled per atom
constexpr float CELU_ALPHA = 0.1f;
// 1/alpha, exact (10): kernels multiply by it instead of dividing by the rounded 0.1f, which is both
// closer to the definition and free of the division sequence that dominated the network epilogues
constexpr float CELU_INV_ALPHA = 10.0f;

// element index of an atomic number, -1 when outside the table
__host__ __device__ inline int element_of(int z) {
  switch (z) {
    case 1: return 0;
    case 6: return 1;
    case 7: return 2;
    case 8: return 3;
    case 9: return 4;
    case 16: return 5;
    case 17: return 6;
    default: return -1;
  }
}

// ---------------------------------------------------------------------------------------- status
// Sticky device-side status: the first error posted wins; fnn_sync reads and clears it.
struct DevStatus {
  int code;
  int pad;
  long long info;
};

__device__ inline void post_status(DevStatus *st, int code, long long info) {
  if (atomicCAS(&st->code, 0, code) == 0) st->info = info;
}

// ---------------------------------------------------------------------------------------- params
struct AevParams {
  float rc_rad, rc_ang;
  float eta_r, eta_a, zeta;
  float pi_rc_rad, pi_rc_ang;   // pi / rc
  float inv_rc_rad, inv_rc_ang; // 1 / rc
  float shf_r[NSR];
  float shf_a[NSA];
  float cos_z[NSZ], sin_z[NSZ]; // cos / sin of the section centres
  float hcos_z[NSZ], hsin_z[NSZ];   // the same halved
  float qcos_z[NSZ];            // 0.475 cos: the cos term of d(base)/dc in the adjoint
  float eta_a_l2;               // -eta_a log2(e): the angular Gaussian as a power of two
  float eta_r_l2;               // -eta_r log2(e): the radial one
  int sw_kind;                  // fnn_switch
  float sw_pm1;                 // polynomial envelope: p - 1, and the coefficients of d^p, d^(p+1), d^(p+2)
  float sw_c0, sw_c1, sw_c2;
  float sw_k;                   // p (p+1) (p+2) / 2: f'(d) = -sw_k d^(p-1) (1 - d)^2
  // the same constants side by side for the packed FP32 pair instructions: negated shifts (k, k + 1) and
  // the section constants (s, s + 1)
  float2 nshr2[NSR / 2], nsha2[NSA / 2];
  float2 hcos2[NSZ / 2], hsin2[NSZ / 2], qcos2[NSZ / 2];
};

// The switching function and its derivative at r < rc (section II.A): cosine, polynomial envelope
// (Gasteiger et al. 2020), exponential (SpookyNet); the kind is uniform over a launch.
// sin and cos of y = (pi / 2) min(x, 1 - x), 0 <= x <= 1, by their Taylor series to y^9 and y^8 (y <= pi / 4:
// truncation below 2e-9 and 3e-8).  The cosine switch is cos^2(pi x / 2) = 1/2 cos(pi x) + 1/2 with
// x = r / rc: c^2 for x <= 1/2, s^2 above (never negative, accurate to the last bits near the cutoff), and
// its derivative -(pi / rc) s c.
__device__ __forceinline__ void quarter_sincos(float x, float &s, float &c) {
  const float y = 1.57079632679489662f * fminf(x, 1.f - x), z = y * y;
  s = y * fmaf(z, fmaf(z, fmaf(z, fmaf(z, 2.75573192e-6f, -1.98412698e-4f), 8.33333333e-3f), -1.66666667e-1f), 1.f);
  c = fmaf(z, fmaf(z, fmaf(z, fmaf(z, 2.48015873e-5f, -1.38888889e-3f), 4.16666667e-2f), -0.5f), 1.f);
}
__device__ __forceinline__ float switch_f(const AevParams &P, float r, float rc, float inv_rc) {
  if (P.sw_kind == FNN_SWITCH_POLYNOMIAL) {
    // near the cutoff the terms cancel to O(float eps), which may fall just below zero: clamped, since the
    // angular terms take the logarithm of switch products
    const float d = r * inv_rc;
    return fminf(fmaxf(1.f + powf(d, P.sw_pm1) * d * (P.sw_c0 + d * (P.sw_c1 + d * P.sw_c2)), 0.f), 1.f);
  }
  if (P.sw_kind == FNN_SWITCH_EXPONENTIAL) return expf(-r * r / ((rc - r) * (rc + r)));
  const float x = r * inv_rc;
  float sn, cs;
  quarter_sincos(x, sn, cs);
  return x <= 0.5f ? cs * cs : sn * sn;
}
__device__ __forceinline__ float switch_df(const AevParams &P, float r, float rc, float inv_rc, float pi_rc) {
  if (P.sw_kind == FNN_SWITCH_POLYNOMIAL) {
    const float d = r * inv_rc, om = 1.f - d;
    return -P.sw_k * powf(d, P.sw_pm1) * om * om * inv_rc;
  }
  if (P.sw_kind == FNN_SWITCH_EXPONENTIAL) {
    const float q = (rc - r) * (rc + r);
    return -expf(-r * r / q) * 2.f * r * rc * rc / (q * q);
  }
  float sn, cs;
  quarter_sincos(r * inv_rc, sn, cs);
  return -pi_rc * sn * cs;
}

// the lanes of a 32-entry chunk whose element is q, from the three bit planes of the lanes' elements
__device__ __forceinline__ unsigned elem_lanes(int q, unsigned b0, unsigned b1, unsigned b2) {
  return (q & 1 ? b0 : ~b0) & (q & 2 ? b1 : ~b1) & (q & 4 ? b2 : ~b2);
}

// per-structure cell-list geometry
struct MolGrid {
  float ox, oy, oz;       // origin of the grid (gas phase: bounding-box minimum; periodic: 0)
  float ix, iy, iz;       // cells per A along each axis
  float Lx, Ly, Lz;       // periodic box edges (0 when not periodic)
  int dx, dy, dz;         // cells per axis
  int cell_base;          // unused (first cells come from the scanned per-structure counts)
  int pbc;
  float iLx, iLy, iLz;    // 1 / box edge (0 when not periodic)
  float tau;              // float32 error band of the neighbour predicate for every pair of the structure
};

// ---------------------------------------------------------------------------------------- handles
struct DeviceWeights {
  int M = 0;
  // FP32, element-major concatenations for the member-fused layers
  float *W1cat = nullptr;   // [7][M*256][1008]
  float *b1cat = nullptr;   // [7][M*256]
  float *W1Tcat = nullptr;  // [7][1008][M*256]
  float *W2 = nullptr;      // [M][7][192][256]
  float *b2 = nullptr;      // [M][7][192]
  float *W2T = nullptr;     // [M][7][256][192]
  float *W3 = nullptr;      // [M][7][160][192]
  float *b3 = nullptr;      // [M][7][160]
  float *W3T = nullptr;     // [M][7][192][160]
  float *w4 = nullptr;      // [M][7][160]
  float *b4 = nullptr;      // [M][7]
  void *tc = nullptr;       // tensor-core forms (mlp_tc.cu)
};

struct Workspace {
  size_t rows = 0;          // padded row capacity
  int M = 0;
  float *aev = nullptr;     // [rows][1008]
  float *h1 = nullptr;      // [rows][M*256]
  float *h2 = nullptr;      // [rows][M*192]
  float *g3 = nullptr;      // [rows][M*160]
  float *g2 = nullptr;      // [rows][M*192]
  float *g1 = nullptr;      // [rows][M*256]
  float *gaev = nullptr;    // [rows][1008]
  float *ypart = nullptr;   // [rows][M][4]
  double *e_part = nullptr; // [rows] slice sums of the structure energies
  unsigned *e_ticket = nullptr;  // [rows] slices finished per structure (zero between launches)
  void *tc = nullptr;       // tensor-core buffers (mlp_tc.cu)
  size_t tc_rows = 0;
};

}  // namespace fnn

namespace fnn {
// Kernel timing: when enabled, each launch is bracketed by CUDA events on its stream.
struct Profiler {
  struct Rec {
    const char *name;
    cudaEvent_t a, b;
  };
  bool on = false;
  long long launches = 0;        // every kernel this context launched (always counted)
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
};
}  // namespace fnn

struct fnn_ctx {
  fnn::Profiler prof;
  fnn_config cfg;
  fnn::AevParams aev;
  int device = 0;
  int num_sms = 148;
  fnn::DevStatus *status = nullptr;   // device
  int32_t *pinned_flag = nullptr;      // 64 pinned host bytes: device scalars read between eager MD steps
  void *grid_bar = nullptr;            // the small-system kernel's finish counter and output-layer sums (device)
  fnn::DeviceWeights w;
  bool has_weights = false;
  fnn::Workspace ws;
  void *train = nullptr;                // training-gradient buffers (train.cu)
  // a second stream for independent work inside one call (fork: side waits for the caller's stream;
  // join: the caller's stream waits for side), so captured graphs get parallel branches
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::string last_error;
  // bumped whenever a device buffer that a recorded graph may reference is (re)allocated
  long long gen = 0;
  // host-call staging (fnn_energy_forces_host)
  struct HostStage {
    int32_t n_atoms = -1, n_mol = -1;
    int32_t *Z = nullptr, *mol_offsets = nullptr;
    float *pos = nullptr, *cell = nullptr;
    uint8_t *pbc = nullptr;
    float *pos3 = nullptr;
    double *E = nullptr, *virial = nullptr;
    float *F = nullptr;
    fnn_nlist *nl = nullptr;
    cudaStream_t own = nullptr;        // the entry point's stream when the caller gives none
    fnn_graph *graph = nullptr;        // the device part of the last repeated call, replayed
    long long gkey = -1, last_key = -1;
    fnn::DevStatus *status = nullptr;  // pinned: the device status read back in the call's own stream order
    long long ggen = -1;               // ctx->gen when graph was recorded
  } host;
};

struct fnn_nlist {
  fnn_ctx *ctx = nullptr;
  int64_t capacity = 0;       // entries
  bool auto_size = false;     // created without a capacity: grows to 160 entries per atom with the system
  int32_t atom_cap = 0, mol_cap = 0, cell_cap = 0, pad_cap = 0;
  int32_t n_atoms = 0, n_mol = 0;
  double R = 0.0;
  bool built = false;
  cudaStream_t stream = nullptr;
  // list
  int32_t *row_ptr = nullptr;   // [N+1]
  int32_t *nbr = nullptr;       // [cap]
  char4 *shift = nullptr;       // [cap]
  // per atom
  int32_t *atom_mol = nullptr;  // [N]
  uint8_t *elem = nullptr;      // [N]
  int32_t *cell_of = nullptr;   // [N]
  int32_t *cell_tmp = nullptr;  // [N]
  int32_t *cell_atoms = nullptr;// [N]
  float4 *cell_pos = nullptr;   // [N] positions in cell_atoms order
  int32_t *counts = nullptr;    // [N + 1]
  int32_t *stage_nbr = nullptr; // [N][128] first pass of the pair search, one slot per atom
  char4 *stage_shift = nullptr; // [N][128]
  // per structure
  fnn::MolGrid *grid = nullptr; // [n_mol]
  float *bbox = nullptr;        // [n_mol][6] bounding box (min xyz, max xyz)
  int32_t *mol_cells = nullptr; // [n_mol + 1]
  // per cell
  int32_t *cell_count = nullptr;// [cells + 1]
  int32_t *cell_start = nullptr;// [cells + 1]
  // species order
  int32_t *perm = nullptr;      // [N] atom -> padded species-sorted row
  int32_t *inv = nullptr;       // [pad_cap] row -> atom, -1 for padding
  int32_t *tile_elem = nullptr; // [pad_cap / 128] element of each 128-row tile, -1 beyond the end
  int32_t *blk_count = nullptr; // [blocks][8]
  int32_t *meta = nullptr;      // device scalars, see META_*
  int32_t *scan_tmp = nullptr;  // scan block sums
  int64_t scan_tmp_len = 0;
};

namespace fnn {

// META_BAD: 1 when the structure offsets are inconsistent (written once per build by k_check_cover's first
// block; every later setup kernel then treats all atoms as outside every structure)
enum { META_CELLS = 0, META_NNZ = 1, META_NPAD = 2, META_BAD = 3, META_SEG = 4 /* [8] segment starts */, META_LEN = 16 };

// ---------------------------------------------------------------------------------------- helpers
#define FNN_CUDA_TRY(ctx, call)                                                        \
  do {                                                                                 \
    cudaError_t err__ = (call);                                                        \
    if (err__ != cudaSuccess) {                                                        \
      (ctx)->last_error = std::string(#call) + ": " + cudaGetErrorString(err__);      \
      return FNN_E_CUDA;                                                               \
    }                                                                                  \
  } while (0)

fnn_status check_launch(fnn_ctx *ctx, const char *what);

// FP32 SIMT product C[r, n] = epi(sum_k A[r, k] B[n, k]) over 128-row species tiles (mlp_simt.cu)
enum { EPI_BIAS_CELU = 0, EPI_L3 = 1, EPI_DCELU = 2, EPI_SCALE = 3, EPI_L3_H = 4 };
struct GemmP {
  const float *A;
  long long lda, a_mstride;
  const float *B;
  long long ldb, b_estride, b_mstride;
  float *C;
  long long ldc, c_mstride;
  int N, K;
  const int32_t *tile_elem;
  const float *bias;
  long long bias_estride, bias_mstride;
  const float *aux;              // h of the previous layer (EPI_DCELU)
  long long ldaux, aux_mstride;
  const float *w4;               // EPI_L3, EPI_L3_H
  long long w4_estride, w4_mstride;
  float *ypart;                  // [rows][M][4]
  int M;
  float scale;
};
fnn_status launch_gemm_f32(fnn_ctx *ctx, const char *name, int epi, const GemmP &p, int row_tiles, int members,
                           cudaStream_t s);

// Scope around one kernel launch: counts it and, when profiling, records events around it.
struct KScope {
  fnn_ctx *ctx;
  cudaStream_t s;
  int idx = -1;
  KScope(fnn_ctx *c, const char *name, cudaStream_t st);
  ~KScope();
};
#define FNN_CAT2(a, b) a##b
#define FNN_CAT(a, b) FNN_CAT2(a, b)
#define FNN_KERNEL(ctx, name, s) ::fnn::KScope FNN_CAT(kscope_, __LINE__)(ctx, name, s)

// exclusive scan of n int32 values in place; total written to *total_dev (device) when non-null
fnn_status exclusive_scan(fnn_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, int32_t *total_dev, int32_t *tmp,
                          int64_t tmp_len, cudaStream_t s, const int32_t *n_dev = nullptr, int32_t *out2 = nullptr,
                          int64_t cap = -1, bool zeroed = false);
int64_t scan_tmp_needed(int64_t n);
// work enqueued on ctx->side between side_fork(s) and side_join(s) runs after what s held at the fork
// and before what s gets after the join
fnn_status side_fork(fnn_ctx *ctx, cudaStream_t s);
fnn_status side_join(fnn_ctx *ctx, cudaStream_t s);

// kernels' host launchers (defined in their .cu files)
fnn_status launch_aev_forward(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, float *out,
                              const int32_t *inv, cudaStream_t s);
fnn_status launch_aev_adjoint(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *gaev,
                              const int32_t *inv, float *F, double *virial, cudaStream_t s);
fnn_status launch_aev_tangent(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *V, float *out,
                              const int32_t *inv, cudaStream_t s);
// bf16 tangent rows, and (out_fwd != NULL) the bf16 AEV rows of the same pass, equal to launch_aev_forward_bf16's
fnn_status launch_aev_tangent_bf16(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *V,
                                   __nv_bfloat16 *out, __nv_bfloat16 *out_fwd, const int32_t *inv, cudaStream_t s);
fnn_status mlp_fp32_forward_backward(fnn_ctx *ctx, const fnn_nlist *nl, cudaStream_t s);
fnn_status tc_energy(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, fnn_precision prec, double *E,
                     cudaStream_t s);
fnn_status upload_tc_weights(fnn_ctx *ctx, int M, const float *W1cat, const float *W1Tcat, const float *W2,
                             const float *W2T, const float *W3, const float *W3T);
void free_tc(fnn_ctx *ctx);
fnn_status fp8_calibrate(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, cudaStream_t s);
void free_train(fnn_ctx *ctx);
fnn_status tc_param_grads(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const double *dLdE,
                          const float *dLdF, const fnn_grads *g, cudaStream_t s);
fnn_status energy_reduce(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, double *E, cudaStream_t s);
fnn_status energy_reduce_rows(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *ypart,
                              int ntile, double *E, cudaStream_t s);
fnn_status ensure_workspace(fnn_ctx *ctx, size_t rows);
// energies, forces and virials of a small system in one launch of thread-block clusters (FP32 networks), aev.cu
fnn_status launch_small_eval(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, double *E, float *F,
                             double *virial, cudaStream_t s);

// ------------------------------------------------------------------------------------------- MD (md.cu)
// device state of one MD run: the rebuild schedule and the skin guard
struct MdState {
  int since_build;      // evaluations since the last rebuild
  unsigned max_d2;      // largest |x - x_ref|^2 since the last rebuild (float bits, non-negative)
  int rebuilds, guard_rebuilds;
  unsigned max_seen;    // largest max_d2 any rebuild decision saw (float bits)
  int need;             // the last decision
};
// one integrator update after an evaluation: NVE velocity Verlet, or BAOAB Langevin when gamma > 0
struct MdUpdate {
  const int32_t *mol_step = nullptr, *mol_nsteps = nullptr;   // per structure, or NULL: step / nsteps for all
  const float *mol_dt = nullptr;                              // per structure, or NULL: dt for all
  int step = 0, nsteps = 0;
  double dt = 0.0;
  double gamma = 0.0, temperature = 0.0;   // 1/fs, K
  uint64_t seed = 0, step0 = 0;            // noise key and the counter of evaluation 0
  const float4 *xref = nullptr;            // positions at the last rebuild (guard), or NULL
  unsigned *max_d2 = nullptr;              // max |x - xref|^2 (float bits) accumulated by atomicMax, or NULL
  double *K = nullptr;                     // kinetic energies K[k * K_stride + m] (kcal/mol), or NULL
  int64_t K_stride = 0;
};
fnn_status launch_md_update(fnn_ctx *ctx, const fnn_nlist *nl, int n, float4 *pos, float4 *vel, const float *F,
                            const MdUpdate &u, cudaStream_t s);
fnn_status launch_record_energy(fnn_ctx *ctx, int n_mol, const double *E, const int32_t *mol_step,
                                const int32_t *mol_nsteps, const int64_t *hist_off, double *hist, int step,
                                int64_t stride, cudaStream_t s);
fnn_status launch_advance_steps(fnn_ctx *ctx, int n_mol, int32_t *mol_step, MdState *st, cudaStream_t s);
fnn_status launch_md_ref(fnn_ctx *ctx, int n, const float4 *pos, float4 *xref, cudaStream_t s);

}  // namespace fnn
