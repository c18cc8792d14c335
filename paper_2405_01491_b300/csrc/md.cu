// Device-resident NVE velocity Verlet (section V.D: the native engine integrates NVE runs with velocity
// Verlet, all on the GPU).  n force evaluations at x_0 .. x_{n-1}; after evaluation k every atom does
//   k < n-1:  v += c a dt with c = 1/2 (k = 0) or 1 (completing the previous half kick too), x += v dt
//   k = n-1:  v += a dt / 2 (k > 0), no drift
// with a = F / m * 4.184e-4 A/fs^2 per kcal/mol/A/amu.  Per-structure step counters let one launch
// advance a ragged batch whose structures joined at different times (the serving loop).
#include "fnn_internal.cuh"

namespace fnn {

// atomic masses (amu) in element order H C N O F S Cl
static const float MASS_AMU[NE] = {1.008f, 12.011f, 14.007f, 15.999f, 18.998f, 32.06f, 35.45f};
static constexpr float ACCEL = 4.184e-4f;

struct VVArgs {
  int n;
  float4 *pos, *vel;
  const float *F;              // [N][3]
  const uint8_t *elem;
  const int32_t *atom_mol;
  const int32_t *mol_step;     // evaluation index per structure, or NULL: `step` for all
  const int32_t *mol_nsteps;   // evaluations per structure, or NULL: `nsteps` for all
  const float *mol_dt;         // time step per structure (fs), or NULL: `dt` for all
  int step, nsteps;
  float dt;
  float acc[NE];               // ACCEL / mass
};

__global__ void k_vv(VVArgs a) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const int mol = a.atom_mol[i];
    if (mol < 0) continue;
    const int k = a.mol_step ? a.mol_step[mol] : a.step;
    const int n = a.mol_nsteps ? a.mol_nsteps[mol] : a.nsteps;
    if (k < 0 || k >= n) continue;
    const bool last = k == n - 1;
    const float c = last ? (k == 0 ? 0.f : 0.5f) : (k == 0 ? 0.5f : 1.f);
    const float dt = a.mol_dt ? a.mol_dt[mol] : a.dt;
    const float s = c * dt * a.acc[a.elem[i]];
    float4 v = a.vel[i];
    v.x += s * a.F[3 * (size_t)i];
    v.y += s * a.F[3 * (size_t)i + 1];
    v.z += s * a.F[3 * (size_t)i + 2];
    a.vel[i] = v;
    if (!last) {
      float4 x = a.pos[i];
      x.x += dt * v.x;
      x.y += dt * v.y;
      x.z += dt * v.z;
      a.pos[i] = x;
    }
  }
}

// copy E[m] of the evaluation just done into each structure's history at hist_off[m] + step[m]
__global__ void k_record_energy(int n_mol, const double *E, const int32_t *mol_step, const int32_t *mol_nsteps,
                                const int64_t *hist_off, double *hist, int step, int64_t stride) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n_mol; m += gridDim.x * blockDim.x) {
    const int k = mol_step ? mol_step[m] : step;
    const int n = mol_nsteps ? mol_nsteps[m] : 0x7fffffff;
    if (k < 0 || k >= n) continue;
    const int64_t at = hist_off ? hist_off[m] + k : (int64_t)k * stride + m;
    hist[at] = E[m];
  }
}

__global__ void k_advance_steps(int n_mol, int32_t *mol_step) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n_mol; m += gridDim.x * blockDim.x) mol_step[m]++;
}

fnn_status launch_vv(fnn_ctx *ctx, const fnn_nlist *nl, int n, float4 *pos, float4 *vel, const float *F,
                     const int32_t *mol_step, const int32_t *mol_nsteps, const float *mol_dt, int step, int nsteps,
                     double dt, cudaStream_t s) {
  if (n <= 0) return FNN_OK;
  VVArgs a;
  a.n = n;
  a.pos = pos;
  a.vel = vel;
  a.F = F;
  a.elem = nl->elem;
  a.atom_mol = nl->atom_mol;
  a.mol_step = mol_step;
  a.mol_nsteps = mol_nsteps;
  a.mol_dt = mol_dt;
  a.step = step;
  a.nsteps = nsteps;
  a.dt = (float)dt;
  for (int e = 0; e < NE; e++) a.acc[e] = ACCEL / MASS_AMU[e];
  int blocks = (n + 255) / 256;
  if (blocks > 8 * ctx->num_sms) blocks = 8 * ctx->num_sms;
  FNN_KERNEL(ctx, "vv_update", s);
  k_vv<<<blocks, 256, 0, s>>>(a);
  return check_launch(ctx, "vv_update");
}

fnn_status launch_record_energy(fnn_ctx *ctx, int n_mol, const double *E, const int32_t *mol_step,
                                const int32_t *mol_nsteps, const int64_t *hist_off, double *hist, int step,
                                int64_t stride, cudaStream_t s) {
  FNN_KERNEL(ctx, "record_energy", s);
  k_record_energy<<<(n_mol + 255) / 256, 256, 0, s>>>(n_mol, E, mol_step, mol_nsteps, hist_off, hist, step, stride);
  return check_launch(ctx, "record_energy");
}

fnn_status launch_advance_steps(fnn_ctx *ctx, int n_mol, int32_t *mol_step, cudaStream_t s) {
  FNN_KERNEL(ctx, "advance_steps", s);
  k_advance_steps<<<(n_mol + 255) / 256, 256, 0, s>>>(n_mol, mol_step);
  return check_launch(ctx, "advance_steps");
}

// One MD step on the device: [list rebuild] -> energies and forces -> energy history row -> velocity
// Verlet update -> step counter.  The step index lives on the device (mol_step), so a sequence of steps
// can be captured once as a CUDA graph and replayed.
static fnn_status md_step(fnn_ctx *ctx, fnn_system *v, float *pos, float *vel, fnn_nlist *nl, fnn_precision prec,
                          bool rebuild, int32_t n_steps, double dt_fs, double *E, double *E_hist, float *F,
                          int32_t *mol_step, int32_t *mol_nsteps, cudaStream_t s) {
  fnn_status st;
  if (rebuild && (st = fnn_build_neighbors(ctx, v, nl, s))) return st;
  if ((st = fnn_energy_forces(ctx, v, nl, prec, E, F, nullptr, s))) return st;
  if (E_hist && (st = launch_record_energy(ctx, v->n_mol, E, mol_step, mol_nsteps, nullptr, E_hist, 0, v->n_mol, s)))
    return st;
  if ((st = launch_vv(ctx, nl, v->n_atoms, reinterpret_cast<float4 *>(pos), reinterpret_cast<float4 *>(vel), F,
                      mol_step, mol_nsteps, nullptr, 0, n_steps, dt_fs, s)))
    return st;
  return launch_advance_steps(ctx, v->n_mol, mol_step, s);
}

__global__ void k_md_init(int n_mol, int32_t n_steps, int32_t *mol_step, int32_t *mol_nsteps) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n_mol; m += gridDim.x * blockDim.x) {
    mol_step[m] = 0;
    mol_nsteps[m] = n_steps;
  }
}

}  // namespace fnn

using namespace fnn;

extern "C" fnn_status fnn_md_run(fnn_ctx *ctx, const fnn_system *sys, float *pos, float *vel, fnn_nlist *nl,
                                 fnn_precision prec, int32_t n_steps, double dt_fs, int32_t rebuild_every,
                                 double *E_hist, float *F, void *stream) {
  if (!ctx || !sys || !pos || !vel || !nl || !F || n_steps < 0 || !(dt_fs > 0) || rebuild_every < 1 ||
      ((uintptr_t)pos & 15) || ((uintptr_t)vel & 15))
    return FNN_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  fnn_system v = *sys;
  v.pos = pos;
  const int nm = v.n_mol > 0 ? v.n_mol : 1;
  // scratch: energies of the current step, per-structure step counters
  char *scratch = nullptr;
  const size_t bytes = (size_t)nm * (sizeof(double) + 2 * sizeof(int32_t)) + 64;
  FNN_CUDA_TRY(ctx, cudaMallocAsync((void **)&scratch, bytes, s));
  double *E = reinterpret_cast<double *>(scratch);
  int32_t *mol_step = reinterpret_cast<int32_t *>(scratch + (size_t)nm * sizeof(double));
  int32_t *mol_nsteps = mol_step + nm;
  fnn_status st = FNN_OK;
  {
    FNN_KERNEL(ctx, "md_init", s);
    k_md_init<<<(nm + 255) / 256, 256, 0, s>>>(nm, n_steps, mol_step, mol_nsteps);
  }
  const int R = rebuild_every;
  int k = 0;
  // the first block eagerly (sizes every buffer, calibrates the FP8 form)
  for (; k < n_steps && k < R && !st; k++)
    st = md_step(ctx, &v, pos, vel, nl, prec, k % R == 0, n_steps, dt_fs, E, E_hist, F, mol_step, mol_nsteps, s);
  // whole blocks of R steps (one rebuild each) as a CUDA graph, when the stream can be captured
  if (!st && s && n_steps - k >= 2 * R) {
    const long long l0 = ctx->prof.launches;
    const bool prof = ctx->prof.on;
    ctx->prof.on = false;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      fnn_status cs = FNN_OK;
      for (int j = 0; j < R && !cs; j++)
        cs = md_step(ctx, &v, pos, vel, nl, prec, j == 0, n_steps, dt_fs, E, E_hist, F, mol_step, mol_nsteps, s);
      const cudaError_t ec = cudaStreamEndCapture(s, &g);
      if (cs || ec != cudaSuccess || !g || cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
    }
    cudaGetLastError();
    ctx->prof.on = prof;
    const long long per_block = ctx->prof.launches - l0;
    ctx->prof.launches = l0;
    if (exec) {
      for (; n_steps - k >= R; k += R) {
        if (cudaGraphLaunch(exec, s) != cudaSuccess) {
          cudaGetLastError();
          ctx->last_error = "cudaGraphLaunch failed";
          st = FNN_E_CUDA;
          break;
        }
        ctx->prof.launches += per_block;
      }
      cudaGraphExecDestroy(exec);
    }
    if (g) cudaGraphDestroy(g);
  }
  // the rest eagerly (also every step when the stream cannot be captured)
  for (; k < n_steps && !st; k++)
    st = md_step(ctx, &v, pos, vel, nl, prec, k % R == 0, n_steps, dt_fs, E, E_hist, F, mol_step, mol_nsteps, s);
  cudaFreeAsync(scratch, s);
  return st;
}
