// Device-resident molecular dynamics (section V.D: the native engine runs entirely on the GPU; NVE uses
// velocity Verlet, Langevin dynamics the BAOAB splitting of Leimkuhler and Matthews).
//
// n force evaluations at x_0 .. x_{n-1}.  After evaluation k every atom does
//   k > 0:      v += a dt/2                      (B: completes step k-1, v = v_k; kinetic energy of v_k)
//   k < n-1:    v += a dt/2                      (B)
//               NVE:      x += v dt
//               Langevin: x += v dt/2 (A), v = c1 v + c2 sqrt(kB T / m) xi (O), x += v dt/2 (A)
// with a = F / m * 4.184e-4 A/fs^2 per kcal/mol/A/amu, c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2), and xi
// three standard normal numbers per atom and evaluation from a Philox-4x32-10 stream (Salmon et al. 2011)
// keyed by the seed, counter (atom, step) -> Box-Muller.  Per-structure step counters let one launch
// advance a ragged batch whose structures joined at different times (the serving loop).
//
// Neighbour-list schedule: the list is rebuilt before evaluation k when k is the first, when
// rebuild_every evaluations have passed since the last rebuild, or (skin guard) when some atom has moved
// more than skin/2 from where it was at the last rebuild -- beyond that two atoms could have closed
// from outside the list radius to inside the cutoff.  The decision is taken on the device (k_md_decide);
// in a CUDA graph it drives a conditional node around the rebuild, so replayed blocks of steps rebuild
// exactly when needed with no host round trip.
#include <cmath>
#include <cstring>
#include <vector>

#include "fnn_internal.cuh"

namespace fnn {

// atomic masses (amu) in element order H C N O F S Cl
static const double MASS_AMU[NE] = {1.008, 12.011, 14.007, 15.999, 18.998, 32.06, 35.45};
static constexpr double ACCEL = 4.184e-4;       // A/fs^2 per kcal/mol/A/amu (and A^2/fs^2 per kcal/mol/amu)
static constexpr double KB_KCAL = 0.0019872041; // Boltzmann constant, kcal/mol/K
static constexpr double HBAR_KCAL_FS = 15.178736; // reduced Planck constant, kcal/mol fs

// ------------------------------------------------------------------------------------ Philox-4x32-10
// Counter-based generator of Salmon, Moraes, Dror and Shaw (SC 2011): ten rounds of two 32x32->64 bit
// products with the published multipliers, the key advanced by the published Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// uniform in (0, 1) from the top 24 bits of a word (exact in float32)
__device__ __forceinline__ float unit24(uint32_t w) { return ((float)(w >> 8) + 0.5f) * 5.9604644775390625e-8f; }

// three standard normal numbers for atom i at noise step t (Box-Muller on words 0,1 and 2,3)
__device__ __forceinline__ float3 langevin_noise(int i, unsigned long long t, uint32_t k0, uint32_t k1) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)t, (uint32_t)(t >> 32), 0u), k0, k1);
  const float r0 = sqrtf(-2.f * logf(unit24(w.x))), r1 = sqrtf(-2.f * logf(unit24(w.z)));
  float s0, c0;
  sincospif(2.f * unit24(w.y), &s0, &c0);
  return make_float3(r0 * c0, r0 * s0, r1 * cospif(2.f * unit24(w.w)));
}

// ------------------------------------------------------------------------------------ update kernel
struct MdKArgs {
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
  float half_m[NE];            // mass / (2 ACCEL): kinetic energy in kcal/mol per (A/fs)^2
  int langevin;
  float c1;                    // exp(-gamma dt)
  float c2sig[NE];             // sqrt(1 - c1^2) sqrt(kB T ACCEL / m)
  uint32_t key0, key1;
  unsigned long long step0;    // noise counter of evaluation k: step0 + k
  const float4 *xref;          // positions at the last rebuild, or NULL: no displacement maximum
  unsigned *max_d2;            // max |x - xref|^2 (float bits, non-negative) over the updated atoms
  double *K;                   // K[k * K_stride + m] += kinetic energy of structure m at evaluation k, or NULL
  long long K_stride;
};

__global__ void __launch_bounds__(256) k_md_update(MdKArgs a) {
  const unsigned FULL = 0xffffffffu;
  for (int i0 = blockIdx.x * blockDim.x; i0 < a.n; i0 += gridDim.x * blockDim.x) {   // warp-uniform trip count
    const int i = i0 + threadIdx.x;
    float d2 = 0.f, ke = 0.f;
    int mol = -1, kk = -1;
    if (i < a.n) {
      const int m = a.atom_mol[i];
      const int k = m < 0 ? -1 : (a.mol_step ? a.mol_step[m] : a.step);
      const int n = m < 0 ? 0 : (a.mol_nsteps ? a.mol_nsteps[m] : a.nsteps);
      if (m >= 0 && k >= 0 && k < n) {
        mol = m;
        kk = k;
        const int e = a.elem[i];
        const float dt = a.mol_dt ? a.mol_dt[m] : a.dt;
        const float h = 0.5f * dt * a.acc[e];
        const float fx = a.F[3 * (size_t)i], fy = a.F[3 * (size_t)i + 1], fz = a.F[3 * (size_t)i + 2];
        float4 v = a.vel[i];
        if (k > 0) {   // completes step k - 1
          v.x = fmaf(h, fx, v.x);
          v.y = fmaf(h, fy, v.y);
          v.z = fmaf(h, fz, v.z);
        }
        ke = a.half_m[e] * (v.x * v.x + v.y * v.y + v.z * v.z);
        if (k < n - 1) {
          v.x = fmaf(h, fx, v.x);
          v.y = fmaf(h, fy, v.y);
          v.z = fmaf(h, fz, v.z);
          float4 x = a.pos[i];
          if (a.langevin) {
            const float hd = 0.5f * dt;
            x.x = fmaf(hd, v.x, x.x);
            x.y = fmaf(hd, v.y, x.y);
            x.z = fmaf(hd, v.z, x.z);
            const float3 xi = langevin_noise(i, a.step0 + (unsigned long long)k, a.key0, a.key1);
            const float c = a.c2sig[e];
            v.x = fmaf(a.c1, v.x, c * xi.x);
            v.y = fmaf(a.c1, v.y, c * xi.y);
            v.z = fmaf(a.c1, v.z, c * xi.z);
            x.x = fmaf(hd, v.x, x.x);
            x.y = fmaf(hd, v.y, x.y);
            x.z = fmaf(hd, v.z, x.z);
          } else {
            x.x = fmaf(dt, v.x, x.x);
            x.y = fmaf(dt, v.y, x.y);
            x.z = fmaf(dt, v.z, x.z);
          }
          a.pos[i] = x;
          if (a.xref) {
            const float4 r = a.xref[i];
            const float dx = x.x - r.x, dy = x.y - r.y, dz = x.z - r.z;
            d2 = dx * dx + dy * dy + dz * dz;
            if (!(d2 == d2)) d2 = __int_as_float(0x7f800000);   // a non-finite position: rebuild (and report)
          }
        }
        a.vel[i] = v;
      }
    }
    if (a.max_d2) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(FULL, d2, o));
      if ((threadIdx.x & 31) == 0 && d2 > 0.f) atomicMax(a.max_d2, __float_as_uint(d2));
    }
    if (a.K) {
      const int m0 = __shfl_sync(FULL, mol, 0), k0 = __shfl_sync(FULL, kk, 0);
      if (__all_sync(FULL, mol == m0 && kk == k0)) {
        float t = ke;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
        if ((threadIdx.x & 31) == 0 && m0 >= 0) atomicAdd(&a.K[(long long)k0 * a.K_stride + m0], (double)t);
      } else if (mol >= 0) {
        atomicAdd(&a.K[(long long)kk * a.K_stride + mol], (double)ke);
      }
    }
  }
}

fnn_status launch_md_update(fnn_ctx *ctx, const fnn_nlist *nl, int n, float4 *pos, float4 *vel, const float *F,
                            const MdUpdate &u, cudaStream_t s) {
  if (n <= 0) return FNN_OK;
  MdKArgs a{};
  a.n = n;
  a.pos = pos;
  a.vel = vel;
  a.F = F;
  a.elem = nl->elem;
  a.atom_mol = nl->atom_mol;
  a.mol_step = u.mol_step;
  a.mol_nsteps = u.mol_nsteps;
  a.mol_dt = u.mol_dt;
  a.step = u.step;
  a.nsteps = u.nsteps;
  a.dt = (float)u.dt;
  a.langevin = u.gamma > 0.0;
  const double c1 = a.langevin ? exp(-u.gamma * u.dt) : 1.0;
  a.c1 = (float)c1;
  for (int e = 0; e < NE; e++) {
    a.acc[e] = (float)(ACCEL / MASS_AMU[e]);
    a.half_m[e] = (float)(0.5 * MASS_AMU[e] / ACCEL);
    a.c2sig[e] = a.langevin ? (float)(sqrt(1.0 - c1 * c1) * sqrt(KB_KCAL * u.temperature * ACCEL / MASS_AMU[e]))
                            : 0.f;
  }
  a.key0 = (uint32_t)u.seed;
  a.key1 = (uint32_t)(u.seed >> 32);
  a.step0 = u.step0;
  a.xref = u.xref;
  a.max_d2 = u.max_d2;
  a.K = u.K;
  a.K_stride = u.K_stride;
  int blocks = (n + 255) / 256;
  if (blocks > 8 * ctx->num_sms) blocks = 8 * ctx->num_sms;
  FNN_KERNEL(ctx, "md_update", s);
  k_md_update<<<blocks, 256, 0, s>>>(a);
  return check_launch(ctx, "md_update");
}

// ------------------------------------------------------------------------------------------ RPMD
// Ring-polymer MD (section V.D, NQE methods): the P beads of one ring polymer are the P structures of the
// batch (bead b's atom i at b N + i), all at the same step.  One warp per (atom, Cartesian component),
// lane = bead: the kicks, the ring-polymer Hamiltonian terms (kinetic + springs 1/2 m wP^2 |x_b - x_(b+1)|^2),
// and the exact free-ring-polymer step in normal modes q~_k = sum_j C_jk x_j (transforms by shuffles).
constexpr int RPMD_MAXP = 32;
struct RpmdKArgs {
  int N, P;
  float4 *pos, *vel;
  const float *F;
  const uint8_t *elem;
  const int32_t *mol_step;
  int nsteps;
  float dt;
  float acc[NE];         // ACCEL / mass
  float half_m[NE];      // mass / (2 ACCEL)
  float half_m_wp2[NE];  // mass wP^2 / (2 ACCEL)
  const float *C;        // [P][P] bead j, mode k
  const float4 *prop;    // [P] per mode: cos(w dt), sin(w dt) / w (dt for w = 0), -w sin(w dt)
  const double *E;       // [P] bead energies of this evaluation
  double *H;             // [nsteps] ring-polymer Hamiltonian, or NULL
  const float4 *xref;    // guard reference positions, or NULL
  unsigned *max_d2;
};

__global__ void __launch_bounds__(256) k_rpmd_update(RpmdKArgs a) {
  __shared__ float Cs[RPMD_MAXP * RPMD_MAXP];
  __shared__ float4 ps[RPMD_MAXP];
  __shared__ double hsum;
  const unsigned FULL = 0xffffffffu;
  const int P = a.P;
  for (int q = threadIdx.x; q < P * P; q += blockDim.x) Cs[q] = a.C[q];
  for (int q = threadIdx.x; q < P; q += blockDim.x) ps[q] = a.prop[q];
  if (threadIdx.x == 0) hsum = 0.0;
  __syncthreads();
  const int k = a.mol_step[0];
  const bool valid = k >= 0 && k < a.nsteps;
  const int lane = threadIdx.x & 31;
  const bool on = lane < P;
  const int nw = 3 * a.N;
  float hacc = 0.f;
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; valid && w < nw; w += (gridDim.x * blockDim.x) >> 5) {
    const int i = w / 3, comp = w - 3 * i;
    const int e = a.elem[i];
    const size_t at = (size_t)(on ? lane : 0) * a.N + i;
    float x = 0.f, v = 0.f, f = 0.f;
    if (on) {
      x = reinterpret_cast<const float *>(a.pos + at)[comp];
      v = reinterpret_cast<const float *>(a.vel + at)[comp];
      f = a.F[3 * at + comp];
    }
    const float h = 0.5f * a.dt * a.acc[e];
    if (k > 0) v = fmaf(h, f, v);   // completes step k - 1
    const float xn = __shfl_sync(FULL, x, on ? (lane + 1) % P : lane);
    if (on) hacc += a.half_m[e] * v * v + a.half_m_wp2[e] * (x - xn) * (x - xn);
    if (k < a.nsteps - 1) {
      v = fmaf(h, f, v);
      float qm = 0.f, pm = 0.f;   // lane m: normal mode m
      for (int j = 0; j < P; j++) {
        const float xj = __shfl_sync(FULL, x, j), vj = __shfl_sync(FULL, v, j);
        const float c = on ? Cs[j * P + lane] : 0.f;
        qm = fmaf(c, xj, qm);
        pm = fmaf(c, vj, pm);
      }
      const float4 pr = on ? ps[lane] : make_float4(1.f, 0.f, 0.f, 0.f);
      const float qn = fmaf(pr.x, qm, pr.y * pm), pn = fmaf(pr.z, qm, pr.x * pm);
      float xb = 0.f, vb = 0.f;   // lane j: bead j again
      for (int m = 0; m < P; m++) {
        const float qq = __shfl_sync(FULL, qn, m), pp = __shfl_sync(FULL, pn, m);
        const float c = on ? Cs[lane * P + m] : 0.f;
        xb = fmaf(c, qq, xb);
        vb = fmaf(c, pp, vb);
      }
      x = xb;
      v = vb;
      if (on) reinterpret_cast<float *>(a.pos + at)[comp] = x;
      if (a.max_d2) {   // 3 d_c^2 bounds |d|^2 from above when it is the largest component's
        float d = 0.f;
        if (on) d = x - reinterpret_cast<const float *>(a.xref + at)[comp];
        float d2 = 3.f * d * d;
        if (!(d2 == d2)) d2 = __int_as_float(0x7f800000);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(FULL, d2, o));
        if (lane == 0 && d2 > 0.f) atomicMax(a.max_d2, __float_as_uint(d2));
      }
    }
    if (on) reinterpret_cast<float *>(a.vel + at)[comp] = v;
  }
  if (a.H && valid) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hacc += __shfl_xor_sync(FULL, hacc, o);
    if (lane == 0 && hacc != 0.f) atomicAdd(&hsum, (double)hacc);
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = hsum;
      if (blockIdx.x == 0)
        for (int b = 0; b < P; b++) t += a.E[b];
      atomicAdd(&a.H[k], t);
    }
  }
}

fnn_status launch_rpmd_update(fnn_ctx *ctx, const fnn_nlist *nl, int N, int P, float4 *pos, float4 *vel,
                              const float *F, const int32_t *mol_step, int nsteps, double dt, double temperature,
                              const float *C, const float4 *prop, const double *E, double *H, const float4 *xref,
                              unsigned *max_d2, cudaStream_t s) {
  if (N <= 0) return FNN_OK;
  RpmdKArgs a{};
  a.N = N;
  a.P = P;
  a.pos = pos;
  a.vel = vel;
  a.F = F;
  a.elem = nl->elem;
  a.mol_step = mol_step;
  a.nsteps = nsteps;
  a.dt = (float)dt;
  const double wP = P * KB_KCAL * temperature / HBAR_KCAL_FS;
  for (int e = 0; e < NE; e++) {
    a.acc[e] = (float)(ACCEL / MASS_AMU[e]);
    a.half_m[e] = (float)(0.5 * MASS_AMU[e] / ACCEL);
    a.half_m_wp2[e] = (float)(0.5 * MASS_AMU[e] * wP * wP / ACCEL);
  }
  a.C = C;
  a.prop = prop;
  a.E = E;
  a.H = H;
  a.xref = xref;
  a.max_d2 = max_d2;
  int blocks = (int)((3LL * N * 32 + 255) / 256);
  if (blocks > 8 * ctx->num_sms) blocks = 8 * ctx->num_sms;
  FNN_KERNEL(ctx, "rpmd_update", s);
  k_rpmd_update<<<blocks, 256, 0, s>>>(a);
  return check_launch(ctx, "rpmd_update");
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

__global__ void k_advance_steps(int n_mol, int32_t *mol_step, MdState *st) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n_mol; m += gridDim.x * blockDim.x) mol_step[m]++;
  if (st && blockIdx.x == 0 && threadIdx.x == 0) st->since_build++;
}

// positions at the rebuild: the reference of the displacement guard
__global__ void k_md_ref(int n, const float4 *pos, float4 *xref) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) xref[i] = pos[i];
}

fnn_status launch_record_energy(fnn_ctx *ctx, int n_mol, const double *E, const int32_t *mol_step,
                                const int32_t *mol_nsteps, const int64_t *hist_off, double *hist, int step,
                                int64_t stride, cudaStream_t s) {
  FNN_KERNEL(ctx, "record_energy", s);
  k_record_energy<<<(n_mol + 255) / 256, 256, 0, s>>>(n_mol, E, mol_step, mol_nsteps, hist_off, hist, step, stride);
  return check_launch(ctx, "record_energy");
}

fnn_status launch_advance_steps(fnn_ctx *ctx, int n_mol, int32_t *mol_step, MdState *st, cudaStream_t s) {
  FNN_KERNEL(ctx, "advance_steps", s);
  k_advance_steps<<<(n_mol + 255) / 256, 256, 0, s>>>(n_mol, mol_step, st);
  return check_launch(ctx, "advance_steps");
}

fnn_status launch_md_ref(fnn_ctx *ctx, int n, const float4 *pos, float4 *xref, cudaStream_t s) {
  if (n <= 0) return FNN_OK;
  int blocks = (n + 255) / 256;
  if (blocks > 4 * ctx->num_sms) blocks = 4 * ctx->num_sms;
  FNN_KERNEL(ctx, "md_ref", s);
  k_md_ref<<<blocks, 256, 0, s>>>(n, pos, xref);
  return check_launch(ctx, "md_ref");
}

// The rebuild decision before an evaluation (one thread): due by the schedule, or an atom moved more than
// skin/2 since the last rebuild (guard).  A rebuild resets the counters; the decision goes to st->need
// (read by the host between eager steps) and, in a graph, to the conditional node around the rebuild.
__global__ void k_md_decide(MdState *st, int rebuild_every, float half_skin2, int guard,
                            cudaGraphConditionalHandle handle, int set_handle) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned d2 = st->max_d2;
  if (d2 > st->max_seen) st->max_seen = d2;
  const bool due = st->since_build >= rebuild_every;
  const bool moved = guard && __uint_as_float(d2) > half_skin2;
  const int need = (due || moved) ? 1 : 0;
  if (need) {
    st->rebuilds++;
    if (!due) st->guard_rebuilds++;
    st->since_build = 0;
    st->max_d2 = 0u;
  }
  st->need = need;
  if (set_handle) cudaGraphSetConditional(handle, (unsigned)need);
}

__global__ void k_md_init(int n_mol, int32_t n_steps, int32_t *mol_step, int32_t *mol_nsteps, MdState *st,
                          int rebuild_every) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n_mol; m += gridDim.x * blockDim.x) {
    mol_step[m] = 0;
    mol_nsteps[m] = n_steps;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *st = MdState{};
    st->since_build = rebuild_every;   // the first evaluation always rebuilds
  }
}

namespace {

struct MdRun {
  fnn_ctx *ctx;
  fnn_system v;
  float *pos, *vel;
  fnn_nlist *nl;
  fnn_precision prec;
  fnn_md_options o;
  double *E, *E_hist, *K_hist;
  float *F;
  int32_t *mol_step, *mol_nsteps;
  MdState *st;
  float4 *xref;
  unsigned *max_d2;
  float half_skin2;
  // ring-polymer MD (fnn_rpmd_run): beads, temperature, normal-mode matrix and propagators, Hamiltonian
  int rp_P = 0;
  double rp_T = 0.0;
  const float *rp_C = nullptr;
  const float4 *rp_prop = nullptr;
  double *H_hist = nullptr;
};

// the rebuild itself: list, then the guard's reference positions
fnn_status md_rebuild(MdRun &r, cudaStream_t s) {
  fnn_status st = fnn_build_neighbors(r.ctx, &r.v, r.nl, s);
  if (st) return st;
  return launch_md_ref(r.ctx, r.v.n_atoms, reinterpret_cast<const float4 *>(r.pos), r.xref, s);
}

// evaluation + history + update + step counters (everything after the rebuild decision)
fnn_status md_after(MdRun &r, cudaStream_t s) {
  fnn_ctx *ctx = r.ctx;
  fnn_status st;
  if ((st = fnn_energy_forces(ctx, &r.v, r.nl, r.prec, r.E, r.F, nullptr, s))) return st;
  if (r.E_hist &&
      (st = launch_record_energy(ctx, r.v.n_mol, r.E, r.mol_step, r.mol_nsteps, nullptr, r.E_hist, 0, r.v.n_mol, s)))
    return st;
  if (r.rp_P > 0) {
    if ((st = launch_rpmd_update(ctx, r.nl, r.v.n_atoms / r.rp_P, r.rp_P, reinterpret_cast<float4 *>(r.pos),
                                 reinterpret_cast<float4 *>(r.vel), r.F, r.mol_step, r.o.n_steps, r.o.dt_fs, r.rp_T,
                                 r.rp_C, r.rp_prop, r.E, r.H_hist, r.xref, r.o.skin_guard ? r.max_d2 : nullptr, s)))
      return st;
    return launch_advance_steps(ctx, r.v.n_mol, r.mol_step, r.st, s);
  }
  MdUpdate u;
  u.mol_step = r.mol_step;
  u.mol_nsteps = r.mol_nsteps;
  u.dt = r.o.dt_fs;
  u.nsteps = r.o.n_steps;
  if (r.o.integrator == FNN_MD_LANGEVIN) {
    u.gamma = r.o.friction_per_fs;
    u.temperature = r.o.temperature_K;
    u.seed = r.o.seed;
    u.step0 = r.o.step0;
  }
  u.xref = r.xref;
  u.max_d2 = r.o.skin_guard ? r.max_d2 : nullptr;
  u.K = r.K_hist;
  u.K_stride = r.v.n_mol;
  if ((st = launch_md_update(ctx, r.nl, r.v.n_atoms, reinterpret_cast<float4 *>(r.pos),
                             reinterpret_cast<float4 *>(r.vel), r.F, u, s)))
    return st;
  return launch_advance_steps(ctx, r.v.n_mol, r.mol_step, r.st, s);
}

fnn_status md_decide(MdRun &r, cudaStream_t s, cudaGraphConditionalHandle h, int set_handle) {
  FNN_KERNEL(r.ctx, "md_decide", s);
  k_md_decide<<<1, 32, 0, s>>>(r.st, r.o.rebuild_every, r.half_skin2, r.o.skin_guard, h, set_handle);
  return check_launch(r.ctx, "md_decide");
}

// One eager step: the decision is read back (one stream synchronisation), then the rebuild if needed.
fnn_status md_step_eager(MdRun &r, cudaStream_t s, int *rebuilds) {
  fnn_ctx *ctx = r.ctx;
  fnn_status st;
  if ((st = md_decide(r, s, 0, 0))) return st;
  FNN_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->pinned_flag, &r.st->need, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FNN_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (*ctx->pinned_flag) {
    ++*rebuilds;
    if ((st = md_rebuild(r, s))) return st;
  }
  return md_after(r, s);
}

// Streams and events of the rebuild bodies' captures.  The neighbour build forks work to the context's
// side stream; by the second captured step that stream has joined the outer capture (through the energy
// call), so a body capture borrowing it would tie one stream to two capture sequences.  Each body is
// therefore captured with its own origin stream, side stream and fork/join events, swapped into the
// context for the duration of the body capture.
struct BodyCapture {
  cudaStream_t origin = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool ok() const { return origin && side && ev_fork && ev_join; }
  void create() {
    if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess) origin = nullptr;
    if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess) side = nullptr;
    if (cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess) ev_fork = nullptr;
    if (cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess) ev_join = nullptr;
    cudaGetLastError();
  }
  void destroy() {
    if (origin) cudaStreamDestroy(origin);
    if (side) cudaStreamDestroy(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    origin = side = nullptr;
    ev_fork = ev_join = nullptr;
  }
};

// One step captured: the decision kernel sets a conditional handle; an IF node holds the rebuild (captured
// into its body from the BodyCapture streams); the rest follows the node.  *body_launches receives the
// kernel launches of the rebuild body.
fnn_status md_step_capture(MdRun &r, cudaStream_t s, BodyCapture &bc, long long *body_launches) {
  fnn_ctx *ctx = r.ctx;
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  FNN_CUDA_TRY(ctx, cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive || !g) {
    ctx->last_error = "md step capture: stream is not capturing";
    return FNN_E_CUDA;
  }
  cudaGraphConditionalHandle h;
  FNN_CUDA_TRY(ctx, cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  fnn_status st;
  if ((st = md_decide(r, s, h, 1))) return st;
  FNN_CUDA_TRY(ctx, cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive || !g) {
    ctx->last_error = "md step capture: capture ended";
    return FNN_E_CUDA;
  }
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  FNN_CUDA_TRY(ctx, cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
  if (!node || !cp.conditional.phGraph_out || !cp.conditional.phGraph_out[0]) {
    ctx->last_error = "md step capture: conditional node without a body graph";
    return FNN_E_CUDA;
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  FNN_CUDA_TRY(ctx, cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  FNN_CUDA_TRY(ctx, cudaStreamBeginCaptureToGraph(bc.origin, body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal));
  const cudaStream_t side = ctx->side;
  const cudaEvent_t ef = ctx->ev_fork, ej = ctx->ev_join;
  ctx->side = bc.side;
  ctx->ev_fork = bc.ev_fork;
  ctx->ev_join = bc.ev_join;
  const long long l0 = ctx->prof.launches;
  fnn_status bs = md_rebuild(r, bc.origin);
  *body_launches = ctx->prof.launches - l0;
  ctx->side = side;
  ctx->ev_fork = ef;
  ctx->ev_join = ej;
  cudaGraph_t out = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(bc.origin, &out);
  if (bs) return bs;
  if (ec != cudaSuccess) {
    ctx->last_error = std::string("md rebuild body capture: ") + cudaGetErrorString(ec);
    return FNN_E_CUDA;
  }
  return md_after(r, s);
}

}  // namespace
}  // namespace fnn

using namespace fnn;

namespace fnn {
namespace {
struct RpmdSetup {   // ring-polymer MD: beads and temperature, and where the histories go
  int P = 0;
  double T = 0.0;
  double *H_hist = nullptr;
};

// The driver of fnn_md_run_ex and fnn_rpmd_run: scratch, the first block eagerly, whole blocks as replays of
// one captured graph with conditional rebuilds, the rest eagerly, counters.
fnn_status md_run_core(fnn_ctx *ctx, const fnn_system *sys, float *pos, float *vel, fnn_nlist *nl, fnn_precision prec,
                       const fnn_md_options *opt, double *E_hist, double *K_hist, float *F, fnn_md_counters *counters,
                       void *stream, const RpmdSetup &rp) {
  if (!ctx->pinned_flag) FNN_CUDA_TRY(ctx, cudaHostAlloc((void **)&ctx->pinned_flag, 64, cudaHostAllocDefault));
  cudaStream_t s = (cudaStream_t)stream;
  MdRun r{};
  r.ctx = ctx;
  r.v = *sys;
  r.v.pos = pos;
  r.pos = pos;
  r.vel = vel;
  r.nl = nl;
  r.prec = prec;
  r.o = *opt;
  r.E_hist = E_hist;
  r.K_hist = K_hist;
  r.F = F;
  const double hs = 0.5 * ctx->cfg.skin;
  r.half_skin2 = (float)(hs * hs);
  const int nm = r.v.n_mol > 0 ? r.v.n_mol : 1;
  const int N = r.v.n_atoms;
  // scratch: energies of the current step, per-structure step counters, the run's state, reference positions
  char *scratch = nullptr;
  const size_t off_step = ((size_t)nm * sizeof(double) + 255) & ~(size_t)255;
  const size_t off_state = (off_step + 2 * (size_t)nm * sizeof(int32_t) + 255) & ~(size_t)255;
  const size_t off_ref = (off_state + sizeof(MdState) + 255) & ~(size_t)255;
  const size_t off_rp = (off_ref + (size_t)(N > 0 ? N : 1) * sizeof(float4) + 255) & ~(size_t)255;
  const size_t bytes = off_rp + (size_t)rp.P * rp.P * sizeof(float) + (size_t)rp.P * sizeof(float4) + 16;
  FNN_CUDA_TRY(ctx, cudaMallocAsync((void **)&scratch, bytes, s));
  r.E = reinterpret_cast<double *>(scratch);
  r.mol_step = reinterpret_cast<int32_t *>(scratch + off_step);
  r.mol_nsteps = r.mol_step + nm;
  r.st = reinterpret_cast<MdState *>(scratch + off_state);
  r.max_d2 = &r.st->max_d2;
  r.xref = reinterpret_cast<float4 *>(scratch + off_ref);
  fnn_status st = FNN_OK;
  if (rp.P > 0) {
    // normal modes of the free ring polymer (real Fourier basis) and their exact one-step propagators
    const int P = rp.P;
    std::vector<float> tab((size_t)P * P + 4 * (size_t)P);
    const double wP = P * KB_KCAL * rp.T / HBAR_KCAL_FS, dt = opt->dt_fs;
    for (int j = 0; j < P; j++)
      for (int k = 0; k < P; k++) {
        double c;
        if (k == 0) c = 1.0 / sqrt((double)P);
        else if (2 * k < P) c = sqrt(2.0 / P) * cos(2.0 * M_PI * j * k / P);
        else if (2 * k == P) c = ((j & 1) ? -1.0 : 1.0) / sqrt((double)P);
        else c = sqrt(2.0 / P) * sin(2.0 * M_PI * j * k / P);
        tab[(size_t)j * P + k] = (float)c;
      }
    float *pr = tab.data() + (size_t)P * P;
    for (int k = 0; k < P; k++) {
      const double w = 2.0 * wP * sin(k * M_PI / P);
      pr[4 * k] = (float)cos(w * dt);
      pr[4 * k + 1] = (float)(w > 0 ? sin(w * dt) / w : dt);
      pr[4 * k + 2] = (float)(-w * sin(w * dt));
      pr[4 * k + 3] = 0.f;
    }
    r.rp_P = P;
    r.rp_T = rp.T;
    r.rp_C = reinterpret_cast<const float *>(scratch + off_rp);
    r.rp_prop = reinterpret_cast<const float4 *>(scratch + off_rp + (((size_t)P * P * sizeof(float) + 15) & ~(size_t)15));
    r.H_hist = rp.H_hist;
    // pageable source: the copies complete before the calls return, so tab may go out of scope
    cudaError_t e = cudaMemcpyAsync(const_cast<float *>(r.rp_C), tab.data(), (size_t)P * P * sizeof(float),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(const_cast<float4 *>(r.rp_prop), pr, (size_t)P * sizeof(float4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && rp.H_hist && opt->n_steps > 0)
      e = cudaMemsetAsync(rp.H_hist, 0, (size_t)opt->n_steps * sizeof(double), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFreeAsync(scratch, s);
      ctx->last_error = "ring-polymer tables";
      return FNN_E_CUDA;
    }
  }
  if (K_hist && opt->n_steps > 0) {
    const cudaError_t e = cudaMemsetAsync(K_hist, 0, (size_t)opt->n_steps * nm * sizeof(double), s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFreeAsync(scratch, s);
      ctx->last_error = "K_hist clear failed";
      return FNN_E_CUDA;
    }
  }
  {
    FNN_KERNEL(ctx, "md_init", s);
    k_md_init<<<(nm + 255) / 256, 256, 0, s>>>(nm, opt->n_steps, r.mol_step, r.mol_nsteps, r.st, opt->rebuild_every);
  }
  const int n_steps = opt->n_steps, B = opt->rebuild_every;
  long long scheduled_rebuild_launches = 0;   // graph replays: launches counted as if rebuilt on schedule
  long long body_launches = 0;
  int k = 0;
  // the first block eagerly (sizes every buffer, calibrates the FP8 form)
  int eager_rebuilds = 0;
  for (; k < n_steps && k < B && !st; k++) st = md_step_eager(r, s, &eager_rebuilds);
  // whole blocks of B steps as replays of one CUDA graph, when the stream can be captured
  int graph_blocks = 0;
  if (!st && s && n_steps - k >= 2 * B) {
    const long long l0 = ctx->prof.launches;
    const bool prof = ctx->prof.on;
    ctx->prof.on = false;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    BodyCapture bc;
    bc.create();
    long long body_total = 0;
    if (bc.ok() && cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      fnn_status cs = FNN_OK;
      for (int j = 0; j < B && !cs; j++) {
        long long bl = 0;
        cs = md_step_capture(r, s, bc, &bl);
        body_total += bl;
      }
      const cudaError_t ec = cudaStreamEndCapture(s, &g);
      if (cs || ec != cudaSuccess || !g || cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
    }
    cudaGetLastError();
    nl->stream = s;   // the capture recorded the rebuild on the helper stream, which is gone
    ctx->prof.on = prof;
    const long long per_block = ctx->prof.launches - l0 - body_total;   // without the rebuild bodies
    body_launches = B > 0 ? body_total / B : 0;
    ctx->prof.launches = l0;
    if (exec) {
      for (; n_steps - k >= B; k += B) {
        if (cudaGraphLaunch(exec, s) != cudaSuccess) {
          cudaGetLastError();
          ctx->last_error = "cudaGraphLaunch failed";
          st = FNN_E_CUDA;
          break;
        }
        ctx->prof.launches += per_block;
        scheduled_rebuild_launches += body_launches;
        graph_blocks++;
      }
      cudaGraphExecDestroy(exec);
    }
    if (g) cudaGraphDestroy(g);
    bc.destroy();   // after the replays: the graph's bodies were recorded from these streams
  }
  // the rest eagerly (also every step when the stream cannot be captured)
  for (; k < n_steps && !st; k++) st = md_step_eager(r, s, &eager_rebuilds);
  if (!st && counters) {
    MdState h{};
    cudaError_t e = cudaMemcpyAsync(ctx->pinned_flag, r.st, sizeof(MdState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      st = FNN_E_CUDA;
    } else {
      memcpy(&h, ctx->pinned_flag, sizeof(MdState));
      float d2;
      memcpy(&d2, &h.max_seen, sizeof(float));
      counters->rebuilds = h.rebuilds;
      counters->guard_rebuilds = h.guard_rebuilds;
      counters->max_displacement = sqrt((double)d2);
      counters->graph_blocks = graph_blocks;
      // the replays' rebuild bodies that ran (the eager steps counted theirs as they launched)
      ctx->prof.launches += (long long)(h.rebuilds - eager_rebuilds) * body_launches;
      scheduled_rebuild_launches = 0;
    }
  }
  // without counters, replays count their rebuild bodies as if rebuilt on schedule (once per block)
  ctx->prof.launches += scheduled_rebuild_launches;
  cudaFreeAsync(scratch, s);
  return st;
}

}  // namespace
}  // namespace fnn

extern "C" fnn_status fnn_md_run_ex(fnn_ctx *ctx, const fnn_system *sys, float *pos, float *vel, fnn_nlist *nl,
                                    fnn_precision prec, const fnn_md_options *opt, double *E_hist, double *K_hist,
                                    float *F, fnn_md_counters *counters, void *stream) {
  if (!ctx || !sys || !pos || !vel || !nl || !F || !opt || opt->n_steps < 0 || !(opt->dt_fs > 0) ||
      opt->rebuild_every < 1 || ((uintptr_t)pos & 15) || ((uintptr_t)vel & 15) ||
      (opt->integrator != FNN_MD_NVE && opt->integrator != FNN_MD_LANGEVIN) ||
      (opt->integrator == FNN_MD_LANGEVIN && (!(opt->friction_per_fs > 0) || !(opt->temperature_K >= 0))))
    return FNN_E_INVALID;
  return md_run_core(ctx, sys, pos, vel, nl, prec, opt, E_hist, K_hist, F, counters, stream, RpmdSetup{});
}

extern "C" fnn_status fnn_rpmd_run(fnn_ctx *ctx, const fnn_system *beads, float *pos, float *vel, fnn_nlist *nl,
                                   fnn_precision prec, const fnn_rpmd_options *opt, double *E_hist, double *H_hist,
                                   float *F, fnn_md_counters *counters, void *stream) {
  if (!ctx || !beads || !pos || !vel || !nl || !F || !opt || opt->n_beads < 1 || opt->n_beads > FNN_RPMD_MAX_BEADS ||
      beads->n_mol != opt->n_beads || beads->n_atoms % opt->n_beads != 0 || opt->n_steps < 0 ||
      !(opt->dt_fs > 0) || !(opt->temperature_K > 0) || opt->rebuild_every < 1 || ((uintptr_t)pos & 15) ||
      ((uintptr_t)vel & 15))
    return FNN_E_INVALID;
  fnn_md_options o{};
  o.n_steps = opt->n_steps;
  o.dt_fs = opt->dt_fs;
  o.rebuild_every = opt->rebuild_every;
  o.skin_guard = opt->skin_guard;
  o.integrator = FNN_MD_NVE;
  RpmdSetup rp;
  rp.P = opt->n_beads;
  rp.T = opt->temperature_K;
  rp.H_hist = H_hist;
  return md_run_core(ctx, beads, pos, vel, nl, prec, &o, E_hist, nullptr, F, counters, stream, rp);
}

extern "C" fnn_status fnn_md_run(fnn_ctx *ctx, const fnn_system *sys, float *pos, float *vel, fnn_nlist *nl,
                                 fnn_precision prec, int32_t n_steps, double dt_fs, int32_t rebuild_every,
                                 double *E_hist, float *F, void *stream) {
  fnn_md_options o{};
  o.n_steps = n_steps;
  o.dt_fs = dt_fs;
  o.rebuild_every = rebuild_every;
  o.skin_guard = 1;
  o.integrator = FNN_MD_NVE;
  return fnn_md_run_ex(ctx, sys, pos, vel, nl, prec, &o, E_hist, nullptr, F, nullptr, stream);
}
