// CRATE angular resource of the first interaction layer (Appendix A, angular resources) and its
// vector-Jacobian product.
//
//   D_ij[c] = f~(r_ij) sum_a B~_a(r_ij) V[e(j)][a][c]       B~_a(r) = exp(-eta_ang (r - A_a)^2), a < 8
//   g_i[n][c] = sum_{j<k} T_n(cos theta_jik) D_ij[c] D_ik[c]   T_n: Chebyshev, T_n(cos t) = cos(n t), n < 4
//
// over the neighbours of i within rc_ang (unordered pairs of distinct list entries), with the context's
// switching function f~ at rc_ang and the angular radial shifts A_a of the ANI constants.  One warp per
// centre atom: its neighbours within rc_ang are staged in shared memory (positions relative to i, unit
// vectors, switch values), D is built with the 32 channels across the lanes, and the triplets run with
// lanes over channels for the products (the Chebyshev values of one row of pairs broadcast from shared
// memory) and lanes over pairs for the angle derivative (a padded shared buffer reduces over channels).
#include "fnn_internal.cuh"

namespace fnn {

static constexpr unsigned CFULL = 0xffffffffu;
constexpr int CR_NB = FNN_CRATE_NB, CR_DA = FNN_CRATE_DA, CR_NT = FNN_CRATE_NT;
static_assert(CR_DA == 32, "one channel per lane");
constexpr int CR_CAP = ANG_CAP;           // neighbours within rc_ang per atom
constexpr int CR_FWD_WARPS = 4, CR_VJP_WARPS = 4;

struct CrateNbr {   // one centre atom's neighbours within rc_ang, in list order
  float4 u[CR_CAP];      // unit vector to the neighbour, distance
  float f[CR_CAP];       // switch f~(r)
  float df[CR_CAP];      // its derivative
  int j[CR_CAP];         // neighbour atom
  unsigned char e[CR_CAP];
};

struct CrateArgs {
  const float4 *pos;
  const int32_t *row_ptr, *nbr;
  const char4 *shift;
  const uint8_t *elem;
  const int32_t *atom_mol;
  const MolGrid *grid;
  int64_t cap;
  int n_atoms;
  AevParams P;
  const float *V;        // [7][8][32]
  float *g;              // forward: [N][4][32]
  const float *G;        // adjoint: dL/dg [N][4][32]
  float *gx;             // adjoint: dL/dx [N][3] (zeroed by the host)
  float *gV;             // adjoint: dL/dV [7][8][32] (zeroed by the host), or NULL
  DevStatus *st;
};

// Stage atom i's neighbours within rc_ang; returns their count, or -1 (after posting FNN_E_CAPACITY with
// info -(i + 1)) when there are more than CR_CAP, or -1 for an atom outside every structure.
__device__ int crate_stage(const CrateArgs &A, int i, CrateNbr &S) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int mol = A.atom_mol[i];
  if (mol < 0) return -1;
  const float4 pi = A.pos[i];
  const MolGrid g = A.grid[mol];
  const float Lx = g.pbc ? g.Lx : 0.f, Ly = g.pbc ? g.Ly : 0.f, Lz = g.pbc ? g.Lz : 0.f;
  const int k0 = (int)min((int64_t)A.row_ptr[i], A.cap), k1 = (int)min((int64_t)A.row_ptr[i + 1], A.cap);
  const float rc = A.P.rc_ang;
  int n = 0;
  for (int kb = k0; kb < k1; kb += 32) {
    const int k = kb + lane;
    bool in = false;
    float dx = 0.f, dy = 0.f, dz = 0.f, r = 0.f;
    int j = 0;
    if (k < k1) {
      j = A.nbr[k];
      const char4 sh = A.shift[k];
      const float4 pj = A.pos[j];
      dx = (pj.x - pi.x) + (float)sh.x * Lx;
      dy = (pj.y - pi.y) + (float)sh.y * Ly;
      dz = (pj.z - pi.z) + (float)sh.z * Lz;
      r = sqrtf(dx * dx + dy * dy + dz * dz);
      in = r < rc;
    }
    const unsigned m = __ballot_sync(CFULL, in);
    const int at = n + __popc(m & lt);
    if (in && at < CR_CAP) {
      const float ir = 1.f / r;
      S.u[at] = make_float4(dx * ir, dy * ir, dz * ir, r);
      S.f[at] = switch_f(A.P, r, rc, A.P.inv_rc_ang);
      S.df[at] = switch_df(A.P, r, rc, A.P.inv_rc_ang, A.P.pi_rc_ang);
      S.j[at] = j;
      S.e[at] = A.elem[j];
    }
    n += __popc(m);
  }
  if (n > CR_CAP) {
    if (lane == 0) post_status(A.st, FNN_E_CAPACITY, -(long long)(i + 1));
    return -1;
  }
  __syncwarp();
  return n;
}

// lane c: D[t][c] for every staged neighbour t (and, for the adjoint, dD/dr into dDdr[t][c])
__device__ __forceinline__ void crate_build_D(const CrateArgs &A, const CrateNbr &S, int n, const float *Vs,
                                              float (*D)[CR_DA], float (*dDdr)[CR_DA]) {
  const int c = threadIdx.x & 31;
  for (int t = 0; t < n; t++) {
    const float r = S.u[t].w;
    const float *v = Vs + (int)S.e[t] * CR_NB * CR_DA + c;
    float sb = 0.f, sbd = 0.f;
#pragma unroll
    for (int a = 0; a < CR_NB; a++) {
      const float dr = r - A.P.shf_a[a];
      const float b = __expf(-A.P.eta_a * dr * dr);
      sb = fmaf(b, v[a * CR_DA], sb);
      sbd = fmaf(-2.f * A.P.eta_a * dr * b, v[a * CR_DA], sbd);
    }
    D[t][c] = S.f[t] * sb;
    if (dDdr) dDdr[t][c] = S.df[t] * sb + S.f[t] * sbd;
  }
  __syncwarp();
}

struct CrateFwdWarp {
  CrateNbr nb;
  float D[CR_CAP][CR_DA];
  float4 row[32];        // T1, T2, T3 of one row of pairs
};

__global__ void __launch_bounds__(CR_FWD_WARPS * 32) k_crate_forward(CrateArgs A) {
  __shared__ float Vs[NE * CR_NB * CR_DA];
  extern __shared__ __align__(16) unsigned char crate_fwd_dyn[];
  CrateFwdWarp *Wsh = reinterpret_cast<CrateFwdWarp *>(crate_fwd_dyn);
  for (int k = threadIdx.x; k < NE * CR_NB * CR_DA; k += blockDim.x) Vs[k] = A.V[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  CrateFwdWarp &W = Wsh[warp];
  for (int i = blockIdx.x * CR_FWD_WARPS + warp; i < A.n_atoms; i += gridDim.x * CR_FWD_WARPS) {
    const int n = crate_stage(A, i, W.nb);
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
    if (n > 1) {
      crate_build_D(A, W.nb, n, Vs, W.D, nullptr);
      for (int j = 0; j + 1 < n; j++) {
        const float Dj = W.D[j][lane];
        const float4 uj = W.nb.u[j];
        for (int k0 = j + 1; k0 < n; k0 += 32) {
          const int k = k0 + lane;
          if (k < n) {
            const float4 uk = W.nb.u[k];
            const float c = uj.x * uk.x + uj.y * uk.y + uj.z * uk.z;
            W.row[lane] = make_float4(c, 2.f * c * c - 1.f, (4.f * c * c - 3.f) * c, 0.f);
          }
          __syncwarp();
          const int m = min(32, n - k0);
          for (int q = 0; q < m; q++) {
            const float p = Dj * W.D[k0 + q][lane];
            const float4 t = W.row[q];
            acc0 += p;
            acc1 = fmaf(t.x, p, acc1);
            acc2 = fmaf(t.y, p, acc2);
            acc3 = fmaf(t.z, p, acc3);
          }
          __syncwarp();
        }
      }
    }
    // (an atom beyond the neighbour limit gets zeros; its FNN_E_CAPACITY is posted)
    float *out = A.g + (size_t)i * CR_NT * CR_DA + lane;
    out[0] = acc0;
    out[CR_DA] = acc1;
    out[2 * CR_DA] = acc2;
    out[3 * CR_DA] = acc3;
    __syncwarp();
  }
}

struct CrateVjpWarp {
  CrateNbr nb;
  float D[CR_CAP][CR_DA];
  float dD[CR_CAP][CR_DA];     // dL/dD per neighbour and channel
  float4 row[32];              // T1, T2, T3 of one row of pairs
  float4 drow[32];             // dT1/dc, dT2/dc, dT3/dc
  float h[32][CR_DA + 1];      // per pair of the row, per channel: the angle derivative's terms (padded)
  float gd[CR_CAP][3];         // dL/dd per neighbour (d = x_j - x_i)
};

__global__ void __launch_bounds__(CR_VJP_WARPS * 32) k_crate_vjp(CrateArgs A) {
  __shared__ float Vs[NE * CR_NB * CR_DA];
  __shared__ float gVs[NE * CR_NB * CR_DA];
  extern __shared__ __align__(16) unsigned char crate_dyn[];
  CrateVjpWarp *Wsh = reinterpret_cast<CrateVjpWarp *>(crate_dyn);
  for (int k = threadIdx.x; k < NE * CR_NB * CR_DA; k += blockDim.x) {
    Vs[k] = A.V[k];
    gVs[k] = 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  CrateVjpWarp &W = Wsh[warp];
  for (int i = blockIdx.x * CR_VJP_WARPS + warp; i < A.n_atoms; i += gridDim.x * CR_VJP_WARPS) {
    const int n = crate_stage(A, i, W.nb);
    if (n < 2) continue;   // uniform over the warp
    crate_build_D(A, W.nb, n, Vs, W.D, nullptr);
    const float *Gi = A.G + (size_t)i * CR_NT * CR_DA + lane;
    const float G0 = Gi[0], G1 = Gi[CR_DA], G2 = Gi[2 * CR_DA], G3 = Gi[3 * CR_DA];
    for (int t = 0; t < n; t++) W.dD[t][lane] = 0.f;
    for (int t = lane; t < n; t += 32) W.gd[t][0] = W.gd[t][1] = W.gd[t][2] = 0.f;
    __syncwarp();
    for (int j = 0; j + 1 < n; j++) {
      const float Dj = W.D[j][lane];
      const float4 uj = W.nb.u[j];
      float dDj = 0.f;
      float gjx = 0.f, gjy = 0.f, gjz = 0.f;   // lane kk's share of dL/dd_j through the angles
      for (int k0 = j + 1; k0 < n; k0 += 32) {
        const int k = k0 + lane;
        float c = 0.f;
        float4 uk = make_float4(0.f, 0.f, 0.f, 1.f);
        if (k < n) {
          uk = W.nb.u[k];
          c = uj.x * uk.x + uj.y * uk.y + uj.z * uk.z;
          W.row[lane] = make_float4(c, 2.f * c * c - 1.f, (4.f * c * c - 3.f) * c, 0.f);
          W.drow[lane] = make_float4(1.f, 4.f * c, 12.f * c * c - 3.f, 0.f);
        }
        __syncwarp();
        const int m = min(32, n - k0);
        // lanes over channels: dL/dD of both ends, and each pair's per-channel angle term
        for (int q = 0; q < m; q++) {
          const float Dk = W.D[k0 + q][lane];
          const float4 t = W.row[q], dt = W.drow[q];
          const float w = fmaf(G3, t.z, fmaf(G2, t.y, fmaf(G1, t.x, G0)));
          dDj = fmaf(w, Dk, dDj);
          W.dD[k0 + q][lane] = fmaf(w, Dj, W.dD[k0 + q][lane]);
          W.h[q][lane] = fmaf(G3, dt.z, fmaf(G2, dt.y, G1 * dt.x)) * Dj * Dk;
        }
        __syncwarp();
        // lanes over pairs: dL/dc of pair (j, k) summed over channels, chained to both unit vectors
        if (lane < m) {
          float hs = 0.f;
#pragma unroll 8
          for (int cc = 0; cc < CR_DA; cc++) hs += W.h[lane][cc];
          const float rj = uj.w, rk = uk.w;
          // dc/dd_j = (u_k - c u_j) / r_j, dc/dd_k = (u_j - c u_k) / r_k
          const float sj = hs / rj, sk = hs / rk;
          gjx = fmaf(sj, uk.x - c * uj.x, gjx);
          gjy = fmaf(sj, uk.y - c * uj.y, gjy);
          gjz = fmaf(sj, uk.z - c * uj.z, gjz);
          W.gd[k][0] = fmaf(sk, uj.x - c * uk.x, W.gd[k][0]);
          W.gd[k][1] = fmaf(sk, uj.y - c * uk.y, W.gd[k][1]);
          W.gd[k][2] = fmaf(sk, uj.z - c * uk.z, W.gd[k][2]);
        }
        __syncwarp();
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        gjx += __shfl_xor_sync(CFULL, gjx, o);
        gjy += __shfl_xor_sync(CFULL, gjy, o);
        gjz += __shfl_xor_sync(CFULL, gjz, o);
      }
      W.dD[j][lane] += dDj;
      if (lane == 0) {
        W.gd[j][0] += gjx;
        W.gd[j][1] += gjy;
        W.gd[j][2] += gjz;
      }
      __syncwarp();
    }
    // per neighbour: dL/dr through D (summed over channels), and dL/dV
    for (int t = 0; t < n; t++) {
      const float dDt = W.dD[t][lane];
      // dD/dr of this channel, recomputed: f~' sum_a B~_a V + f~ sum_a B~_a' V
      const float r = W.nb.u[t].w;
      const float *v = Vs + (int)W.nb.e[t] * CR_NB * CR_DA + lane;
      float sb = 0.f, sbd = 0.f;
#pragma unroll
      for (int a = 0; a < CR_NB; a++) {
        const float dr = r - A.P.shf_a[a];
        const float bb = __expf(-A.P.eta_a * dr * dr);
        sb = fmaf(bb, v[a * CR_DA], sb);
        sbd = fmaf(-2.f * A.P.eta_a * dr * bb, v[a * CR_DA], sbd);
      }
      float s = dDt * (W.nb.df[t] * sb + W.nb.f[t] * sbd);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(CFULL, s, o);
      if (lane == 0) {
        const float4 u = W.nb.u[t];
        W.gd[t][0] = fmaf(s, u.x, W.gd[t][0]);
        W.gd[t][1] = fmaf(s, u.y, W.gd[t][1]);
        W.gd[t][2] = fmaf(s, u.z, W.gd[t][2]);
      }
      if (A.gV) {
        const float ft = W.nb.f[t] * dDt;
        float *gv = gVs + (int)W.nb.e[t] * CR_NB * CR_DA + lane;
#pragma unroll
        for (int a = 0; a < CR_NB; a++) {
          const float dr = r - A.P.shf_a[a];
          atomicAdd(gv + a * CR_DA, ft * __expf(-A.P.eta_a * dr * dr));
        }
      }
    }
    __syncwarp();
    // scatter: d = x_j - x_i + shift, so dL/dx_j += dL/dd and dL/dx_i -= dL/dd
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int t = lane; t < n; t += 32) {
      const float gx = W.gd[t][0], gy = W.gd[t][1], gz = W.gd[t][2];
      const int jj = W.nb.j[t];
      atomicAdd(A.gx + 3 * (size_t)jj, gx);
      atomicAdd(A.gx + 3 * (size_t)jj + 1, gy);
      atomicAdd(A.gx + 3 * (size_t)jj + 2, gz);
      sx += gx;
      sy += gy;
      sz += gz;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(CFULL, sx, o);
      sy += __shfl_xor_sync(CFULL, sy, o);
      sz += __shfl_xor_sync(CFULL, sz, o);
    }
    if (lane == 0) {
      atomicAdd(A.gx + 3 * (size_t)i, -sx);
      atomicAdd(A.gx + 3 * (size_t)i + 1, -sy);
      atomicAdd(A.gx + 3 * (size_t)i + 2, -sz);
    }
    __syncwarp();
  }
  if (A.gV) {
    __syncthreads();
    for (int k = threadIdx.x; k < NE * CR_NB * CR_DA; k += blockDim.x)
      if (gVs[k] != 0.f) atomicAdd(A.gV + k, gVs[k]);
  }
}

static CrateArgs crate_args(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *V) {
  CrateArgs a{};
  a.pos = reinterpret_cast<const float4 *>(sys->pos);
  a.row_ptr = nl->row_ptr;
  a.nbr = nl->nbr;
  a.shift = nl->shift;
  a.elem = nl->elem;
  a.atom_mol = nl->atom_mol;
  a.grid = nl->grid;
  a.cap = nl->capacity;
  a.n_atoms = sys->n_atoms;
  a.P = ctx->aev;
  a.V = V;
  a.st = ctx->status;
  return a;
}

static int crate_grid(fnn_ctx *ctx, int n_atoms, int warps, int per_sm) {
  int blocks = (n_atoms + warps - 1) / warps;
  const int cap = per_sm * ctx->num_sms;
  return blocks < cap ? (blocks > 0 ? blocks : 1) : cap;
}

static fnn_status crate_check(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl) {
  if (!ctx || !sys || !nl || nl->ctx != ctx) return FNN_E_INVALID;
  if (!nl->built || nl->n_atoms != sys->n_atoms || nl->n_mol != sys->n_mol) {
    ctx->last_error = "neighbour list was not built for this system";
    return FNN_E_STATE;
  }
  return FNN_OK;
}

}  // namespace fnn

using namespace fnn;

extern "C" fnn_status fnn_crate_angular(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *V,
                                        float *g, void *stream) {
  fnn_status st = crate_check(ctx, sys, nl);
  if (st) return st;
  if (!V || (!g && sys->n_atoms > 0)) return FNN_E_INVALID;
  if (sys->n_atoms == 0) return FNN_OK;
  cudaStream_t s = (cudaStream_t)stream;
  CrateArgs a = crate_args(ctx, sys, nl, V);
  a.g = g;
  const size_t dyn = CR_FWD_WARPS * sizeof(CrateFwdWarp);
  static bool attr_set = false;   // per-warp staging beyond the 48 KB default needs the opt-in
  if (!attr_set) {
    FNN_CUDA_TRY(ctx, cudaFuncSetAttribute(k_crate_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    attr_set = true;
  }
  {
    FNN_KERNEL(ctx, "crate_forward", s);
    k_crate_forward<<<crate_grid(ctx, sys->n_atoms, CR_FWD_WARPS, 4), CR_FWD_WARPS * 32, dyn, s>>>(a);
  }
  return check_launch(ctx, "crate_forward");
}

extern "C" fnn_status fnn_crate_angular_vjp(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *V,
                                            const float *G, float *grad_x, float *grad_V, void *stream) {
  fnn_status st = crate_check(ctx, sys, nl);
  if (st) return st;
  if (!V || (sys->n_atoms > 0 && (!G || !grad_x))) return FNN_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (grad_V) FNN_CUDA_TRY(ctx, cudaMemsetAsync(grad_V, 0, NE * CR_NB * CR_DA * sizeof(float), s));
  if (sys->n_atoms == 0) return FNN_OK;
  FNN_CUDA_TRY(ctx, cudaMemsetAsync(grad_x, 0, (size_t)sys->n_atoms * 3 * sizeof(float), s));
  CrateArgs a = crate_args(ctx, sys, nl, V);
  a.G = G;
  a.gx = grad_x;
  a.gV = grad_V;
  const size_t dyn = CR_VJP_WARPS * sizeof(CrateVjpWarp);
  static bool attr_set = false;   // the dynamic shared memory above 48 KB needs the opt-in
  if (!attr_set) {
    FNN_CUDA_TRY(ctx, cudaFuncSetAttribute(k_crate_vjp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    attr_set = true;
  }
  {
    FNN_KERNEL(ctx, "crate_vjp", s);
    k_crate_vjp<<<crate_grid(ctx, sys->n_atoms, CR_VJP_WARPS, 2), CR_VJP_WARPS * 32, dyn, s>>>(a);
  }
  return check_launch(ctx, "crate_vjp");
}
