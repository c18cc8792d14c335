// C ABI: contexts, parameters, workspaces and the energy / force entry points.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fnn_internal.cuh"

namespace fnn {

fnn_status check_launch(fnn_ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return FNN_E_CUDA;
  }
  return FNN_OK;
}

static cudaEvent_t take_event(Profiler &P) {
  if (!P.pool.empty()) {
    cudaEvent_t e = P.pool.back();
    P.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

KScope::KScope(fnn_ctx *c, const char *name, cudaStream_t st) : ctx(c), s(st) {
  ctx->prof.launches++;
  if (ctx->prof.on) {
    Profiler::Rec r{name, take_event(ctx->prof), take_event(ctx->prof)};
    cudaEventRecord(r.a, s);
    idx = (int)ctx->prof.recs.size();
    ctx->prof.recs.push_back(r);
  }
}

KScope::~KScope() {
  if (idx >= 0) cudaEventRecord(ctx->prof.recs[idx].b, s);
}

template <typename T>
static fnn_status dalloc(fnn_ctx *ctx, T **p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void **)p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    ctx->last_error = "cudaMalloc failed";
    return FNN_E_OOM;
  }
  return FNN_OK;
}

fnn_status ensure_workspace(fnn_ctx *ctx, size_t rows) {
  Workspace &ws = ctx->ws;
  const int M = ctx->w.M;
  if (rows <= ws.rows && M == ws.M) return FNN_OK;
  ctx->gen++;
  rows = rows + rows / 8;  // headroom against small growth
  fnn_status st;
  if ((st = dalloc(ctx, &ws.aev, rows * NAEV)) || (st = dalloc(ctx, &ws.h1, rows * M * H1)) ||
      (st = dalloc(ctx, &ws.h2, rows * M * H2)) || (st = dalloc(ctx, &ws.g3, rows * M * H3)) ||
      (st = dalloc(ctx, &ws.g2, rows * M * H2)) || (st = dalloc(ctx, &ws.g1, rows * M * H1)) ||
      (st = dalloc(ctx, &ws.gaev, rows * NAEV)) || (st = dalloc(ctx, &ws.ypart, rows * M * 4)) ||
      (st = dalloc(ctx, &ws.e_part, rows)) || (st = dalloc(ctx, &ws.e_ticket, rows))) {
    ws.rows = 0;
    return st;
  }
  cudaMemset(ws.ypart, 0, rows * M * 4 * sizeof(float));
  cudaMemset(ws.e_ticket, 0, rows * sizeof(unsigned));
  ws.rows = rows;
  ws.M = M;
  return FNN_OK;
}

static void free_weights(DeviceWeights &w) {
  float *ptrs[] = {w.W1cat, w.b1cat, w.W1Tcat, w.W2, w.b2, w.W2T, w.W3, w.b3, w.W3T, w.w4, w.b4};
  for (float *p : ptrs)
    if (p) cudaFree(p);
  void *tc = w.tc;
  w = DeviceWeights();
  w.tc = tc;
}

static void free_workspace(Workspace &ws) {
  float *ptrs[] = {ws.aev, ws.h1, ws.h2, ws.g3, ws.g2, ws.g1, ws.gaev, ws.ypart};
  for (float *p : ptrs)
    if (p) cudaFree(p);
  if (ws.e_part) cudaFree(ws.e_part);
  if (ws.e_ticket) cudaFree(ws.e_ticket);
  void *tc = ws.tc;
  size_t tr = ws.tc_rows;
  ws = Workspace();
  ws.tc = tc;
  ws.tc_rows = tr;
}

template <typename T>
static fnn_status upload(fnn_ctx *ctx, T **dst, const std::vector<T> &src) {
  fnn_status st = dalloc(ctx, dst, src.size());
  if (st) return st;
  FNN_CUDA_TRY(ctx, cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FNN_OK;
}

}  // namespace fnn

using namespace fnn;

extern "C" void fnn_config_default(fnn_config *c) {
  if (!c) return;
  c->rc_rad = 5.1;
  c->rc_ang = 3.5;
  c->eta_rad = 19.7;
  c->eta_ang = 12.5;
  c->zeta = 14.1;
  c->shift_rad0 = 0.8;
  c->shift_ang0 = 0.8;
  c->skin = 0.0;
  c->n_members = 1;
  c->switch_kind = FNN_SWITCH_COSINE;
  c->switch_p = 6.0;
}

extern "C" fnn_status fnn_create(fnn_ctx **out, const fnn_config *cfg) {
  if (!out || !cfg) return FNN_E_INVALID;
  *out = nullptr;
  const fnn_config &c = *cfg;
  if (!(c.rc_rad > 0) || !(c.rc_ang > 0) || c.rc_ang > c.rc_rad || !(c.eta_rad >= 0) || !(c.eta_ang >= 0) ||
      !(c.zeta >= 0) || !(c.skin >= 0) || c.n_members < 1 || c.n_members > MAXM || !(c.shift_rad0 < c.rc_rad) ||
      !(c.shift_ang0 < c.rc_ang) || c.switch_kind < FNN_SWITCH_COSINE || c.switch_kind > FNN_SWITCH_EXPONENTIAL ||
      !(c.switch_p > 0))
    return FNN_E_INVALID;
  fnn_ctx *ctx = new fnn_ctx();
  ctx->cfg = c;
  cudaGetDevice(&ctx->device);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (ctx->num_sms <= 0) ctx->num_sms = 148;
  AevParams &P = ctx->aev;
  P.rc_rad = (float)c.rc_rad;
  P.rc_ang = (float)c.rc_ang;
  P.eta_r = (float)c.eta_rad;
  P.eta_a = (float)c.eta_ang;
  P.zeta = (float)c.zeta;
  P.pi_rc_rad = (float)(M_PI / c.rc_rad);
  P.pi_rc_ang = (float)(M_PI / c.rc_ang);
  P.inv_rc_rad = (float)(1.0 / c.rc_rad);
  P.inv_rc_ang = (float)(1.0 / c.rc_ang);
  for (int k = 0; k < NSR; k++) P.shf_r[k] = (float)(c.shift_rad0 + k * (c.rc_rad - c.shift_rad0) / NSR);
  for (int m = 0; m < NSA; m++) P.shf_a[m] = (float)(c.shift_ang0 + m * (c.rc_ang - c.shift_ang0) / NSA);
  for (int s = 0; s < NSZ; s++) {
    double th = M_PI / 8.0 + s * M_PI / 4.0;
    P.cos_z[s] = (float)cos(th);
    P.sin_z[s] = (float)sin(th);
    P.hcos_z[s] = (float)(0.5 * cos(th));
    P.hsin_z[s] = (float)(0.5 * sin(th));
    P.qcos_z[s] = (float)(0.475 * cos(th));
  }
  P.eta_a_l2 = (float)(-c.eta_ang / M_LN2);
  P.eta_r_l2 = (float)(-c.eta_rad / M_LN2);
  for (int k = 0; k < NSR / 2; k++) P.nshr2[k] = make_float2(-P.shf_r[2 * k], -P.shf_r[2 * k + 1]);
  for (int m = 0; m < NSA / 2; m++) P.nsha2[m] = make_float2(-P.shf_a[2 * m], -P.shf_a[2 * m + 1]);
  for (int s = 0; s < NSZ / 2; s++) {
    P.hcos2[s] = make_float2(P.hcos_z[2 * s], P.hcos_z[2 * s + 1]);
    P.hsin2[s] = make_float2(P.hsin_z[2 * s], P.hsin_z[2 * s + 1]);
    P.qcos2[s] = make_float2(P.qcos_z[2 * s], P.qcos_z[2 * s + 1]);
  }
  P.sw_kind = c.switch_kind;
  {
    const double p = c.switch_p;
    P.sw_pm1 = (float)(p - 1.0);
    P.sw_c0 = (float)(-0.5 * (p + 1.0) * (p + 2.0));
    P.sw_c1 = (float)(p * (p + 2.0));
    P.sw_c2 = (float)(-0.5 * p * (p + 1.0));
    P.sw_k = (float)(0.5 * p * (p + 1.0) * (p + 2.0));
  }
  if (cudaMalloc(&ctx->status, sizeof(DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return FNN_E_OOM;
  }
  cudaMemset(ctx->status, 0, sizeof(DevStatus));
  if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    fnn_destroy(ctx);
    return FNN_E_CUDA;
  }
  *out = ctx;
  return FNN_OK;
}

namespace fnn {
fnn_status side_fork(fnn_ctx *ctx, cudaStream_t s) {
  FNN_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_fork, s));
  FNN_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  return FNN_OK;
}
fnn_status side_join(fnn_ctx *ctx, cudaStream_t s) {
  FNN_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_join, ctx->side));
  FNN_CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->ev_join, 0));
  return FNN_OK;
}
}  // namespace fnn

extern "C" fnn_status fnn_destroy(fnn_ctx *ctx) {
  if (!ctx) return FNN_E_INVALID;
  cudaDeviceSynchronize();
  free_weights(ctx->w);
  free_workspace(ctx->ws);
  free_tc(ctx);
  free_train(ctx);
  auto &h = ctx->host;
  void *hp[] = {h.Z, h.mol_offsets, h.pos, h.cell, h.pbc, h.pos3, h.E, h.virial, h.F};
  for (void *p : hp)
    if (p) cudaFree(p);
  if (h.graph) fnn_graph_destroy(h.graph);
  if (ctx->pinned_flag) cudaFreeHost(ctx->pinned_flag);
  if (ctx->grid_bar) cudaFree(ctx->grid_bar);
  if (h.nl) fnn_nlist_destroy(h.nl);
  if (h.own) cudaStreamDestroy(h.own);
  if (h.status) cudaFreeHost(h.status);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->status) cudaFree(ctx->status);
  for (auto &r : ctx->prof.recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
  delete ctx;
  return FNN_OK;
}

extern "C" const char *fnn_last_error(const fnn_ctx *ctx) {
  if (!ctx) return "null context";
  return ctx->last_error.c_str();
}

static fnn_status load_weights_host(fnn_ctx *ctx, const fnn_weights *hw) {
  const int M = hw->n_members;
  if (M != ctx->cfg.n_members || !hw->W1 || !hw->b1 || !hw->W2 || !hw->b2 || !hw->W3 || !hw->b3 || !hw->w4 ||
      !hw->b4) {
    ctx->last_error = "weights: member count differs from the context or an array is NULL";
    return FNN_E_INVALID;
  }
  free_weights(ctx->w);
  DeviceWeights &w = ctx->w;
  const size_t n1 = (size_t)H1 * NAEV, n2 = (size_t)H2 * H1, n3 = (size_t)H3 * H2;
  std::vector<float> W1cat((size_t)NE * M * n1), W1Tcat((size_t)NE * M * n1), b1cat((size_t)NE * M * H1);
  for (int e = 0; e < NE; e++)
    for (int m = 0; m < M; m++) {
      const float *src = hw->W1 + ((size_t)m * NE + e) * n1;
      for (int n = 0; n < H1; n++) {
        memcpy(&W1cat[((size_t)e * M * H1 + (size_t)m * H1 + n) * NAEV], src + (size_t)n * NAEV, NAEV * sizeof(float));
        for (int k = 0; k < NAEV; k++)
          W1Tcat[((size_t)e * NAEV + k) * M * H1 + (size_t)m * H1 + n] = src[(size_t)n * NAEV + k];
        b1cat[(size_t)e * M * H1 + (size_t)m * H1 + n] = hw->b1[((size_t)m * NE + e) * H1 + n];
      }
    }
  std::vector<float> W2(hw->W2, hw->W2 + (size_t)M * NE * n2), W2T((size_t)M * NE * n2);
  std::vector<float> W3(hw->W3, hw->W3 + (size_t)M * NE * n3), W3T((size_t)M * NE * n3);
  for (size_t me = 0; me < (size_t)M * NE; me++) {
    for (int n = 0; n < H2; n++)
      for (int k = 0; k < H1; k++) W2T[me * n2 + (size_t)k * H2 + n] = W2[me * n2 + (size_t)n * H1 + k];
    for (int n = 0; n < H3; n++)
      for (int k = 0; k < H2; k++) W3T[me * n3 + (size_t)k * H3 + n] = W3[me * n3 + (size_t)n * H2 + k];
  }
  std::vector<float> b2(hw->b2, hw->b2 + (size_t)M * NE * H2), b3(hw->b3, hw->b3 + (size_t)M * NE * H3);
  std::vector<float> w4(hw->w4, hw->w4 + (size_t)M * NE * H3), b4(hw->b4, hw->b4 + (size_t)M * NE);
  fnn_status st;
  if ((st = upload(ctx, &w.W1cat, W1cat)) || (st = upload(ctx, &w.W1Tcat, W1Tcat)) || (st = upload(ctx, &w.b1cat, b1cat)) ||
      (st = upload(ctx, &w.W2, W2)) || (st = upload(ctx, &w.W2T, W2T)) || (st = upload(ctx, &w.b2, b2)) ||
      (st = upload(ctx, &w.W3, W3)) || (st = upload(ctx, &w.W3T, W3T)) || (st = upload(ctx, &w.b3, b3)) ||
      (st = upload(ctx, &w.w4, w4)) || (st = upload(ctx, &w.b4, b4)))
    return st;
  w.M = M;
  if ((st = upload_tc_weights(ctx, M, W1cat.data(), W1Tcat.data(), W2.data(), W2T.data(), W3.data(), W3T.data())))
    return st;
  ctx->has_weights = true;
  return FNN_OK;
}

extern "C" fnn_status fnn_load_weights(fnn_ctx *ctx, const char *path, const fnn_weights *host) {
  if (!ctx || (!path) == (!host)) return FNN_E_INVALID;
  ctx->gen++;
  if (host) return load_weights_host(ctx, host);
  FILE *f = fopen(path, "rb");
  if (!f) {
    ctx->last_error = std::string("cannot open ") + path;
    return FNN_E_INVALID;
  }
  char magic[4];
  int32_t version = 0, M = 0;
  bool ok = fread(magic, 1, 4, f) == 4 && memcmp(magic, "FNNW", 4) == 0 && fread(&version, 4, 1, f) == 1 &&
            version == 1 && fread(&M, 4, 1, f) == 1 && M >= 1 && M <= MAXM;
  std::vector<float> arr[8];
  const size_t sizes[8] = {(size_t)M * NE * H1 * NAEV, (size_t)M * NE * H1, (size_t)M * NE * H2 * H1, (size_t)M * NE * H2,
                           (size_t)M * NE * H3 * H2, (size_t)M * NE * H3, (size_t)M * NE * H3, (size_t)M * NE};
  for (int a = 0; ok && a < 8; a++) {
    arr[a].resize(sizes[a]);
    ok = fread(arr[a].data(), sizeof(float), sizes[a], f) == sizes[a];
  }
  fclose(f);
  if (!ok) {
    ctx->last_error = std::string("malformed weight file ") + path;
    return FNN_E_INVALID;
  }
  fnn_weights hw{M, arr[0].data(), arr[1].data(), arr[2].data(), arr[3].data(),
                 arr[4].data(), arr[5].data(), arr[6].data(), arr[7].data()};
  return load_weights_host(ctx, &hw);
}

extern "C" fnn_status fnn_aev(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, float *aev, void *stream) {
  if (!ctx || !sys || !nl || !aev) return FNN_E_INVALID;
  if ((uintptr_t)aev & 15) {
    ctx->last_error = "aev must be 16-byte aligned";
    return FNN_E_INVALID;
  }
  if (!nl->built || nl->n_atoms != sys->n_atoms || nl->n_mol != sys->n_mol) {
    ctx->last_error = "neighbour list was not built for this system";
    return FNN_E_STATE;
  }
  return launch_aev_forward(ctx, sys, nl, aev, nullptr, (cudaStream_t)stream);
}

extern "C" fnn_status fnn_aev_jvp(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *V, float *T,
                                  void *stream) {
  if (!ctx || !sys || !nl || !V || !T) return FNN_E_INVALID;
  if (!nl->built || nl->n_atoms != sys->n_atoms || nl->n_mol != sys->n_mol) {
    ctx->last_error = "neighbour list was not built for this system";
    return FNN_E_STATE;
  }
  return launch_aev_tangent(ctx, sys, nl, V, T, nullptr, (cudaStream_t)stream);
}

extern "C" fnn_status fnn_energy_forces(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, fnn_precision prec,
                                        double *E, float *F, double *virial, void *stream) {
  if (!ctx || !sys || !nl || !E || !F) return FNN_E_INVALID;
  if (!ctx->has_weights) {
    ctx->last_error = "no weights loaded";
    return FNN_E_STATE;
  }
  if (!nl->built || nl->n_atoms != sys->n_atoms || nl->n_mol != sys->n_mol) {
    ctx->last_error = "neighbour list was not built for this system";
    return FNN_E_STATE;
  }
  if (prec != FNN_FP32 && prec != FNN_BF16 && prec != FNN_FP8 && prec != FNN_FP32X3 && prec != FNN_BF16_FUSED)
    return FNN_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  fnn_status st;
  if ((st = ensure_workspace(ctx, nl->pad_cap))) return st;
  // small systems in the FP32 forms: one launch of thread-block clusters spread over the SMs (FP32 FFMA
  // networks, exact FP32 products, so also for the FP32X3 form) instead of a pipeline of single-SM
  // tensor-core tiles
  if ((prec == FNN_FP32 || prec == FNN_FP32X3) && sys->n_atoms > 0 && sys->n_atoms <= SMALL_BUILD_ATOMS &&
      (long long)sys->n_atoms * ctx->cfg.n_members <= SMALL_EVAL_ROWS)
    return launch_small_eval(ctx, sys, nl, E, F, virial, s);
  if (prec == FNN_FP32) {
    if ((st = launch_aev_forward(ctx, sys, nl, ctx->ws.aev, nl->inv, s))) return st;
    if ((st = mlp_fp32_forward_backward(ctx, nl, s))) return st;
    if ((st = energy_reduce(ctx, sys, nl, E, s))) return st;
  } else if ((st = tc_energy(ctx, sys, nl, prec, E, s))) {
    return st;
  }
  FNN_CUDA_TRY(ctx, cudaMemsetAsync(F, 0, (size_t)sys->n_atoms * 3 * sizeof(float), s));
  if (virial) FNN_CUDA_TRY(ctx, cudaMemsetAsync(virial, 0, (size_t)sys->n_mol * 9 * sizeof(double), s));
  return launch_aev_adjoint(ctx, sys, nl, ctx->ws.gaev, nl->inv, F, virial, s);
}

extern "C" fnn_status fnn_calibrate_fp8(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, void *stream) {
  if (!ctx || !sys || !nl) return FNN_E_INVALID;
  if (!ctx->has_weights) {
    ctx->last_error = "no weights loaded";
    return FNN_E_STATE;
  }
  if (!nl->built || nl->n_atoms != sys->n_atoms || nl->n_mol != sys->n_mol) {
    ctx->last_error = "neighbour list was not built for this system";
    return FNN_E_STATE;
  }
  return fp8_calibrate(ctx, sys, nl, (cudaStream_t)stream);
}

__global__ void k_pack_pos(int n, const float *p3, float4 *p4) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p4[i] = make_float4(p3[3 * i], p3[3 * i + 1], p3[3 * i + 2], 0.f);
}

extern "C" fnn_status fnn_energy_forces_host(fnn_ctx *ctx, int32_t N, int32_t NM, const int32_t *mol_offsets,
                                             const int32_t *Z, const float *pos, const float *cell, const uint8_t *pbc,
                                             fnn_precision prec, double *E, float *F, double *virial, void *stream) {
  if (!ctx || N < 0 || NM < 1 || !mol_offsets || (N > 0 && (!Z || !pos)) || !E || !F || (pbc && !cell))
    return FNN_E_INVALID;
  auto &h = ctx->host;
  if (!stream && !h.own) FNN_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&h.own, cudaStreamNonBlocking));
  if (!stream) stream = h.own;   // synchronous either way; a stream of its own can be captured
  cudaStream_t s = (cudaStream_t)stream;
  fnn_status st;
  if (N > h.n_atoms || NM > h.n_mol) {
    if (h.graph) {   // bound to the buffers about to be replaced
      fnn_graph_destroy(h.graph);
      h.graph = nullptr;
      h.gkey = h.last_key = -1;
    }
    int32_t na = N > h.n_atoms ? N : h.n_atoms, nm = NM > h.n_mol ? NM : h.n_mol;
    if ((st = dalloc(ctx, &h.Z, na)) || (st = dalloc(ctx, &h.pos, (size_t)na * 4)) ||
        (st = dalloc(ctx, &h.pos3, (size_t)na * 3)) || (st = dalloc(ctx, &h.F, (size_t)na * 3)) ||
        (st = dalloc(ctx, &h.mol_offsets, (size_t)nm + 1)) || (st = dalloc(ctx, &h.cell, (size_t)nm * 9)) ||
        (st = dalloc(ctx, &h.pbc, nm)) || (st = dalloc(ctx, &h.E, nm)) || (st = dalloc(ctx, &h.virial, (size_t)nm * 9)))
      return st;
    h.n_atoms = na;
    h.n_mol = nm;
  }
  if (!h.nl && (st = fnn_nlist_create(ctx, &h.nl, 0))) return st;
  if (!h.status) FNN_CUDA_TRY(ctx, cudaMallocHost(&h.status, sizeof(DevStatus)));
  if (h.graph && h.ggen != ctx->gen) {   // a buffer the recorded step references was reallocated since
    fnn_graph_destroy(h.graph);
    h.graph = nullptr;
    h.gkey = -1;
  }
  FNN_CUDA_TRY(ctx, cudaMemcpyAsync(h.mol_offsets, mol_offsets, ((size_t)NM + 1) * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
  if (N > 0) {
    FNN_CUDA_TRY(ctx, cudaMemcpyAsync(h.Z, Z, (size_t)N * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    FNN_CUDA_TRY(ctx, cudaMemcpyAsync(h.pos3, pos, (size_t)N * 3 * sizeof(float), cudaMemcpyHostToDevice, s));
    int nb = (N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024;
    FNN_KERNEL(ctx, "pack_pos", s);
    k_pack_pos<<<nb, 256, 0, s>>>(N, h.pos3, (float4 *)h.pos);
  }
  if (pbc) {
    FNN_CUDA_TRY(ctx, cudaMemcpyAsync(h.cell, cell, (size_t)NM * 9 * sizeof(float), cudaMemcpyHostToDevice, s));
    FNN_CUDA_TRY(ctx, cudaMemcpyAsync(h.pbc, pbc, (size_t)NM, cudaMemcpyHostToDevice, s));
  }
  fnn_system sys{N, NM, h.mol_offsets, h.Z, h.pos, pbc ? h.cell : nullptr, pbc ? h.pbc : nullptr};
  // a call repeating the previous one's shape replays the device part as a CUDA graph (created on the
  // second such call, whose own evaluation is the graph's eager step)
  const long long key = ((((long long)N * 2 + (pbc != nullptr)) * 2 + (virial != nullptr)) * 8 + (long long)prec) *
                            (1LL << 20) + NM;
  bool done = false;
  if (h.graph && key == h.gkey) {
    if ((st = fnn_graph_launch(h.graph, stream))) return st;
    done = true;
  } else if (key == h.last_key && stream != nullptr) {
    if (h.graph) fnn_graph_destroy(h.graph);
    h.graph = nullptr;
    if (fnn_graph_create(ctx, &sys, h.nl, prec, h.E, h.F, virial ? h.virial : nullptr, 1, stream, &h.graph) ==
        FNN_OK) {
      h.gkey = key;
      h.ggen = ctx->gen;
      done = true;
    } else {
      h.graph = nullptr;
      h.gkey = -1;
    }
  }
  h.last_key = key;
  if (!done) {
    if ((st = fnn_build_neighbors(ctx, &sys, h.nl, stream))) return st;
    if ((st = fnn_energy_forces(ctx, &sys, h.nl, prec, h.E, h.F, virial ? h.virial : nullptr, stream))) return st;
  }
  FNN_CUDA_TRY(ctx, cudaMemcpyAsync(E, h.E, (size_t)NM * sizeof(double), cudaMemcpyDeviceToHost, s));
  FNN_CUDA_TRY(ctx, cudaMemcpyAsync(F, h.F, (size_t)N * 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (virial)
    FNN_CUDA_TRY(ctx, cudaMemcpyAsync(virial, h.virial, (size_t)NM * 9 * sizeof(double), cudaMemcpyDeviceToHost, s));
  // the device status read back and cleared in stream order: one wait for the whole call
  FNN_CUDA_TRY(ctx, cudaMemcpyAsync(h.status, ctx->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  FNN_CUDA_TRY(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), s));
  FNN_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  const int64_t info = h.status->info;
  st = (fnn_status)h.status->code;
  if (st == FNN_E_CAPACITY && info > 0) {
    // the list outgrew its capacity: grow it and evaluate again (once)
    if (h.graph) {
      fnn_graph_destroy(h.graph);
      h.graph = nullptr;
    }
    h.gkey = h.last_key = -1;
    if ((st = fnn_nlist_reserve(h.nl, N, NM, info + info / 4))) return st;
    return fnn_energy_forces_host(ctx, N, NM, mol_offsets, Z, pos, cell, pbc, prec, E, F, virial, stream);
  }
  return st;
}

extern "C" fnn_status fnn_profile_enable(fnn_ctx *ctx, int on) {
  if (!ctx) return FNN_E_INVALID;
  ctx->prof.on = on != 0;
  return FNN_OK;
}

extern "C" fnn_status fnn_profile_read(fnn_ctx *ctx, char *names, double *ms, int64_t *launches, int32_t cap,
                                       int32_t *count) {
  if (!ctx || !count) return FNN_E_INVALID;
  FNN_CUDA_TRY(ctx, cudaDeviceSynchronize());
  std::vector<std::string> keys;
  std::vector<double> tot;
  std::vector<int64_t> n;
  for (auto &r : ctx->prof.recs) {
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    size_t k = 0;
    while (k < keys.size() && keys[k] != r.name) k++;
    if (k == keys.size()) {
      keys.push_back(r.name);
      tot.push_back(0.0);
      n.push_back(0);
    }
    tot[k] += t;
    n[k] += 1;
    ctx->prof.pool.push_back(r.a);
    ctx->prof.pool.push_back(r.b);
  }
  ctx->prof.recs.clear();
  *count = (int32_t)keys.size();
  for (int32_t k = 0; k < *count && k < cap; k++) {
    if (names) {
      strncpy(names + 48 * k, keys[k].c_str(), 47);
      names[48 * k + 47] = 0;
    }
    if (ms) ms[k] = tot[k];
    if (launches) launches[k] = n[k];
  }
  return FNN_OK;
}

extern "C" fnn_status fnn_launch_count(const fnn_ctx *ctx, int64_t *n) {
  if (!ctx || !n) return FNN_E_INVALID;
  *n = ctx->prof.launches;
  return FNN_OK;
}

extern "C" fnn_status fnn_sync(fnn_ctx *ctx, void *stream, int64_t *info) {
  if (!ctx) return FNN_E_INVALID;
  FNN_CUDA_TRY(ctx, cudaStreamSynchronize((cudaStream_t)stream));
  DevStatus h{};
  FNN_CUDA_TRY(ctx, cudaMemcpy(&h, ctx->status, sizeof(DevStatus), cudaMemcpyDeviceToHost));
  FNN_CUDA_TRY(ctx, cudaMemset(ctx->status, 0, sizeof(DevStatus)));
  if (info) *info = h.info;
  return (fnn_status)h.code;
}

// ------------------------------------------------------------------------------------- CUDA graphs
struct fnn_graph {
  fnn_ctx *ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;   // kernel launches one replay performs
  long long gen = 0;       // ctx->gen at recording: its buffers are the ones the graph references
};

extern "C" fnn_status fnn_graph_create(fnn_ctx *ctx, const fnn_system *sys, fnn_nlist *nl, fnn_precision prec,
                                       double *E, float *F, double *virial, int32_t rebuild, void *stream,
                                       fnn_graph **out) {
  if (!ctx || !sys || !nl || !E || !F || !out) return FNN_E_INVALID;
  if (!stream) {
    ctx->last_error = "graph capture needs a stream other than the legacy default stream";
    return FNN_E_INVALID;
  }
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  fnn_status st;
  // one eager step first: every buffer, calibration and kernel attribute is in place before capture
  if (rebuild && (st = fnn_build_neighbors(ctx, sys, nl, stream))) return st;
  if (!rebuild && (!nl->built || nl->n_atoms != sys->n_atoms || nl->n_mol != sys->n_mol)) {
    ctx->last_error = "neighbour list was not built for this system";
    return FNN_E_STATE;
  }
  if ((st = fnn_energy_forces(ctx, sys, nl, prec, E, F, virial, stream))) return st;
  int64_t info = 0;
  if ((st = fnn_sync(ctx, stream, &info))) {
    ctx->last_error = "the eager step before capture posted a device status";
    return st;
  }
  const long long l0 = ctx->prof.launches;
  const bool prof = ctx->prof.on;
  ctx->prof.on = false;   // no per-kernel events inside the graph
  FNN_CUDA_TRY(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  st = FNN_OK;
  if (rebuild) st = fnn_build_neighbors(ctx, sys, nl, stream);
  if (!st) st = fnn_energy_forces(ctx, sys, nl, prec, E, F, virial, stream);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(s, &g);
  ctx->prof.on = prof;
  const long long kernels = ctx->prof.launches - l0;
  ctx->prof.launches = l0;   // capture launches nothing
  if (st || ec != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (!st) {
      ctx->last_error = std::string("stream capture failed: ") + cudaGetErrorString(ec);
      st = FNN_E_CUDA;
    }
    return st;
  }
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    ctx->last_error = "cudaGraphInstantiate failed";
    return FNN_E_CUDA;
  }
  fnn_graph *G = new fnn_graph();
  G->ctx = ctx;
  G->graph = g;
  G->exec = exec;
  G->kernels = kernels;
  G->gen = ctx->gen;
  *out = G;
  return FNN_OK;
}

extern "C" fnn_status fnn_graph_launch(fnn_graph *g, void *stream) {
  if (!g) return FNN_E_INVALID;
  if (g->gen != g->ctx->gen) {
    g->ctx->last_error = "the context reallocated buffers this graph references (weights reloaded or a larger "
                         "system evaluated): record the graph again";
    return FNN_E_STATE;
  }
  FNN_CUDA_TRY(g->ctx, cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  g->ctx->prof.launches += g->kernels;
  return FNN_OK;
}

extern "C" fnn_status fnn_graph_kernels(const fnn_graph *g, int64_t *kernels) {
  if (!g || !kernels) return FNN_E_INVALID;
  *kernels = g->kernels;
  return FNN_OK;
}

extern "C" fnn_status fnn_graph_destroy(fnn_graph *g) {
  if (!g) return FNN_E_INVALID;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return FNN_OK;
}
