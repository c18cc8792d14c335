// Parameter gradients of a training loss L(E, F) (section IV): energy term by backpropagation, force term
// by forward-mode tangents through the networks and a reverse pass over primal and tangent.
//
// With F = -dE/dx and v = dL/dF, the force term of the loss depends on the parameters only through
// G = dE/dAEV:  dL_F/dtheta = -d/dtheta <t, G(theta)>,  t = (dAEV/dx) v  (the AEV tangent, aev.cu).
// <t, G> is the directional derivative of the networks' output along t, so with z_l = W_l h_{l-1} + b_l,
// h_l = CELU(z_l), tangents zd_l = W_l hd_{l-1}, hd_l = CELU'(z_l) zd_l (hd_0 = t), and Phi = L_E - <t, G>:
//   output:  gb3 = dPhi/dhd_3 = -(1/M) w4,  g3 = dPhi/dh_3 = (1/M) dL/dE w4
//   each l:  gbz_l = CELU'(z_l) gb_l,  gz_l = CELU'(z_l) g_l + CELU''(z_l) zd_l gb_l
//            dW_l += gbz_l hd_{l-1}^T + gz_l h_{l-1}^T,  db_l += gz_l,
//            gb_{l-1} = W_l^T gbz_l,  g_{l-1} = W_l^T gz_l
//   dw4 += (1/M) dL/dE h_3 - (1/M) hd_3,  db4 += (1/M) dL/dE.
// CELU' and CELU''/CELU' come from h alone (h > 0: 1 and 0; else 1 + h/alpha and 1/alpha), so neither z nor
// zd is stored.  FP32 throughout (SIMT products of mlp_simt.cu plus the kernels below).
#include "fnn_internal.cuh"

namespace fnn {

struct TrainWs {
  size_t rows = 0;
  int M = 0;
  float *buf = nullptr;
  float *t, *h3, *hd1, *hd2, *hd3, *gb3, *gz3, *gb2, *gz2, *gb1, *gz1;
};

static fnn_status train_ws(fnn_ctx *ctx, TrainWs &T, size_t rows) {
  const int M = ctx->w.M;
  if (T.buf && rows <= T.rows && T.M == M) return FNN_OK;
  if (T.buf) cudaFree(T.buf);
  T.buf = nullptr;
  rows = rows + rows / 8;
  const size_t per = NAEV + (size_t)M * (H3 + H1 + H2 + H3 + 2 * H3 + 2 * H2 + 2 * H1);
  if (cudaMalloc(&T.buf, rows * per * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    ctx->last_error = "cudaMalloc failed for the training workspace";
    return FNN_E_OOM;
  }
  float *p = T.buf;
  T.t = p; p += rows * NAEV;
  T.h3 = p; p += rows * M * H3;
  T.hd1 = p; p += rows * M * H1;
  T.hd2 = p; p += rows * M * H2;
  T.hd3 = p; p += rows * M * H3;
  T.gb3 = p; p += rows * M * H3;
  T.gz3 = p; p += rows * M * H3;
  T.gb2 = p; p += rows * M * H2;
  T.gz2 = p; p += rows * M * H2;
  T.gb1 = p; p += rows * M * H1;
  T.gz1 = p;
  T.rows = rows;
  T.M = M;
  return FNN_OK;
}

__device__ __forceinline__ float dcelu_h(float h) { return h > 0.f ? 1.f : 1.f + h * CELU_INV_ALPHA; }
__device__ __forceinline__ float ddcelu_ratio(float h) { return h > 0.f ? 0.f : CELU_INV_ALPHA; }

// output layer: gb3, gz3 per (row, member, unit); dw4 and db4 summed per tile, one atomic per thread
__global__ void k_out_reverse(int M, const int32_t *tile_elem, const int32_t *inv, const int32_t *atom_mol,
                              const double *dLdE, const float *w4, const float *h3, const float *hd3, float *gb3,
                              float *gz3, float *dw4, float *db4) {
  const int tile = blockIdx.x, m = blockIdx.y, n = threadIdx.x;   // blockDim.x = H3
  const int e = tile_elem[tile];
  if (e < 0) return;
  const float w = w4[((size_t)m * NE + e) * H3 + n];
  const float c = 1.f / (float)M;
  float acc_w = 0.f, acc_b = 0.f;
  for (int rr = 0; rr < ROW_TILE; rr++) {
    const size_t r = (size_t)tile * ROW_TILE + rr;
    const int i = inv[r];
    const size_t o = r * (size_t)M * H3 + (size_t)m * H3 + n;
    const int mol = i < 0 ? -1 : atom_mol[i];   // -1: padding, or an atom outside every structure
    if (mol < 0) {
      gb3[o] = 0.f;
      gz3[o] = 0.f;
      continue;
    }
    const float cE = (float)dLdE[mol] * c;
    const float h = h3[o], hd = hd3[o];
    const float s1 = dcelu_h(h);
    const float gb = -c * w, g = cE * w;
    gb3[o] = s1 * gb;
    gz3[o] = s1 * g + ddcelu_ratio(h) * hd * gb;
    acc_w += cE * h - c * hd;
    acc_b += cE;
  }
  atomicAdd(&dw4[((size_t)m * NE + e) * H3 + n], acc_w);
  if (n == 0) atomicAdd(&db4[(size_t)m * NE + e], acc_b);
}

// hidden layer l: (gb, g) -> (gbz, gz) in place, from h_l and hd_l
__global__ void k_act_reverse(size_t count, size_t row_width, const int32_t *tile_elem, const float *h,
                              const float *hd, float *gb, float *g) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count; k += (size_t)gridDim.x * blockDim.x) {
    if (tile_elem[k / row_width / ROW_TILE] < 0) continue;   // rows past the last tile are never read
    const float hv = h[k], s1 = dcelu_h(hv), b = gb[k];
    gb[k] = s1 * b;
    g[k] = s1 * g[k] + ddcelu_ratio(hv) * hd[k] * b;
  }
}

// dW[m][e][o][i] += sum over the rows of element e of D1[r][o] X1[r][i] + D2[r][o] X2[r][i]; db[m][e][o] += sum D2
struct WgradP {
  const float *D1, *D2, *X1, *X2;
  long long ldd, d_mstride, ldx, x_mstride;
  float *dW, *db;
  int O, I;                 // output and input widths of the layer
  int n_tiles, tiles_per_block;
  const int32_t *tile_elem;
};

constexpr int WG_T = 64, WG_R = 32;

__global__ void __launch_bounds__(256) k_wgrad(WgradP p) {
  const int ot = blockIdx.x / ((p.I + WG_T - 1) / WG_T), it = blockIdx.x % ((p.I + WG_T - 1) / WG_T);
  const int m = blockIdx.z;
  const int o0 = ot * WG_T, i0 = it * WG_T;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  __shared__ float Ds[WG_R][WG_T + 1], Xs[WG_R][WG_T + 1];
  float acc[4][4] = {};
  float bacc[4] = {0, 0, 0, 0};
  int cur_e = -1;
  auto flush = [&]() {
    if (cur_e < 0) return;
    float *W = p.dW + ((size_t)m * NE + cur_e) * p.O * p.I;
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int b = 0; b < 4; b++) {
        const int o = o0 + ty * 4 + a, i = i0 + tx * 4 + b;
        if (o < p.O && i < p.I && acc[a][b] != 0.f) atomicAdd(&W[(size_t)o * p.I + i], acc[a][b]);
        acc[a][b] = 0.f;
      }
    if (p.db && it == 0 && tx == 0)
#pragma unroll
      for (int a = 0; a < 4; a++) {
        const int o = o0 + ty * 4 + a;
        if (o < p.O && bacc[a] != 0.f) atomicAdd(&p.db[((size_t)m * NE + cur_e) * p.O + o], bacc[a]);
        bacc[a] = 0.f;
      }
  };
  const int t_begin = blockIdx.y * p.tiles_per_block, t_end = min(p.n_tiles, t_begin + p.tiles_per_block);
  for (int t = t_begin; t < t_end; t++) {
    const int e = p.tile_elem[t];
    if (e < 0) continue;
    if (e != cur_e) {
      flush();
      cur_e = e;
    }
    for (int term = 0; term < 2; term++) {
      const float *D = term ? p.D2 : p.D1, *X = term ? p.X2 : p.X1;
      for (int r0 = 0; r0 < ROW_TILE; r0 += WG_R) {
        const size_t rbase = (size_t)t * ROW_TILE + r0;
        __syncthreads();
        for (int k = tid; k < WG_R * WG_T; k += 256) {
          const int rr = k / WG_T, cc = k % WG_T;
          const size_t r = rbase + rr;
          Ds[rr][cc] = (o0 + cc < p.O) ? D[r * p.ldd + m * p.d_mstride + o0 + cc] : 0.f;
          Xs[rr][cc] = (i0 + cc < p.I) ? X[r * p.ldx + m * p.x_mstride + i0 + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < WG_R; rr++) {
          float dv[4], xv[4];
#pragma unroll
          for (int a = 0; a < 4; a++) dv[a] = Ds[rr][ty * 4 + a];
#pragma unroll
          for (int b = 0; b < 4; b++) xv[b] = Xs[rr][tx * 4 + b];
#pragma unroll
          for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) acc[a][b] = fmaf(dv[a], xv[b], acc[a][b]);
          if (term == 1 && tx == 0)
#pragma unroll
            for (int a = 0; a < 4; a++) bacc[a] += dv[a];
        }
      }
    }
  }
  flush();
}

static fnn_status wgrad(fnn_ctx *ctx, const char *name, const WgradP &p0, int M, cudaStream_t s) {
  WgradP p = p0;
  const int n_o = (p.O + WG_T - 1) / WG_T, n_i = (p.I + WG_T - 1) / WG_T;
  // enough row groups to cover the GPU about twice, at least 4 tiles each
  int groups = (2 * ctx->num_sms + n_o * n_i * M - 1) / (n_o * n_i * M);
  if (groups < 1) groups = 1;
  p.tiles_per_block = (p.n_tiles + groups - 1) / groups;
  if (p.tiles_per_block < 4) p.tiles_per_block = 4;
  groups = (p.n_tiles + p.tiles_per_block - 1) / p.tiles_per_block;
  dim3 grid(n_o * n_i, groups, M);
  FNN_KERNEL(ctx, name, s);
  k_wgrad<<<grid, 256, 0, s>>>(p);
  return check_launch(ctx, name);
}

void free_train(fnn_ctx *ctx) {
  if (!ctx->train) return;
  TrainWs *T = reinterpret_cast<TrainWs *>(ctx->train);
  if (T->buf) cudaFree(T->buf);
  delete T;
  ctx->train = nullptr;
}

}  // namespace fnn

using namespace fnn;

extern "C" fnn_status fnn_param_grads(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, fnn_precision prec,
                                      const double *dLdE, const float *dLdF, const fnn_grads *g, void *stream) {
  if (!ctx || !sys || !nl || !dLdE || !dLdF || !g || !g->W1 || !g->b1 || !g->W2 || !g->b2 || !g->W3 || !g->b3 ||
      !g->w4 || !g->b4)
    return FNN_E_INVALID;
  if (!ctx->has_weights) {
    ctx->last_error = "no weights loaded";
    return FNN_E_STATE;
  }
  if (!nl->built || nl->n_atoms != sys->n_atoms || nl->n_mol != sys->n_mol) {
    ctx->last_error = "neighbour list was not built for this system";
    return FNN_E_STATE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == FNN_BF16) return tc_param_grads(ctx, sys, nl, dLdE, dLdF, g, s);
  if (prec != FNN_FP32) {
    ctx->last_error = "parameter gradients are built for the FP32 and BF16 forms";
    return FNN_E_INVALID;
  }
  if (!ctx->train) ctx->train = new TrainWs();
  TrainWs &T = *reinterpret_cast<TrainWs *>(ctx->train);
  fnn_status st;
  if ((st = ensure_workspace(ctx, nl->pad_cap)) || (st = train_ws(ctx, T, nl->pad_cap))) return st;
  const DeviceWeights &w = ctx->w;
  Workspace &ws = ctx->ws;
  const int M = w.M;
  const int tiles = nl->pad_cap / ROW_TILE;
  // primal AEV and its tangent along dL/dF
  if ((st = launch_aev_forward(ctx, sys, nl, ws.aev, nl->inv, s))) return st;
  if ((st = launch_aev_tangent(ctx, sys, nl, dLdF, T.t, nl->inv, s))) return st;
  GemmP p{};
  p.tile_elem = nl->tile_elem;
  p.M = M;
  // ---- forward, keeping h1, h2, h3
  p.A = ws.aev; p.lda = NAEV; p.a_mstride = 0;
  p.B = w.W1cat; p.ldb = NAEV; p.b_estride = (long long)M * H1 * NAEV; p.b_mstride = 0;
  p.C = ws.h1; p.ldc = (long long)M * H1; p.c_mstride = 0;
  p.N = M * H1; p.K = NAEV;
  p.bias = w.b1cat; p.bias_estride = (long long)M * H1; p.bias_mstride = 0;
  if ((st = launch_gemm_f32(ctx, "tr_l1_fwd", EPI_BIAS_CELU, p, tiles, 1, s))) return st;
  p.A = ws.h1; p.lda = (long long)M * H1; p.a_mstride = H1;
  p.B = w.W2; p.ldb = H1; p.b_estride = (long long)H2 * H1; p.b_mstride = (long long)NE * H2 * H1;
  p.C = ws.h2; p.ldc = (long long)M * H2; p.c_mstride = H2;
  p.N = H2; p.K = H1;
  p.bias = w.b2; p.bias_estride = H2; p.bias_mstride = (long long)NE * H2;
  if ((st = launch_gemm_f32(ctx, "tr_l2_fwd", EPI_BIAS_CELU, p, tiles, M, s))) return st;
  p.A = ws.h2; p.lda = (long long)M * H2; p.a_mstride = H2;
  p.B = w.W3; p.ldb = H2; p.b_estride = (long long)H3 * H2; p.b_mstride = (long long)NE * H3 * H2;
  p.C = T.h3; p.ldc = (long long)M * H3; p.c_mstride = H3;
  p.N = H3; p.K = H2;
  p.bias = w.b3; p.bias_estride = H3; p.bias_mstride = (long long)NE * H3;
  p.w4 = w.w4; p.w4_estride = H3; p.w4_mstride = (long long)NE * H3;
  p.ypart = ws.ypart;
  if ((st = launch_gemm_f32(ctx, "tr_l3_fwd", EPI_L3_H, p, tiles, M, s))) return st;
  // ---- tangents hd_l = CELU'(z_l) (W_l hd_{l-1}), hd_0 = t
  p.A = T.t; p.lda = NAEV; p.a_mstride = 0;
  p.B = w.W1cat; p.ldb = NAEV; p.b_estride = (long long)M * H1 * NAEV; p.b_mstride = 0;
  p.C = T.hd1; p.ldc = (long long)M * H1; p.c_mstride = 0;
  p.N = M * H1; p.K = NAEV;
  p.aux = ws.h1; p.ldaux = (long long)M * H1; p.aux_mstride = 0;
  if ((st = launch_gemm_f32(ctx, "tr_l1_tan", EPI_DCELU, p, tiles, 1, s))) return st;
  p.A = T.hd1; p.lda = (long long)M * H1; p.a_mstride = H1;
  p.B = w.W2; p.ldb = H1; p.b_estride = (long long)H2 * H1; p.b_mstride = (long long)NE * H2 * H1;
  p.C = T.hd2; p.ldc = (long long)M * H2; p.c_mstride = H2;
  p.N = H2; p.K = H1;
  p.aux = ws.h2; p.ldaux = (long long)M * H2; p.aux_mstride = H2;
  if ((st = launch_gemm_f32(ctx, "tr_l2_tan", EPI_DCELU, p, tiles, M, s))) return st;
  p.A = T.hd2; p.lda = (long long)M * H2; p.a_mstride = H2;
  p.B = w.W3; p.ldb = H2; p.b_estride = (long long)H3 * H2; p.b_mstride = (long long)NE * H3 * H2;
  p.C = T.hd3; p.ldc = (long long)M * H3; p.c_mstride = H3;
  p.N = H3; p.K = H2;
  p.aux = T.h3; p.ldaux = (long long)M * H3; p.aux_mstride = H3;
  if ((st = launch_gemm_f32(ctx, "tr_l3_tan", EPI_DCELU, p, tiles, M, s))) return st;
  // ---- output layer reverse (+ dw4, db4)
  {
    FNN_KERNEL(ctx, "tr_out_rev", s);
    k_out_reverse<<<dim3(tiles, M), H3, 0, s>>>(M, nl->tile_elem, nl->inv, nl->atom_mol, dLdE, w.w4, T.h3, T.hd3,
                                                T.gb3, T.gz3, g->w4, g->b4);
  }
  WgradP q{};
  q.n_tiles = tiles;
  q.tile_elem = nl->tile_elem;
  // ---- layer 3: dW3, then (gb2, g2) = W3^T (gb3, gz3), then CELU' at layer 2
  q.D1 = T.gb3; q.D2 = T.gz3; q.ldd = (long long)M * H3; q.d_mstride = H3;
  q.X1 = T.hd2; q.X2 = ws.h2; q.ldx = (long long)M * H2; q.x_mstride = H2;
  q.dW = g->W3; q.db = g->b3; q.O = H3; q.I = H2;
  if ((st = wgrad(ctx, "tr_l3_wgrad", q, M, s))) return st;
  p.aux = nullptr;
  p.B = w.W3T; p.ldb = H3; p.b_estride = (long long)H2 * H3; p.b_mstride = (long long)NE * H2 * H3;
  p.lda = (long long)M * H3; p.a_mstride = H3; p.ldc = (long long)M * H2; p.c_mstride = H2;
  p.N = H2; p.K = H3; p.scale = 1.f;
  p.A = T.gb3; p.C = T.gb2;
  if ((st = launch_gemm_f32(ctx, "tr_l3_rev", EPI_SCALE, p, tiles, M, s))) return st;
  p.A = T.gz3; p.C = T.gz2;
  if ((st = launch_gemm_f32(ctx, "tr_l3_rev", EPI_SCALE, p, tiles, M, s))) return st;
  {
    const size_t count = (size_t)nl->pad_cap * M * H2;
    FNN_KERNEL(ctx, "tr_act_rev", s);
    k_act_reverse<<<(unsigned)((count + 255) / 256 < 65535 ? (count + 255) / 256 : 65535), 256, 0, s>>>(
        count, (size_t)M * H2, nl->tile_elem, ws.h2, T.hd2, T.gb2, T.gz2);
  }
  // ---- layer 2
  q.D1 = T.gb2; q.D2 = T.gz2; q.ldd = (long long)M * H2; q.d_mstride = H2;
  q.X1 = T.hd1; q.X2 = ws.h1; q.ldx = (long long)M * H1; q.x_mstride = H1;
  q.dW = g->W2; q.db = g->b2; q.O = H2; q.I = H1;
  if ((st = wgrad(ctx, "tr_l2_wgrad", q, M, s))) return st;
  p.B = w.W2T; p.ldb = H2; p.b_estride = (long long)H1 * H2; p.b_mstride = (long long)NE * H1 * H2;
  p.lda = (long long)M * H2; p.a_mstride = H2; p.ldc = (long long)M * H1; p.c_mstride = H1;
  p.N = H1; p.K = H2;
  p.A = T.gb2; p.C = T.gb1;
  if ((st = launch_gemm_f32(ctx, "tr_l2_rev", EPI_SCALE, p, tiles, M, s))) return st;
  p.A = T.gz2; p.C = T.gz1;
  if ((st = launch_gemm_f32(ctx, "tr_l2_rev", EPI_SCALE, p, tiles, M, s))) return st;
  {
    const size_t count = (size_t)nl->pad_cap * M * H1;
    FNN_KERNEL(ctx, "tr_act_rev", s);
    k_act_reverse<<<(unsigned)((count + 255) / 256 < 65535 ? (count + 255) / 256 : 65535), 256, 0, s>>>(
        count, (size_t)M * H1, nl->tile_elem, ws.h1, T.hd1, T.gb1, T.gz1);
  }
  // ---- layer 1: dW1[m][e] from the member's 256 columns against the AEV and its tangent
  q.D1 = T.gb1; q.D2 = T.gz1; q.ldd = (long long)M * H1; q.d_mstride = H1;
  q.X1 = T.t; q.X2 = ws.aev; q.ldx = NAEV; q.x_mstride = 0;
  q.dW = g->W1; q.db = g->b1; q.O = H1; q.I = NAEV;
  return wgrad(ctx, "tr_l1_wgrad", q, M, s);
}
