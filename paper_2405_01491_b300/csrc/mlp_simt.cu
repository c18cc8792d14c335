// Per-element networks 1008-256-192-160-1 with CELU (section II.B, ChemicalNet) and their
// input gradient, FP32 form: SIMT FFMA GEMMs over species-sorted, 128-row padded segments.
//
// Every product is C[r, n] = sum_k A[r, k] B[n, k] with both operands K-contiguous ("TN"):
// forward weights are W[out][in], backward weights are stored transposed.  A 128-row tile
// belongs to one element (tile_elem), blockIdx.z selects the ensemble member.
//   L1   h1 = CELU(aev W1^T + b1)           all members at once: N = M*256
//   L2   h2 = CELU(h1_m W2^T + b2)          per member
//   L3   h3 = CELU(h2_m W3^T + b3); y_m partial = h3 . w4 (per 64-column tile);
//        g3 = (1/M) w4 * CELU'(z3)          fused epilogue
//   L3'  g2 = (g3_m W3) * CELU'(z2)         CELU' recovered from h: 1 if h > 0 else 1 + h/alpha
//   L2'  g1 = (g2_m W2) * CELU'(z1)
//   L1'  dE/dAEV = g1 W1cat                 K = M*256 sums the members
#include "fnn_internal.cuh"

namespace fnn {

constexpr int BM = 128, BN = 64, BK = 16, GNT = 256;

__device__ __forceinline__ float celu(float z) { return z > 0.f ? z : CELU_ALPHA * expm1f(z * CELU_INV_ALPHA); }
__device__ __forceinline__ float dcelu_from_h(float h) { return h > 0.f ? 1.f : 1.f + h * CELU_INV_ALPHA; }

// (three blocks per SM: 80 registers, a few bytes of epilogue spills; 6.72 -> 6.22 ms for the FP32 step)
template <int EPI>
__global__ void __launch_bounds__(GNT, 3) k_gemm_f32(GemmP p) {
  int e = p.tile_elem[blockIdx.y];
  if (e < 0) return;
  const int m = blockIdx.z;
  const long long row0 = (long long)blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  const float *A = p.A + row0 * p.lda + m * p.a_mstride;
  const float *B = p.B + e * p.b_estride + m * p.b_mstride;

  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;

  // global -> register prefetch
  const int ar = tid >> 2, akc = (tid & 3) * 4;   // A rows ar, ar + 64
  const int bn = tid >> 2, bkc = (tid & 3) * 4;   // B row n0 + bn
  float4 ra[2], rb;
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 2; q++) ra[q] = *reinterpret_cast<const float4 *>(A + (long long)(ar + 64 * q) * p.lda + k0 + akc);
    if (n0 + bn < p.N)
      rb = *reinterpret_cast<const float4 *>(B + (long long)(n0 + bn) * p.ldb + k0 + bkc);
    else
      rb = make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 2; q++) {
      As[buf][akc + 0][ar + 64 * q] = ra[q].x;
      As[buf][akc + 1][ar + 64 * q] = ra[q].y;
      As[buf][akc + 2][ar + 64 * q] = ra[q].z;
      As[buf][akc + 3][ar + 64 * q] = ra[q].w;
    }
    Bs[buf][bkc + 0][bn] = rb.x;
    Bs[buf][bkc + 1][bn] = rb.y;
    Bs[buf][bkc + 2][bn] = rb.z;
    Bs[buf][bkc + 3][bn] = rb.w;
  };

  // acc2[i][j] = (C[2i][j], C[2i + 1][j]): rows in pairs, each pair one packed FP32 fma per k (the same
  // fma per element as a scalar loop, half the instructions)
  float2 acc2[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc2[i][j] = make_float2(0.f, 0.f);

  const int nk = p.K / BK;
  load(0);
  store(0);
  __syncthreads();
  for (int kt = 0; kt < nk; kt++) {
    int buf = kt & 1;
    if (kt + 1 < nk) load((kt + 1) * BK);
#pragma unroll
    for (int k = 0; k < BK; k++) {
      float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 8]);
      float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 8 + 4]);
      float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
      const float2 av[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                            make_float2(a1.z, a1.w)};
      const float bv[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const float2 bj = make_float2(bv[j], bv[j]);
#pragma unroll
        for (int i = 0; i < 4; i++) acc2[i][j] = __ffma2_rn(av[i], bj, acc2[i][j]);
      }
    }
    if (kt + 1 < nk) store(buf ^ 1);
    __syncthreads();
  }

  // epilogue
  float *C = p.C + row0 * p.ldc + m * p.c_mstride;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    int r = ty * 8 + i;
    float ysum = 0.f;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      int n = n0 + tx * 4 + j;
      if (n >= p.N) continue;
      float v = (i & 1) ? acc2[i >> 1][j].y : acc2[i >> 1][j].x;
      float o;
      if (EPI == EPI_BIAS_CELU) {
        o = celu(v + p.bias[e * p.bias_estride + m * p.bias_mstride + n]);
      } else if (EPI == EPI_L3) {
        float z = v + p.bias[e * p.bias_estride + m * p.bias_mstride + n];
        float w = p.w4[e * p.w4_estride + m * p.w4_mstride + n];
        ysum += celu(z) * w;
        o = p.scale * w * (z > 0.f ? 1.f : expf(z * CELU_INV_ALPHA));
      } else if (EPI == EPI_L3_H) {   // keep h3 itself (training) and the output-layer partials
        float z = v + p.bias[e * p.bias_estride + m * p.bias_mstride + n];
        float h = celu(z);
        ysum += h * p.w4[e * p.w4_estride + m * p.w4_mstride + n];
        o = h;
      } else if (EPI == EPI_DCELU) {
        float h = p.aux[(row0 + r) * p.ldaux + m * p.aux_mstride + n];
        o = v * dcelu_from_h(h);
      } else {
        o = v * p.scale;
      }
      C[(long long)r * p.ldc + n] = o;
    }
    if (EPI == EPI_L3 || EPI == EPI_L3_H) {
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) ysum += __shfl_xor_sync(0xffffffffu, ysum, o);
      if (tx == 0) p.ypart[((row0 + r) * p.M + m) * 4 + blockIdx.x] = ysum;
    }
  }
}

template <int EPI>
static void launch(fnn_ctx *ctx, const char *name, const GemmP &p, int row_tiles, int members, cudaStream_t s) {
  dim3 grid((p.N + BN - 1) / BN, row_tiles, members);
  FNN_KERNEL(ctx, name, s);
  k_gemm_f32<EPI><<<grid, GNT, 0, s>>>(p);
}

fnn_status launch_gemm_f32(fnn_ctx *ctx, const char *name, int epi, const GemmP &p, int row_tiles, int members,
                           cudaStream_t s) {
  switch (epi) {
    case EPI_BIAS_CELU: launch<EPI_BIAS_CELU>(ctx, name, p, row_tiles, members, s); break;
    case EPI_L3: launch<EPI_L3>(ctx, name, p, row_tiles, members, s); break;
    case EPI_DCELU: launch<EPI_DCELU>(ctx, name, p, row_tiles, members, s); break;
    case EPI_SCALE: launch<EPI_SCALE>(ctx, name, p, row_tiles, members, s); break;
    case EPI_L3_H: launch<EPI_L3_H>(ctx, name, p, row_tiles, members, s); break;
    default: ctx->last_error = "unknown epilogue"; return FNN_E_INVALID;
  }
  return check_launch(ctx, name);
}

fnn_status mlp_fp32_forward_backward(fnn_ctx *ctx, const fnn_nlist *nl, cudaStream_t s) {
  const DeviceWeights &w = ctx->w;
  Workspace &ws = ctx->ws;
  const int M = w.M;
  const int tiles = nl->pad_cap / ROW_TILE;
  GemmP p{};
  p.tile_elem = nl->tile_elem;
  p.M = M;
  // L1
  p.A = ws.aev; p.lda = NAEV; p.a_mstride = 0;
  p.B = w.W1cat; p.ldb = NAEV; p.b_estride = (long long)M * H1 * NAEV; p.b_mstride = 0;
  p.C = ws.h1; p.ldc = (long long)M * H1; p.c_mstride = 0;
  p.N = M * H1; p.K = NAEV;
  p.bias = w.b1cat; p.bias_estride = (long long)M * H1; p.bias_mstride = 0;
  launch<EPI_BIAS_CELU>(ctx, "f32_l1_fwd", p, tiles, 1, s);
  // L2
  p.A = ws.h1; p.lda = (long long)M * H1; p.a_mstride = H1;
  p.B = w.W2; p.ldb = H1; p.b_estride = (long long)H2 * H1; p.b_mstride = (long long)NE * H2 * H1;
  p.C = ws.h2; p.ldc = (long long)M * H2; p.c_mstride = H2;
  p.N = H2; p.K = H1;
  p.bias = w.b2; p.bias_estride = H2; p.bias_mstride = (long long)NE * H2;
  launch<EPI_BIAS_CELU>(ctx, "f32_l2_fwd", p, tiles, M, s);
  // L3 + output layer + g3
  p.A = ws.h2; p.lda = (long long)M * H2; p.a_mstride = H2;
  p.B = w.W3; p.ldb = H2; p.b_estride = (long long)H3 * H2; p.b_mstride = (long long)NE * H3 * H2;
  p.C = ws.g3; p.ldc = (long long)M * H3; p.c_mstride = H3;
  p.N = H3; p.K = H2;
  p.bias = w.b3; p.bias_estride = H3; p.bias_mstride = (long long)NE * H3;
  p.w4 = w.w4; p.w4_estride = H3; p.w4_mstride = (long long)NE * H3;
  p.ypart = ws.ypart;
  p.scale = 1.f / (float)M;
  launch<EPI_L3>(ctx, "f32_l3_fwd", p, tiles, M, s);
  // L3 backward
  p.A = ws.g3; p.lda = (long long)M * H3; p.a_mstride = H3;
  p.B = w.W3T; p.ldb = H3; p.b_estride = (long long)H2 * H3; p.b_mstride = (long long)NE * H2 * H3;
  p.C = ws.g2; p.ldc = (long long)M * H2; p.c_mstride = H2;
  p.N = H2; p.K = H3;
  p.aux = ws.h2; p.ldaux = (long long)M * H2; p.aux_mstride = H2;
  launch<EPI_DCELU>(ctx, "f32_l3_bwd", p, tiles, M, s);
  // L2 backward
  p.A = ws.g2; p.lda = (long long)M * H2; p.a_mstride = H2;
  p.B = w.W2T; p.ldb = H2; p.b_estride = (long long)H1 * H2; p.b_mstride = (long long)NE * H1 * H2;
  p.C = ws.g1; p.ldc = (long long)M * H1; p.c_mstride = H1;
  p.N = H1; p.K = H2;
  p.aux = ws.h1; p.ldaux = (long long)M * H1; p.aux_mstride = H1;
  launch<EPI_DCELU>(ctx, "f32_l2_bwd", p, tiles, M, s);
  // L1 backward: dE/dAEV, K = M*256 sums the members
  p.A = ws.g1; p.lda = (long long)M * H1; p.a_mstride = 0;
  p.B = w.W1Tcat; p.ldb = (long long)M * H1; p.b_estride = (long long)NAEV * M * H1; p.b_mstride = 0;
  p.C = ws.gaev; p.ldc = NAEV; p.c_mstride = 0;
  p.N = NAEV; p.K = M * H1;
  p.scale = 1.f;
  launch<EPI_SCALE>(ctx, "f32_l1_bwd", p, tiles, 1, s);
  return check_launch(ctx, "mlp_fp32");
}

// ---------------------------------------------------------------------------- energy reduction
// e_i = (1/M) sum_m (b4 + y partials of atom i's row), then E_mol = sum of e_i over the structure's
// contiguous atoms in float64 (section II.E) in a fixed order: slice y of gridDim.y sums its atoms in
// a fixed tree; with more than one slice the last slice block of a structure to finish adds the slice
// sums (lane-strided, then a fixed shuffle tree) and rearms the structure's ticket for the next launch.
__device__ __forceinline__ double atom_energy(int i, const int32_t *perm, const uint8_t *elem, const float *ypart,
                                              const float *b4, int M, int ntile) {
  const int row = perm[i], e = elem[i];
  const float4 *yp = reinterpret_cast<const float4 *>(ypart) + (size_t)row * M;
  float v = 0.f;
#pragma unroll 4
  for (int m = 0; m < M; m++) {
    const float4 q = __ldg(yp + m);
    float ym = b4[m * NE + e];
    ym += q.x;
    if (ntile > 1) ym += q.y;
    if (ntile > 2) ym += q.z;
    if (ntile > 3) ym += q.w;
    v += ym;
  }
  return (double)v / (double)M;
}

__global__ void k_energy(int n_mol, int n_atoms, const int32_t *mol_offsets, const int32_t *perm,
                         const uint8_t *elem, const float *ypart, const float *b4, int M, int ntile, double *part,
                         unsigned *ticket, double *E, DevStatus *st) {
  __shared__ double red[32];
  __shared__ int last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int S = gridDim.y, y = blockIdx.y;
  for (int mol = blockIdx.x; mol < n_mol; mol += gridDim.x) {
    const int a0 = max(mol_offsets[mol], 0), a1 = min(mol_offsets[mol + 1], n_atoms);
    const int per = (max(a1 - a0, 0) + S - 1) / S;
    const int s0 = a0 + y * per, s1 = min(a1, s0 + per);
    double acc = 0.0;
    for (int i = s0 + threadIdx.x; i < s1; i += blockDim.x) acc += atom_energy(i, perm, elem, ypart, b4, M, ntile);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < nwarp; q++) t += red[q];
      if (S == 1) {
        E[mol] = t;
        if (!isfinite(t)) post_status(st, FNN_E_NONFINITE, -(long long)(mol + 1));
        last = 0;
      } else {
        part[(size_t)mol * S + y] = t;
        __threadfence();
        last = atomicAdd(&ticket[mol], 1u) == (unsigned)(S - 1);
      }
    }
    __syncthreads();
    if (last && w == 0) {
      __threadfence();
      const volatile double *pv = part + (size_t)mol * S;
      double t = 0.0;
      for (int q = lane; q < S; q += 32) t += pv[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) {
        E[mol] = t;
        ticket[mol] = 0u;
        if (!isfinite(t)) post_status(st, FNN_E_NONFINITE, -(long long)(mol + 1));
      }
    }
    __syncthreads();
  }
}

fnn_status energy_reduce_rows(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, const float *ypart,
                              int ntile, double *E, cudaStream_t s) {
  const int NM = sys->n_mol;
  if (NM <= 0) return FNN_OK;
  // slices of about 256 atoms for large structures (a thread per atom or two, spread over SMs)
  const long long avg = sys->n_atoms / NM;
  int S = (int)((avg + 255) / 256);
  if (S < 1) S = 1;
  if (S > 256) S = 256;
  while (S > 1 && (size_t)NM * S > ctx->ws.rows) S--;
  const int blocks = NM < 8 * ctx->num_sms ? NM : 8 * ctx->num_sms;
  FNN_KERNEL(ctx, "energy_reduce", s);
  k_energy<<<dim3(blocks, S), 128, 0, s>>>(NM, sys->n_atoms, sys->mol_offsets, nl->perm, nl->elem, ypart, ctx->w.b4,
                                           ctx->w.M, ntile, ctx->ws.e_part, ctx->ws.e_ticket, E, ctx->status);
  return check_launch(ctx, "energy_reduce");
}

fnn_status energy_reduce(fnn_ctx *ctx, const fnn_system *sys, const fnn_nlist *nl, double *E, cudaStream_t s) {
  return energy_reduce_rows(ctx, sys, nl, ctx->ws.ypart, (H3 + BN - 1) / BN, E, s);
}

}  // namespace fnn
